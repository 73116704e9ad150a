// Term sweep: for each (sample x, group g) the sector test of the flip x' = x ^ m_g and, for the
// groups that keep x' in the (n_up, n_dn) sector, the grouped matrix-element sum
//     S_g(x) = sum_{k in g} c'_k (-1)^{popcount(x & z_k)}            (paper Eq. mtx_element)
// with c'_k = c_k (-i)^{r_k} folded in by the grouping pass.  A flip changes n_alpha spin-up
// bits; x' stays in the sector iff exactly half of them are occupied in x (same for spin down),
// which needs two popcounts per (sample, group).  Out-of-sector flips have f(x') = 0 under the
// Hamming-weight constraint (Section 4), so they contribute exactly zero and are skipped.
//
// Work decomposition: a CTA owns a tile of SWEEP_GT groups and a batch of SWEEP_SB samples.
// Pass 1 (count, one thread per group) writes for every sample its validity bitmap over the
// tile's groups and the number of valid groups per (sample, tile); an exclusive scan turns the
// counts into row offsets, so rows come out sample-major, tile-major, group-minor -- a
// deterministic layout independent of scheduling.  Pass 2 (emit, one warp per sample at a
// time) walks each sample's bitmap in group order, numbering the valid pairs as it goes, and
// sums their terms from a shared-memory copy of the tile's terms.
//
// A sample outside the (n_up, n_dn) sector gets exactly one row, x' = x with S = NaN, in its
// first group tile and no other: the rows stay within the per-sample bound of the feasible
// groups, and every local-energy reduction over that sample's rows returns NaN.
#include "nqs_internal.h"

namespace nqs {
namespace {

constexpr int SWEEP_NW = SWEEP_GT / 32;
constexpr long long SWEEP_WAIT_CYCLES = 2ll * 1000 * 1000 * 1000;   // ~1 s at the boost clock

// The two spin species' bits of a 64-bit word packed into one 32-bit word each: the even
// (spin-up) bits of the high half move to the odd positions of the low half, and the odd
// (spin-down) bits to the even positions, so one POPC counts a species over all 64 qubits.
__device__ __forceinline__ uint32_t up_bits(uint64_t v) {
    return ((uint32_t)v & 0x55555555u) | (((uint32_t)(v >> 32) & 0x55555555u) << 1);
}
__device__ __forceinline__ uint32_t dn_bits(uint64_t v) {
    return ((uint32_t)v & 0xAAAAAAAAu) | (((uint32_t)(v >> 32) & 0xAAAAAAAAu) >> 1);
}

// Species words of a configuration: {up, dn} for one word, {up of word 0, up of word 1, dn of
// word 0, dn of word 1} for two words.
struct Sp1 {
    uint32_t u, d;
};
struct Sp2 {
    uint32_t u0, u1, d0, d1;
};
__device__ __forceinline__ Sp1 species(uint64_t v) { return Sp1{up_bits(v), dn_bits(v)}; }
__device__ __forceinline__ Sp2 species(const U128& v) {
    return Sp2{up_bits(v.lo), up_bits(v.hi), dn_bits(v.lo), dn_bits(v.hi)};
}
template <class BT> struct SpOf { using type = Sp1; };
template <> struct SpOf<U128> { using type = Sp2; };

__device__ __forceinline__ int pop_up(const Sp1& a, const Sp1& b) { return __popc(a.u & b.u); }
__device__ __forceinline__ int pop_dn(const Sp1& a, const Sp1& b) { return __popc(a.d & b.d); }
__device__ __forceinline__ int pop_up(const Sp2& a, const Sp2& b) { return __popc(a.u0 & b.u0) + __popc(a.u1 & b.u1); }
__device__ __forceinline__ int pop_dn(const Sp2& a, const Sp2& b) { return __popc(a.d0 & b.d0) + __popc(a.d1 & b.d1); }
__device__ __forceinline__ int cnt_up(const Sp1& a) { return __popc(a.u); }
__device__ __forceinline__ int cnt_dn(const Sp1& a) { return __popc(a.d); }
__device__ __forceinline__ int cnt_up(const Sp2& a) { return __popc(a.u0) + __popc(a.u1); }
__device__ __forceinline__ int cnt_dn(const Sp2& a) { return __popc(a.d0) + __popc(a.d1); }

template <class BT>
__device__ __forceinline__ bool sample_in_sector(const BT& x, int n_up, int n_dn) {
    const auto sp = species(x);
    return cnt_up(sp) == n_up && cnt_dn(sp) == n_dn;
}

// Parity of popcount(x & z) in bit 31 (the float sign bit), x and z given as their 32-bit
// halves: the halves of x & z are XOR-folded first, which keeps the parity, so one 32-bit POPC
// serves a 64-bit mask.
__device__ __forceinline__ uint32_t sign_flip(uint32_t xl, uint32_t xh, uint32_t zl, uint32_t zh) {
    return (uint32_t)__popc((xl & zl) ^ (xh & zh)) << 31;
}

// (-1)^{popcount(x & z)} as the float sign bit (bit 31)
__device__ __forceinline__ uint32_t parity_bit(uint64_t x, uint64_t z) {
    return sign_flip((uint32_t)x, (uint32_t)(x >> 32), (uint32_t)z, (uint32_t)(z >> 32));
}
__device__ __forceinline__ uint32_t parity_bit(const U128& x, const U128& z) {
    const U128 v = x & z;
    return (uint32_t)__popc((uint32_t)v.lo ^ (uint32_t)(v.lo >> 32) ^ (uint32_t)v.hi ^ (uint32_t)(v.hi >> 32)) << 31;
}

// uint4 per term record: one for one-word masks, two for two-word masks
template <class BT> __host__ __device__ constexpr int rec_of() { return (int)(sizeof(BT) / 8); }

// Knuth's TwoSum: s + e == a + b exactly, accumulated into the error term.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
}

// One term of S_g(x): c' (-1)^{popc(x & z)} into the real or (odd sigma_2 count) imaginary sum.
// Term k is its record at tp (see HamDev::term).  IMAG: the Hamiltonian has odd-sigma_2 terms
// somewhere (else the imaginary branch is compiled out).
template <bool COMP>
__device__ __forceinline__ void acc_term(bool imag, float hi, float lo, float& re, float& re_e, float& im,
                                         float& im_e) {
    if (COMP) {
        if (imag) { two_sum_acc(im, im_e, hi); im_e += lo; }
        else      { two_sum_acc(re, re_e, hi); re_e += lo; }
    } else {
        if (imag) im += hi; else re += hi;
    }
}

template <bool COMP, bool IMAG>
__device__ __forceinline__ void add_term(uint64_t x, uint64_t mg, bool has_imag, const uint4* tp, uint32_t k,
                                         float& re, float& re_e, float& im, float& im_e) {
    const uint4 t = tp[k];
    const uint32_t flip = sign_flip((uint32_t)x, (uint32_t)(x >> 32), t.x, t.y);
    const bool imag = IMAG && has_imag && (__popc(((uint32_t)mg & t.x) ^ ((uint32_t)(mg >> 32) & t.y)) & 1);
    acc_term<COMP>(imag, __uint_as_float(t.z ^ flip), __uint_as_float(t.w ^ flip), re, re_e, im, im_e);
}

template <bool COMP, bool IMAG>
__device__ __forceinline__ void add_term(const U128& x, const U128& mg, bool has_imag, const uint4* tp, uint32_t k,
                                         float& re, float& re_e, float& im, float& im_e) {
    const uint4 z = tp[2 * k], c = tp[2 * k + 1];
    const uint32_t v = ((uint32_t)x.lo & z.x) ^ ((uint32_t)(x.lo >> 32) & z.y) ^ ((uint32_t)x.hi & z.z) ^
                       ((uint32_t)(x.hi >> 32) & z.w);
    const uint32_t flip = (uint32_t)__popc(v) << 31;
    bool imag = false;
    if (IMAG && has_imag) {
        const uint32_t u = ((uint32_t)mg.lo & z.x) ^ ((uint32_t)(mg.lo >> 32) & z.y) ^ ((uint32_t)mg.hi & z.z) ^
                           ((uint32_t)(mg.hi >> 32) & z.w);
        imag = __popc(u) & 1;
    }
    acc_term<COMP>(imag, __uint_as_float(c.x ^ flip), __uint_as_float(c.y ^ flip), re, re_e, im, im_e);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}

// Bounded wait on the staging barrier; false after the clock budget.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > SWEEP_WAIT_CYCLES) return false;
    return true;
}

// Count pass: the sector test of every (sample, group) pair of a tile of SWEEP_GT groups and a
// batch of SWEEP_SB samples (thread = group, the batch's samples in shared memory as their
// spin-up and spin-down bit words, the group's flip mask split the same way once).  Each warp's
// ballot of sample s is the validity word of s over the warp's 32 groups; lane s keeps it, so
// the pass writes the tile's validity bitmap per sample, stored [batch][tile][warp][sample],
// and the number of valid groups per (sample, tile).
template <class BT>
__global__ void __launch_bounds__(SWEEP_GT)
sweep_count_kernel(HamDev h, int n_up, int n_dn, const BT* __restrict__ bits,
                   int64_t B, int32_t* __restrict__ cnt, int64_t ntiles, uint32_t* __restrict__ valid) {
    using Sp = typename SpOf<BT>::type;
    __shared__ Sp xs[SWEEP_SB];
    __shared__ int32_t wcnt[SWEEP_NW][SWEEP_SB];
    __shared__ uint32_t okm;              // in-sector samples of the batch
    const int tile = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * SWEEP_SB;
    const int nb = (int)(B - s0 < SWEEP_SB ? B - s0 : SWEEP_SB);
    const int64_t g = (int64_t)tile * SWEEP_GT + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool live = g < h.G;
    const BT m = live ? reinterpret_cast<const BT*>(h.grp_mask)[g] : bits_zero<BT>();
    const uint32_t meta = live ? h.grp_meta[g] : 0;
    const Sp ms = species(m);
    // the occupied flipped bits each species needs: half its flipped bits (an odd count, or a
    // group past the end, can never match: 1024 is out of range)
    const uint32_t na = meta & 0xffu, nbt = (meta >> 8) & 0xffu;
    const int ta = (!live || (na & 1u)) ? 1024 : (int)(na >> 1), tb = (nbt & 1u) ? 1024 : (int)(nbt >> 1);
    if (threadIdx.x < SWEEP_SB) {
        const BT x = threadIdx.x < nb ? bits[s0 + threadIdx.x] : bits_zero<BT>();
        xs[threadIdx.x] = species(x);
        const bool ok = threadIdx.x < nb && sample_in_sector(x, n_up, n_dn);
        const unsigned bb = __ballot_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) okm = bb;
    }
    __syncthreads();
    uint32_t mine = 0;
#pragma unroll
    for (int s = 0; s < SWEEP_SB; ++s) {
        const Sp xv = xs[s];
        const bool v = pop_up(xv, ms) == ta && pop_dn(xv, ms) == tb;
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == s) mine = bal;
    }
    if (!((okm >> lane) & 1u)) mine = 0;       // samples past the batch or outside the sector
    valid[(((int64_t)blockIdx.x * ntiles + tile) * SWEEP_NW + warp) * SWEEP_SB + lane] = mine;
    wcnt[warp][lane] = __popc(mine);
    __syncthreads();
    if (threadIdx.x < nb) {
        int32_t c = 0;
#pragma unroll
        for (int w = 0; w < SWEEP_NW; ++w) c += wcnt[w][threadIdx.x];
        // out-of-sector sample: one NaN row in tile 0
        if (!((okm >> threadIdx.x) & 1u)) c = tile == 0 ? 1 : 0;
        cnt[(s0 + threadIdx.x) * ntiles + tile] = c;
    }
}

// Emit pass.  A CTA takes one tile of SWEEP_GT groups and the SWEEP_SB samples of a count
// batch, with the batch's validity bitmaps.  The tile's terms (z masks and coefficients,
// contiguous in the grouped table) are copied once into shared memory by a bulk asynchronous
// copy (cp.async.bulk, completion on an mbarrier) and serve every sample of the batch.  Warp w
// takes group word w of the tile (32 groups) for all the batch's samples: lane s holds sample
// s's validity bits over the word and counts its valid groups in the words before, so the row of
// each valid pair (its rank among the sample's valid groups of the tile) is that count plus a
// popcount -- the deterministic row order sample-major, tile-major, group-minor.  The pairs of
// small groups (at most SWEEP_SMALL terms: the double excitations) are numbered by a warp scan
// of the per-sample counts and summed 32 at a time, one lane per pair (tabulated groups by one
// table entry); the few large groups (the diagonal and the single excitations) are summed by the
// whole warp at once, lanes over terms with a TwoSum butterfly.
template <bool COMP, bool IMAG, class BT>
__device__ __forceinline__ void sweep_pair_sum(const BT& x, const BT& mg, bool has_imag, const uint4* tp,
                                               uint32_t a0, uint32_t a1, uint32_t step, float& re,
                                               float& re_e, float& im, float& im_e) {
    for (uint32_t k = a0; k < a1; k += step) add_term<COMP, IMAG>(x, mg, has_imag, tp, k, re, re_e, im, im_e);
}

template <bool COMP, bool IMAG, class BT>
__global__ void __launch_bounds__(SWEEP_GT)
sweep_emit_kernel(HamDev h, int n_up, int n_dn, const BT* __restrict__ bits, int64_t B,
                  const int64_t* __restrict__ off, int64_t ntiles, const uint32_t* __restrict__ valid,
                  BT* __restrict__ xprime, float4* __restrict__ S, int* __restrict__ status) {
    constexpr int REC = rec_of<BT>();                   // uint4 per term record
    constexpr uint32_t STAGE = SWEEP_STAGE;             // terms that fit the staging buffer
    extern __shared__ __align__(128) unsigned char sweep_smem[];
    uint4* ts = reinterpret_cast<uint4*>(sweep_smem);                         // staged term records
    __shared__ BT xs[SWEEP_SB];
    __shared__ int64_t obase[SWEEP_SB];
    __shared__ uint32_t vb[SWEEP_NW * SWEEP_SB];       // validity words [warp][sample]
    __shared__ uint32_t lmask[SWEEP_NW];               // large groups of each group word
    __shared__ __align__(8) uint64_t bar;
    __shared__ BT g_mask[SWEEP_GT];                    // the tile's groups: flip mask, meta, term range
    __shared__ uint32_t g_meta[SWEEP_GT], g_k0[SWEEP_GT], g_k1[SWEEP_GT];
    __shared__ int32_t g_tab[SWEEP_GT];                // tabulated groups: table, flipped qubits, common z
    __shared__ uint32_t g_pos[SWEEP_GT];
    __shared__ BT g_zc[SWEEP_GT];

    const int tile = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * SWEEP_SB;
    const int nb = (int)(B - s0 < SWEEP_SB ? B - s0 : SWEEP_SB);
    const int64_t g0 = (int64_t)tile * SWEEP_GT;
    const int64_t g = g0 + threadIdx.x;
    const bool live = g < h.G;
    const int64_t g_end = g0 + SWEEP_GT < h.G ? g0 + SWEEP_GT : h.G;
    // the tile's term range (16- or 32-byte records: every range is a valid bulk copy)
    const uint32_t t0 = h.grp_off[g0];
    const uint32_t t1 = h.grp_off[g_end];
    const bool staged = t1 - t0 <= STAGE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0 && staged) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const uint32_t bytes = (t1 - t0) * 16u * REC;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(smem_u32(&bar)), "r"(bytes) : "memory");
        if (bytes)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(ts)), "l"(h.term + (size_t)t0 * REC), "r"(bytes), "r"(smem_u32(&bar))
                         : "memory");
    }
    const uint32_t k0 = live ? h.grp_off[g] : 0, k1 = live ? h.grp_off[g + 1] : 0;
    g_mask[threadIdx.x] = live ? reinterpret_cast<const BT*>(h.grp_mask)[g] : bits_zero<BT>();
    g_meta[threadIdx.x] = live ? h.grp_meta[g] : 0;
    g_tab[threadIdx.x] = live ? h.grp_tab[g] : -1;
    g_pos[threadIdx.x] = live ? h.grp_pos[g] : 0u;
    g_zc[threadIdx.x] = live ? reinterpret_cast<const BT*>(h.grp_zc)[g] : bits_zero<BT>();
    g_k0[threadIdx.x] = k0 - t0;                       // term indices relative to the tile's range
    g_k1[threadIdx.x] = k1 - t0;
    const unsigned lg = __ballot_sync(0xffffffffu, live && k1 - k0 > (uint32_t)SWEEP_SMALL);
    if (lane == 0) lmask[warp] = lg;
    vb[threadIdx.x] = valid[((int64_t)blockIdx.x * ntiles + tile) * SWEEP_GT + threadIdx.x];
    if (threadIdx.x < nb) {
        xs[threadIdx.x] = bits[s0 + threadIdx.x];
        obase[threadIdx.x] = off[(s0 + threadIdx.x) * ntiles + tile];
        // an out-of-sector sample gets its single NaN row here
        if (tile == 0 && !sample_in_sector(xs[threadIdx.x], n_up, n_dn)) {
            xprime[obase[threadIdx.x]] = xs[threadIdx.x];
            S[obase[threadIdx.x]] = make_float4(__int_as_float(0x7fc00000), 0.f, __int_as_float(0x7fc00000), 0.f);
        }
    }
    __syncthreads();
    if (staged && !mbar_wait_bounded(&bar, 0)) {
        // the staging copy did not complete in time: report it, wait (bounded) once more so no
        // copy is left writing into this CTA's shared memory, and leave the tile's rows unwritten
        atomicExch(status, 2);
        mbar_wait_bounded(&bar, 0);
        return;
    }
    const uint4* tp = staged ? ts : h.term + (size_t)t0 * REC;
    // Warp w owns the tile's group word w (groups 32 w .. 32 w + 31) for all nb samples; lane s
    // holds sample s's validity bits over the word and its valid groups in the words before w,
    // so the row of pair (s, g) is obase[s] + pre_s + (valid groups of s below g in the word).
    const uint32_t lm = lmask[warp];
    uint32_t bal = 0u;
    int pre = 0;
    if (lane < nb) {
        bal = vb[warp * SWEEP_SB + lane];
        for (int j = 0; j < warp; ++j) pre += __popc(vb[j * SWEEP_SB + lane]);
    }
    // small groups: the warp's pairs numbered by an exclusive scan of the per-sample counts and
    // handed out 32 at a time, one per lane
    const uint32_t smask = bal & ~lm;
    const int cnt = __popc(smask);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int excl = incl - cnt;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        // the pair's sample: the last lane whose first pair number is <= p
        int s = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int cand = s + step;
            const int e = __shfl_sync(0xffffffffu, excl, cand & 31);
            if (cand < 32 && e <= p) s = cand;
        }
        const int es = __shfl_sync(0xffffffffu, excl, s);
        const uint32_t ms = __shfl_sync(0xffffffffu, smask, s);
        const uint32_t bs = __shfl_sync(0xffffffffu, bal, s);
        const int ps = __shfl_sync(0xffffffffu, pre, s);
        uint32_t v = ms;                                      // the (p - es)-th valid small group
        for (int i = es; i < p && v; ++i) v &= v - 1u;
        if (p < total && v) {
            const int bpos = __ffs(v) - 1;
            const int gl = 32 * warp + bpos;
            const BT x = xs[s], mg = g_mask[gl];
            float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
            const int tb = g_tab[gl];
            if (tb >= 0) {
                // tabulated group: common parity times the table entry of x's flipped bits
                const uint32_t pk = g_pos[gl], meta = g_meta[gl];
                const int nbits = (int)((meta & 0xffu) + ((meta >> 8) & 0xffu));
                int idx = 0;
                for (int i = 0; i < nbits; ++i) idx |= qbit(x, (int)((pk >> (8 * i)) & 0xffu)) << i;
                const uint32_t flip = parity_bit(x, g_zc[gl]);
                const float2 t = __ldg(h.tab + (int64_t)tb * SWEEP_TAB_SIZE + idx);
                re = __uint_as_float(__float_as_uint(t.x) ^ flip);
                re_e = COMP ? __uint_as_float(__float_as_uint(t.y) ^ flip) : 0.f;
            } else {
                sweep_pair_sum<COMP, IMAG>(x, mg, (g_meta[gl] & META_HAS_IMAG) != 0, tp, g_k0[gl], g_k1[gl], 1u, re,
                                           re_e, im, im_e);
            }
            const int64_t row = obase[s] + ps + __popc(bs & ((1u << bpos) - 1u));
            xprime[row] = x ^ mg;
            S[row] = make_float4(re, re_e, im, im_e);
        }
    }
    // large groups (the diagonal and the single excitations): the whole warp per pair, lanes over
    // terms, TwoSum butterfly
    const uint32_t lgm = bal & lm;
    for (unsigned who = __ballot_sync(0xffffffffu, lgm != 0u); who; who &= who - 1u) {
        const int s = __ffs(who) - 1;
        const uint32_t ls = __shfl_sync(0xffffffffu, lgm, s);
        const uint32_t bs = __shfl_sync(0xffffffffu, bal, s);
        const int ps = __shfl_sync(0xffffffffu, pre, s);
        const BT x = xs[s];
        for (uint32_t big = ls; big; big &= big - 1u) {
            const int bpos = __ffs(big) - 1, gl = 32 * warp + bpos;
            const BT mg = g_mask[gl];
            float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
            sweep_pair_sum<COMP, IMAG>(x, mg, (g_meta[gl] & META_HAS_IMAG) != 0, tp, g_k0[gl] + lane, g_k1[gl],
                                       32u, re, re_e, im, im_e);
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) {
                // (the imaginary sums are zero unless the Hamiltonian has odd-sigma_2 terms, the
                // error terms unless the sums are compensated: neither is exchanged then)
                const float ore = __shfl_xor_sync(0xffffffffu, re, d);
                const float oree = COMP ? __shfl_xor_sync(0xffffffffu, re_e, d) : 0.f;
                const float oim = IMAG ? __shfl_xor_sync(0xffffffffu, im, d) : 0.f;
                const float oime = (IMAG && COMP) ? __shfl_xor_sync(0xffffffffu, im_e, d) : 0.f;
                // both lanes form the same pair sum: order the operands by lane
                const bool low = (lane & d) == 0;
                if (COMP) {
                    float a = low ? re : ore, bb = low ? ore : re;
                    float ae = (low ? re_e : oree) + (low ? oree : re_e);
                    two_sum_acc(a, ae, bb);
                    re = a; re_e = ae;
                    if (IMAG) {
                        float c2 = low ? im : oim, d2 = low ? oim : im;
                        float ce = (low ? im_e : oime) + (low ? oime : im_e);
                        two_sum_acc(c2, ce, d2);
                        im = c2; im_e = ce;
                    }
                } else {
                    re = low ? re + ore : ore + re;
                    if (IMAG) im = low ? im + oim : oim + im;
                }
            }
            if (lane == 0) {
                const int64_t row = obase[s] + ps + __popc(bs & ((1u << bpos) - 1u));
                xprime[row] = x ^ mg;
                S[row] = make_float4(re, re_e, im, im_e);
            }
        }
    }
}

__global__ void unpack_rows_kernel(const int64_t* __restrict__ off, int64_t ntiles, int64_t B,
                                   const float4* __restrict__ S, int64_t* __restrict__ row_offset,
                                   float* __restrict__ s_re, float* __restrict__ s_im,
                                   const int64_t* __restrict__ total) {
    const int64_t n = *total;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < max(n, B + 1);
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i <= B) row_offset[i] = i == B ? n : off[i * ntiles];
        if (i < n) {
            const float4 v = S[i];
            s_re[i] = v.x + v.y;
            s_im[i] = v.z + v.w;
        }
    }
}

}  // namespace

int64_t sweep_tiles(const HamDev& h) { return (h.G + SWEEP_GT - 1) / SWEEP_GT; }



int64_t sweep_valid_words(const HamDev& h, int64_t B) {
    return std::max<int64_t>(1, (B + SWEEP_SB - 1) / SWEEP_SB) * sweep_tiles(h) * SWEEP_GT;
}

// Bits of one configuration: `words` uint64 (HamDev::words); the kernels take them as uint64_t
// or U128.
int launch_sweep_count(const HamDev& h, int n_up, int n_dn, const uint64_t* bits,
                       int64_t B, int32_t* cnt, uint32_t* valid, cudaStream_t s) {
    if (B <= 0) return NQS_OK;
    const int64_t T = sweep_tiles(h);
    dim3 grid((unsigned)((B + SWEEP_SB - 1) / SWEEP_SB), (unsigned)T);
    if (h.words == 2)
        sweep_count_kernel<U128><<<grid, SWEEP_GT, 0, s>>>(h, n_up, n_dn, reinterpret_cast<const U128*>(bits), B, cnt, T,
                                                           valid);
    else
        sweep_count_kernel<uint64_t><<<grid, SWEEP_GT, 0, s>>>(h, n_up, n_dn, bits, B, cnt, T, valid);
    NQS_LAUNCHED();
    return NQS_OK;
}

template <class BT>
static int sweep_emit_as(const HamDev& h, int n_up, int n_dn, int compensated, const uint64_t* bits, int64_t B,
                         const int64_t* off, const uint32_t* valid, uint64_t* xprime, float4* S, cudaStream_t s) {
    const int64_t T = sweep_tiles(h);
    dim3 grid((unsigned)((B + SWEEP_SB - 1) / SWEEP_SB), (unsigned)T);
    constexpr size_t smem = (size_t)SWEEP_STAGE * 16 * rec_of<BT>();   // 32 KB (one word) or 64 KB (two)
    static int attr_dev = -1;
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        NQS_CK(cudaFuncSetAttribute(sweep_emit_kernel<true, false, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NQS_CK(cudaFuncSetAttribute(sweep_emit_kernel<false, false, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NQS_CK(cudaFuncSetAttribute(sweep_emit_kernel<true, true, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NQS_CK(cudaFuncSetAttribute(sweep_emit_kernel<false, true, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_dev = dev;
    }
    int* status = nullptr;
    NQS_TRY(device_status_ptr(&status));
    const BT* b = reinterpret_cast<const BT*>(bits);
    BT* xp = reinterpret_cast<BT*>(xprime);
    auto go = [&](auto kernel) { kernel<<<grid, SWEEP_GT, smem, s>>>(h, n_up, n_dn, b, B, off, T, valid, xp, S, status); };
    if (h.any_imag) {
        if (compensated) go(sweep_emit_kernel<true, true, BT>); else go(sweep_emit_kernel<false, true, BT>);
    } else {
        if (compensated) go(sweep_emit_kernel<true, false, BT>); else go(sweep_emit_kernel<false, false, BT>);
    }
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_sweep_emit(const HamDev& h, int n_up, int n_dn, int compensated,
                      const uint64_t* bits, int64_t B, const int64_t* off, const uint32_t* valid,
                      uint64_t* xprime, float4* S, cudaStream_t s) {
    if (B <= 0) return NQS_OK;
    if (h.words == 2) return sweep_emit_as<U128>(h, n_up, n_dn, compensated, bits, B, off, valid, xprime, S, s);
    return sweep_emit_as<uint64_t>(h, n_up, n_dn, compensated, bits, B, off, valid, xprime, S, s);
}

int launch_unpack_rows(const int64_t* off, int64_t ntiles, int64_t B, const float4* S,
                       int64_t* row_offset, float* s_re, float* s_im, int64_t rows_cap,
                       const int64_t* total, cudaStream_t s) {
    const int64_t work = std::max<int64_t>(rows_cap, B + 1);
    const int grid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)num_sms() * 8);
    unpack_rows_kernel<<<grid, 256, 0, s>>>(off, ntiles, B, S, row_offset, s_re, s_im, total);
    NQS_LAUNCHED();
    return NQS_OK;
}

}  // namespace nqs
