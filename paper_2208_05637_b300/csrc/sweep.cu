// Term sweep: for each (sample x, group g) the sector test of the flip x' = x ^ m_g and, for the
// groups that keep x' in the (n_up, n_dn) sector, the grouped matrix-element sum
//     S_g(x) = sum_{k in g} c'_k (-1)^{popcount(x & z_k)}            (paper Eq. mtx_element)
// with c'_k = c_k (-i)^{r_k} folded in by the grouping pass.  A flip changes n_alpha spin-up
// bits; x' stays in the sector iff exactly half of them are occupied in x (same for spin down),
// which needs two popcounts per (sample, group).  Out-of-sector flips have f(x') = 0 under the
// Hamming-weight constraint (Section 4), so they contribute exactly zero and are skipped.
//
// Work decomposition: a CTA owns a tile of SWEEP_GT groups (one thread per group) and a batch
// of SWEEP_SB samples held in shared memory.  Pass 1 (count) writes the number of valid
// groups per (sample, tile); an exclusive scan turns these into row offsets, so rows come out
// sample-major, tile-major, group-minor -- a deterministic layout independent of scheduling.
// Pass 2 (emit) compacts the valid (sample, group) pairs of the batch into shared memory with
// warp ballots and lets every thread take pairs from that list, so no lane idles on an
// invalid group while its neighbours sum terms.
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

// x' = x ^ m stays in the sector iff exactly half of the flipped bits of each species are
// occupied in x: 2 popc(x & m & A) == n_alpha(m) and the same for spin down.
__device__ __forceinline__ bool sector_ok(uint64_t x, uint64_t m, uint32_t meta) {
    const uint64_t v = x & m;
    return 2u * (uint32_t)__popc(up_bits(v)) == (meta & 0xffu) &&
           2u * (uint32_t)__popc(dn_bits(v)) == ((meta >> 8) & 0xffu);
}

__device__ __forceinline__ bool sample_in_sector(uint64_t x, int n_up, int n_dn) {
    return __popc(up_bits(x)) == n_up && __popc(dn_bits(x)) == n_dn;
}

// Parity of popcount(x & z) in bit 31 (the float sign bit): the two halves are XOR-folded first,
// which keeps the parity, so one 32-bit POPC serves a 64-bit mask.
__device__ __forceinline__ uint32_t sign_flip(uint64_t x, uint64_t z) {
    const uint64_t v = x & z;
    return (uint32_t)__popc((uint32_t)v ^ (uint32_t)(v >> 32)) << 31;
}

// Knuth's TwoSum: s + e == a + b exactly, accumulated into the error term.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
}

// One term of S_g(x): c' (-1)^{popc(x & z)} into the real or (odd sigma_2 count) imaginary sum.
template <bool COMP>
__device__ __forceinline__ void add_term(uint64_t x, uint64_t mg, bool has_imag, uint64_t z, float2 c,
                                         float& re, float& re_e, float& im, float& im_e) {
    const uint32_t flip = sign_flip(x, z);
    const float hi = __uint_as_float(__float_as_uint(c.x) ^ flip);
    const float lo = __uint_as_float(__float_as_uint(c.y) ^ flip);
    const bool imag = has_imag && (__popcll(mg & z) & 1);
    if (COMP) {
        if (imag) { two_sum_acc(im, im_e, hi); im_e += lo; }
        else      { two_sum_acc(re, re_e, hi); re_e += lo; }
    } else {
        if (imag) im += hi; else re += hi;
    }
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
// batch of SWEEP_SB samples.  Writes the number of valid groups per (sample, tile) and, for the
// emit pass, each group's validity bits over the batch (one word per group and batch).
__global__ void __launch_bounds__(SWEEP_GT)
sweep_count_kernel(HamDev h, int n_up, int n_dn, const uint64_t* __restrict__ bits,
                   int64_t B, int32_t* __restrict__ cnt, int64_t ntiles, uint32_t* __restrict__ valid) {
    __shared__ uint64_t xs[SWEEP_SB];
    __shared__ int32_t wcnt[SWEEP_SB][SWEEP_NW];
    __shared__ uint32_t oos;              // out-of-sector samples of the batch
    const int tile = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * SWEEP_SB;
    const int nb = (int)(B - s0 < SWEEP_SB ? B - s0 : SWEEP_SB);
    const int64_t g = (int64_t)tile * SWEEP_GT + threadIdx.x;
    const bool live = g < h.G;
    const uint64_t m = live ? h.grp_mask[g] : 0;
    const uint32_t meta = live ? h.grp_meta[g] : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < nb) xs[threadIdx.x] = bits[s0 + threadIdx.x];
    if (warp == 0) {
        const bool bad = lane < nb && !sample_in_sector(bits[s0 + min(lane, nb - 1)], n_up, n_dn);
        const unsigned bb = __ballot_sync(0xffffffffu, bad);
        if (lane == 0) oos = bb;
    }
    __syncthreads();
    uint32_t vmask = 0;
    for (int s = 0; s < nb; ++s) {
        const bool v = live && sector_ok(xs[s], m, meta) && !((oos >> s) & 1u);
        vmask |= (uint32_t)v << s;
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == 0) wcnt[s][warp] = __popc(bal);
    }
    valid[(int64_t)blockIdx.x * ntiles * SWEEP_GT + g] = vmask;
    __syncthreads();
    if (threadIdx.x < nb) {
        int32_t c = 0;
#pragma unroll
        for (int w = 0; w < SWEEP_NW; ++w) c += wcnt[threadIdx.x][w];
        // out-of-sector sample: one NaN row in tile 0
        if ((oos >> threadIdx.x) & 1u) c = tile == 0 ? 1 : 0;
        cnt[(s0 + threadIdx.x) * ntiles + tile] = c;
    }
}

// Emit pass.  A CTA takes one tile of SWEEP_GT groups and the SWEEP_SB samples of a count
// batch, whose validity words it reads back.  The tile's terms (z masks and coefficients,
// contiguous in the grouped table) are copied once into shared memory by a bulk asynchronous
// copy (cp.async.bulk, completion on an mbarrier) while the pairs are numbered, and then serve
// every sample of the batch.  The valid
// (sample, group) pairs are numbered in the deterministic row order (sample-major, group order)
// and split by group size: groups of more than SWEEP_SMALL terms (the diagonal and the
// single-excitation groups) are summed by a whole warp, lanes over terms with a TwoSum warp
// reduction; the others by one thread each, taken in 32-pair chunks from a shared counter so
// the warps stay busy until the tile's work is gone.
template <bool COMP>
__global__ void __launch_bounds__(SWEEP_GT)
sweep_emit_kernel(HamDev h, int n_up, int n_dn, const uint64_t* __restrict__ bits, int64_t B,
                  const int64_t* __restrict__ off, int64_t ntiles, const uint32_t* __restrict__ valid,
                  uint64_t* __restrict__ xprime, float4* __restrict__ S, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char sweep_smem[];
    uint64_t* zs = reinterpret_cast<uint64_t*>(sweep_smem);                   // staged z masks
    float2* cs = reinterpret_cast<float2*>(sweep_smem + 8 * SWEEP_STAGE);     // staged coefficients
    __shared__ uint64_t xs[SWEEP_SB];
    __shared__ int64_t obase[SWEEP_SB];
    __shared__ int32_t woff[SWEEP_SB * SWEEP_NW + 1];
    __shared__ int32_t sstart[SWEEP_SB + 1];
    __shared__ uint32_t plist[SWEEP_SB * SWEEP_GT];    // small pairs from the front, large from the back
    __shared__ int32_t n_small, n_large, next_small;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint64_t g_mask[SWEEP_GT];                  // the tile's groups: flip mask, meta, term range
    __shared__ uint32_t g_meta[SWEEP_GT], g_k0[SWEEP_GT], g_k1[SWEEP_GT];

    const int tile = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * SWEEP_SB;
    const int nb = (int)(B - s0 < SWEEP_SB ? B - s0 : SWEEP_SB);
    const int64_t g0 = (int64_t)tile * SWEEP_GT;
    const int64_t g = g0 + threadIdx.x;
    const bool live = g < h.G;
    const int64_t g_end = g0 + SWEEP_GT < h.G ? g0 + SWEEP_GT : h.G;
    // the tile's term range, widened to even indices (16-byte boundaries of both arrays; the
    // tables carry one padding term)
    const uint32_t t0 = h.grp_off[g0] & ~1u;
    const uint32_t t1 = (h.grp_off[g_end] + 1u) & ~1u;
    const bool staged = t1 - t0 <= (uint32_t)SWEEP_STAGE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        n_small = 0; n_large = 0; next_small = 0;
        if (staged) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            const uint32_t bytes = (t1 - t0) * 8u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(smem_u32(&bar)), "r"(2u * bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(zs)), "l"(h.term_z + t0), "r"(bytes), "r"(smem_u32(&bar)) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(cs)), "l"(h.term_c + t0), "r"(bytes), "r"(smem_u32(&bar)) : "memory");
        }
    }
    const uint32_t k0 = live ? h.grp_off[g] : 0, k1 = live ? h.grp_off[g + 1] : 0;
    const bool large = k1 - k0 > (uint32_t)SWEEP_SMALL;
    g_mask[threadIdx.x] = live ? h.grp_mask[g] : 0;
    g_meta[threadIdx.x] = live ? h.grp_meta[g] : 0;
    g_k0[threadIdx.x] = k0;
    g_k1[threadIdx.x] = k1;
    if (threadIdx.x < nb) {
        xs[threadIdx.x] = bits[s0 + threadIdx.x];
        obase[threadIdx.x] = off[(s0 + threadIdx.x) * ntiles + tile];
    }
    __syncthreads();

    // validity bits of this thread's group over the batch (the count pass's); an out-of-sector
    // sample gets its single NaN row here
    const uint32_t vmask = valid[(int64_t)blockIdx.x * ntiles * SWEEP_GT + g];
    if (tile == 0 && threadIdx.x < nb && !sample_in_sector(xs[threadIdx.x], n_up, n_dn)) {
        xprime[obase[threadIdx.x]] = xs[threadIdx.x];
        S[obase[threadIdx.x]] = make_float4(__int_as_float(0x7fc00000), 0.f, __int_as_float(0x7fc00000), 0.f);
    }
    for (int s = 0; s < SWEEP_SB; ++s) {
        const unsigned bal = __ballot_sync(0xffffffffu, (vmask >> s) & 1u);
        if (lane == 0) woff[s * SWEEP_NW + warp] = __popc(bal);
    }
    __syncthreads();
    // exclusive scan of the EB*NW warp counts (sample-major, warp-minor) by one warp
    if (warp == 0) {
        constexpr int PER = (SWEEP_SB * SWEEP_NW + 31) / 32;
        int32_t loc[PER];
        int32_t run = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = lane * PER + i;
            loc[i] = idx < SWEEP_SB * SWEEP_NW ? woff[idx] : 0;
            run += loc[i];
        }
        int32_t incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        int32_t excl = incl - run;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = lane * PER + i;
            if (idx < SWEEP_SB * SWEEP_NW) woff[idx] = excl;
            excl += loc[i];
        }
        if (lane == 31) woff[SWEEP_SB * SWEEP_NW] = incl;
    }
    __syncthreads();
    // number the pairs and file them by group size: entry = p | s << 13 | group << 18
    const unsigned lt = (1u << lane) - 1u;
    const unsigned lbal = __ballot_sync(0xffffffffu, large && vmask != 0);
    const unsigned sbal = __ballot_sync(0xffffffffu, !large && vmask != 0);
    const int npairs = __popc(vmask);
    int base_l = 0, base_s = 0;
    {
        // per-warp reservation of list slots (one atomic per warp and list)
        int tot_l = 0, tot_s = 0;
        const int mine = npairs;
        int pl = 0, ps = 0;
        const int ml = (lbal >> lane) & 1u ? mine : 0, ms = (sbal >> lane) & 1u ? mine : 0;
        pl = ml; ps = ms;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int yl = __shfl_up_sync(0xffffffffu, pl, d);
            const int ys = __shfl_up_sync(0xffffffffu, ps, d);
            if (lane >= d) { pl += yl; ps += ys; }
        }
        tot_l = __shfl_sync(0xffffffffu, pl, 31);
        tot_s = __shfl_sync(0xffffffffu, ps, 31);
        int wl = 0, ws = 0;
        if (lane == 0) {
            wl = tot_l ? atomicAdd(&n_large, tot_l) : 0;
            ws = tot_s ? atomicAdd(&n_small, tot_s) : 0;
        }
        base_l = __shfl_sync(0xffffffffu, wl, 0) + pl - ml;
        base_s = __shfl_sync(0xffffffffu, ws, 0) + ps - ms;
    }
    for (int s = 0; s < SWEEP_SB; ++s) {
        const unsigned bal = __ballot_sync(0xffffffffu, (vmask >> s) & 1u);
        if ((vmask >> s) & 1u) {
            const uint32_t p = (uint32_t)(woff[s * SWEEP_NW + warp] + __popc(bal & lt));
            const uint32_t e = p | ((uint32_t)s << 13) | ((uint32_t)threadIdx.x << 18);
            if (large) plist[SWEEP_SB * SWEEP_GT - 1 - base_l++] = e;
            else plist[base_s++] = e;
        }
    }
    if (threadIdx.x <= SWEEP_SB) sstart[threadIdx.x] = woff[min((int)threadIdx.x, SWEEP_SB) * SWEEP_NW];
    __syncthreads();
    if (staged && !mbar_wait_bounded(&bar, 0)) {
        // the staging copy did not complete in time: report it, wait (bounded) once more so no
        // copy is left writing into this CTA's shared memory, and leave the tile's rows unwritten
        atomicExch(status, 2);
        mbar_wait_bounded(&bar, 0);
        return;
    }
    const int ns = n_small, nl = n_large;

    // large groups: one warp per pair, lanes over terms, TwoSum butterfly
    for (int i = warp; i < nl; i += SWEEP_NW) {
        const uint32_t e = plist[SWEEP_SB * SWEEP_GT - 1 - i];
        const int p = e & 0x1fff, s = (e >> 13) & 0x1f, gl = e >> 18;
        const uint64_t x = xs[s];
        const uint64_t mg = g_mask[gl];
        const bool has_imag = (g_meta[gl] & META_HAS_IMAG) != 0;
        const uint32_t a0 = g_k0[gl], a1 = g_k1[gl];
        float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
        for (uint32_t k = a0 + lane; k < a1; k += 32) {
            const uint64_t z = staged ? zs[k - t0] : __ldg(h.term_z + k);
            const float2 c = staged ? cs[k - t0] : __ldg(h.term_c + k);
            add_term<COMP>(x, mg, has_imag, z, c, re, re_e, im, im_e);
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            const float ore = __shfl_xor_sync(0xffffffffu, re, d), oree = __shfl_xor_sync(0xffffffffu, re_e, d);
            const float oim = __shfl_xor_sync(0xffffffffu, im, d), oime = __shfl_xor_sync(0xffffffffu, im_e, d);
            if (COMP) {
                // both lanes form the same pair sum: order the operands by lane
                const bool low = (lane & d) == 0;
                float a = low ? re : ore, b = low ? ore : re;
                float ae = (low ? re_e : oree) + (low ? oree : re_e);
                two_sum_acc(a, ae, b);
                re = a; re_e = ae;
                float c2 = low ? im : oim, d2 = low ? oim : im;
                float ce = (low ? im_e : oime) + (low ? oime : im_e);
                two_sum_acc(c2, ce, d2);
                im = c2; im_e = ce;
            } else {
                const bool low = (lane & d) == 0;
                re = low ? re + ore : ore + re;
                im = low ? im + oim : oim + im;
            }
        }
        if (lane == 0) {
            const int64_t row = obase[s] + (p - sstart[s]);
            xprime[row] = x ^ mg;
            S[row] = make_float4(re, re_e, im, im_e);
        }
    }

    // small groups: one thread per pair, 32-pair chunks per warp from a shared counter
    for (;;) {
        int c0 = 0;
        if (lane == 0) c0 = atomicAdd(&next_small, 32);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if (c0 >= ns) break;
        const int i = c0 + lane;
        if (i < ns) {
            const uint32_t e = plist[i];
            const int p = e & 0x1fff, s = (e >> 13) & 0x1f, gl = e >> 18;
            const uint64_t x = xs[s];
            const uint64_t mg = g_mask[gl];
            const bool has_imag = (g_meta[gl] & META_HAS_IMAG) != 0;
            const uint32_t a0 = g_k0[gl], a1 = g_k1[gl];
            float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
            for (uint32_t k = a0; k < a1; ++k) {
                const uint64_t z = staged ? zs[k - t0] : __ldg(h.term_z + k);
                const float2 c = staged ? cs[k - t0] : __ldg(h.term_c + k);
                add_term<COMP>(x, mg, has_imag, z, c, re, re_e, im, im_e);
            }
            const int64_t row = obase[s] + (p - sstart[s]);
            xprime[row] = x ^ mg;
            S[row] = make_float4(re, re_e, im, im_e);
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

int launch_sweep_count(const HamDev& h, int n_up, int n_dn, const uint64_t* bits,
                       int64_t B, int32_t* cnt, uint32_t* valid, cudaStream_t s) {
    if (B <= 0) return NQS_OK;
    const int64_t T = sweep_tiles(h);
    dim3 grid((unsigned)((B + SWEEP_SB - 1) / SWEEP_SB), (unsigned)T);
    sweep_count_kernel<<<grid, SWEEP_GT, 0, s>>>(h, n_up, n_dn, bits, B, cnt, T, valid);
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_sweep_emit(const HamDev& h, int n_up, int n_dn, int compensated,
                      const uint64_t* bits, int64_t B, const int64_t* off, const uint32_t* valid,
                      uint64_t* xprime, float4* S, cudaStream_t s) {
    if (B <= 0) return NQS_OK;
    const int64_t T = sweep_tiles(h);
    dim3 grid((unsigned)((B + SWEEP_SB - 1) / SWEEP_SB), (unsigned)T);
    constexpr size_t smem = (size_t)SWEEP_STAGE * 16;
    static bool attr_set = false;
    if (!attr_set) {
        NQS_CK(cudaFuncSetAttribute(sweep_emit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        NQS_CK(cudaFuncSetAttribute(sweep_emit_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    int* status = nullptr;
    NQS_TRY(device_status_ptr(&status));
    if (compensated)
        sweep_emit_kernel<true><<<grid, SWEEP_GT, smem, s>>>(h, n_up, n_dn, bits, B, off, T, valid, xprime, S, status);
    else
        sweep_emit_kernel<false><<<grid, SWEEP_GT, smem, s>>>(h, n_up, n_dn, bits, B, off, T, valid, xprime, S, status);
    NQS_LAUNCHED();
    return NQS_OK;
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
