// Unique-sample autoregressive sampling with occurrence counts (paper Section 4, Sampling).
//
// The buffer holds distinct prefixes in ascending bit order with their counts; it starts as one
// empty prefix with count N_s.  Step k (qubit q = order[k]):
//   1. the model gives each parent its constrained conditional p = pihat(x_q = 1 | prefix);
//   2. each nominal sample j -- parent s owns j in [start_s, start_s + count_s) with start the
//      exclusive prefix sum of the counts -- draws u = word 0 of Philox4x32-10(counter
//      (j, k, 0, 0), key (seed lo, seed hi)) and counts a one iff u < floor(p * 2^32);
//   3. parent s splits into (bits, count - ones) and (bits | 1 << q, ones); zero counts vanish;
//   4. if more than max_unique entries remain, the top max_unique by (count desc, bits asc)
//      are kept (the paper evicts the lowest counts; ties are broken by bit order here).
// Children keep the ascending order without a sort: parents are sorted and OR-ing the absent
// bit q into every parent preserves their order, so each child list is sorted and the new
// buffer is the merge of the two, done by binary searches.  Everything runs against the
// device-side unique count; the host reads U once, after the last step.
//
// Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11 (ten rounds; multipliers 0xD2511F53, 0xCD9E8D57; Weyl key increments 0x9E3779B9,
// 0xBB67AE85).
#include "nqs_internal.h"

namespace nqs {
namespace {

__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return c0;
}

// U[0] = unique count, U[2] = eviction flag, U[3] = seed (read by the draws, so that a
// captured graph of the steps can be replayed with a new seed)
template <class BT>
__global__ void init_kernel(BT* bits, int64_t* cnt, int64_t* U, int64_t n_samples, uint64_t seed,
                            int64_t* start, int64_t* n1) {
    bits[0] = bits_zero<BT>();
    cnt[0] = n_samples;
    U[0] = 1;
    U[3] = (int64_t)seed;
    start[0] = 0;          // the first step's draw ranges and ones counters (one-CTA bookkeeping)
    start[1] = n_samples;
    n1[0] = 0;
}

// ones per parent: warp-aggregated integer atomics (exact, order-independent)
// sstart_cap > 0: the U + 1 range starts are staged in shared memory (dynamic, sstart_cap
// entries) when they fit, so the parent searches run there instead of in global memory.
__global__ void draw_kernel(int64_t n_samples, const int64_t* __restrict__ start,
                            const int64_t* __restrict__ Udev, const uint64_t* __restrict__ thr,
                            int64_t* __restrict__ n1, int k, int64_t sstart_cap) {
    extern __shared__ int64_t sstart[];
    pdl_wait();
    pdl_trigger();
    const int64_t U = Udev[0];
    const uint64_t seed = (uint64_t)Udev[3];
    const uint32_t key0 = (uint32_t)(seed & 0xffffffffu), key1 = (uint32_t)(seed >> 32);
    const bool staged = U + 1 <= sstart_cap;
    if (staged) {
        for (int64_t i = threadIdx.x; i <= U; i += blockDim.x) sstart[i] = start[i];
        __syncthreads();
    }
    const int64_t* st = staged ? sstart : start;
    // after an eviction the surviving counts sum to less than n_samples: the nominal indices
    // run over [0, start[U]) only
    const int64_t total = min(st[U], n_samples);
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x; j0 < total; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        int64_t s = -1;
        bool one = false;
        if (j < total) {
            // parent = last s with start[s] <= j
            int64_t lo = 0, hi = U - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (st[mid] <= j) lo = mid; else hi = mid - 1;
            }
            s = lo;
            const uint32_t u = philox_word0((uint32_t)j, (uint32_t)k, 0u, 0u, key0, key1);
            one = (uint64_t)u < thr[s];
        }
        const unsigned grp = __match_any_sync(0xffffffffu, one ? s : -1);
        if (one) {
            const int leader = __ffs(grp) - 1;
            if ((int)(threadIdx.x & 31) == leader) atomicAdd((unsigned long long*)&n1[s], (unsigned long long)__popc(grp));
        }
    }
}

__global__ void zero_kernel(int64_t* a, const int64_t* Udev, int64_t cap) {
    const int64_t U = min(*Udev, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < U; i += (int64_t)gridDim.x * blockDim.x) a[i] = 0;
}

__global__ void flags_kernel(const int64_t* __restrict__ cnt, const int64_t* __restrict__ n1,
                             const int64_t* __restrict__ Udev, int64_t* __restrict__ f0,
                             int64_t* __restrict__ f1) {
    const int64_t U = *Udev;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < U; s += (int64_t)gridDim.x * blockDim.x) {
        f0[s] = (cnt[s] - n1[s]) > 0;
        f1[s] = n1[s] > 0;
    }
}

// first index in [0, U) whose key exceeds v, where key(s) = bits[s] | orbit (monotone in s)
template <class BT>
__device__ __forceinline__ int64_t upper(const BT* bits, int64_t U, BT orbit, BT v) {
    int64_t lo = 0, hi = U;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((bits[mid] | orbit) <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <class BT>
__global__ void merge_kernel(const BT* __restrict__ bits, const int64_t* __restrict__ cnt,
                             const int64_t* __restrict__ n1, const int64_t* __restrict__ pos0,
                             const int64_t* __restrict__ pos1, int64_t* __restrict__ Udev,
                             BT qbit, BT* __restrict__ nbits, int64_t* __restrict__ ncnt,
                             int32_t* __restrict__ npar) {
    const int64_t U = *Udev;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < U; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c1 = n1[s], c0 = cnt[s] - c1;
        if (c0 > 0) {
            // children-1 keys below bits[s]: parents whose key (bits | q) is below bits[s]
            const int64_t r = pos1[upper(bits, U, qbit, bits[s])];
            nbits[pos0[s] + r] = bits[s];
            ncnt[pos0[s] + r] = c0;
            if (npar) npar[pos0[s] + r] = (int32_t)s;
        }
        if (c1 > 0) {
            const BT key = bits[s] | qbit;
            const int64_t r = pos0[upper(bits, U, bits_zero<BT>(), key)];
            nbits[pos1[s] + r] = key;
            ncnt[pos1[s] + r] = c1;
            if (npar) npar[pos1[s] + r] = (int32_t)s;
        }
    }
}

__global__ void set_u_kernel(int64_t* Udev, const int64_t* pos0, const int64_t* pos1) {
    const int64_t U = *Udev;
    Udev[0] = pos0[U] + pos1[U];
}

// Keep the top max_unique of the U entries (bits, cnt[, par]) by (count desc, bits asc) into
// (obits, ocnt[, opar]) with their order preserved; one CTA of 1024 threads, U > max_unique.
// scnt, when given, holds the U counts (as uint32) in shared memory and replaces the reads of cnt.
template <class BT>
__device__ void evict_block(const BT* __restrict__ bits, const int64_t* __restrict__ cnt,
                            const int32_t* __restrict__ par, int64_t U, int64_t max_unique,
                            BT* __restrict__ obits, int64_t* __restrict__ ocnt, int32_t* __restrict__ opar,
                            const uint32_t* scnt = nullptr) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_need, s_max;
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t carry_sh;
    auto count_at = [&](int64_t i) -> uint32_t { return scnt ? scnt[i] : (uint32_t)cnt[i]; };
    const int lane = threadIdx.x & 31;
    // the largest count fixes the first radix digit that is not zero for every entry
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    {
        uint32_t m = 0;
        for (int64_t s = threadIdx.x; s < U; s += blockDim.x) m = max(m, count_at(s));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMax(&s_max, m);
    }
    __syncthreads();
    const uint32_t cmax = s_max;
    const int top = cmax >= (1u << 24) ? 24 : cmax >= (1u << 16) ? 16 : cmax >= (1u << 8) ? 8 : 0;
    // radix select of the max_unique-th largest count (counts < 2^31); the digits above `top`
    // are zero for every entry and need no pass
    uint32_t prefix = 0, pmask = top < 24 ? ~0u << (top + 8) : 0u;
    uint32_t need = (uint32_t)max_unique;   // how many still to take at or above prefix
    for (int shift = top; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        // one shared atomic per distinct digit and warp (the low digits repeat heavily)
        for (int64_t base = 0; base < U; base += blockDim.x) {
            const int64_t s = base + threadIdx.x;
            const uint32_t c = s < U ? count_at(s) : 0u;
            const bool in = s < U && (c & pmask) == prefix;
            const uint32_t key = in ? (c >> shift) & 0xffu : 0x100u;
            const unsigned grp = __match_any_sync(0xffffffffu, key);
            if (in && lane == __ffs(grp) - 1) atomicAdd(&hist[key], (uint32_t)__popc(grp));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // highest bin d whose count from the top reaches `need` (else 0), and the count of
            // the bins above it: lane l scans bins 255 - 8l .. 248 - 8l, a warp scan joins them
            uint32_t loc[8], sum = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) { loc[i] = hist[255 - 8 * lane - i]; sum += loc[i]; }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t acc = incl - sum;
            int found = -1;
            uint32_t above = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (found < 0) {
                    if (acc + loc[i] >= need) { found = 255 - 8 * lane - i; above = acc; }
                    else acc += loc[i];
                }
            }
            const unsigned hit = __ballot_sync(0xffffffffu, found >= 0 && found > 0);
            if (hit) {
                if (lane == __ffs(hit) - 1) { s_prefix = prefix | ((uint32_t)found << shift); s_need = need - above; }
            } else if (lane == 31) {
                // no bin above 0 reaches `need`: bin 0, below all the others
                s_prefix = prefix;
                s_need = need - (incl - loc[7]);
            }
        }
        __syncthreads();
        prefix = s_prefix;
        need = s_need;
        pmask |= 0xffu << shift;
        __syncthreads();
    }
    const uint32_t T = prefix;      // threshold count; keep `need` of the entries equal to T
    // ordered compaction: keep c > T, and the first `need` entries with c == T
    int64_t carry_keep = 0, carry_eq = 0;
    for (int64_t base = 0; base < U; base += blockDim.x) {
        const int64_t s = base + threadIdx.x;
        const uint32_t c = s < U ? count_at(s) : 0u;
        const int64_t eq = (s < U && c == T) ? 1 : 0;
        // rank among equals
        const int warp = threadIdx.x >> 5;
        int64_t incl = eq;
        for (int d = 1; d < 32; d <<= 1) { const int64_t y = __shfl_up_sync(0xffffffffu, incl, d); if (lane >= d) incl += y; }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0, wi = w;
            for (int d = 1; d < 32; d <<= 1) { const int64_t y = __shfl_up_sync(0xffffffffu, wi, d); if (lane >= d) wi += y; }
            if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = wi - w;
            if (lane == 31) carry_sh = wi;
        }
        __syncthreads();
        const int64_t eq_rank = carry_eq + warp_sums[warp] + incl - eq;
        const int64_t tot_eq = carry_sh;
        __syncthreads();
        const int64_t keep = (s < U && (c > T || (c == T && eq_rank < (int64_t)need))) ? 1 : 0;
        incl = keep;
        for (int d = 1; d < 32; d <<= 1) { const int64_t y = __shfl_up_sync(0xffffffffu, incl, d); if (lane >= d) incl += y; }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0, wi = w;
            for (int d = 1; d < 32; d <<= 1) { const int64_t y = __shfl_up_sync(0xffffffffu, wi, d); if (lane >= d) wi += y; }
            if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = wi - w;
            if (lane == 31) carry_sh = wi;
        }
        __syncthreads();
        if (keep) {
            const int64_t pos = carry_keep + warp_sums[warp] + incl - keep;
            obits[pos] = bits[s];
            ocnt[pos] = c;
            if (par) opar[pos] = par[s];
        }
        carry_keep += carry_sh;
        carry_eq += tot_eq;
        __syncthreads();
    }
}

template <class BT>
__global__ void __launch_bounds__(1024)
evict_kernel(const BT* __restrict__ bits, const int64_t* __restrict__ cnt,
             int64_t* __restrict__ Udev, int64_t max_unique, BT* __restrict__ obits,
             int64_t* __restrict__ ocnt, int32_t* __restrict__ did, const int32_t* __restrict__ par,
             int32_t* __restrict__ opar) {
    const int64_t U = *Udev;
    if (U <= max_unique) { if (threadIdx.x == 0) *did = 0; return; }
    evict_block(bits, cnt, par, U, max_unique, obits, ocnt, opar);
    if (threadIdx.x == 0) { *Udev = max_unique; *did = 1; }
}

// ---------------------------------------------------------------- one-CTA step bookkeeping
// For buffers of at most SAMPLER_GRAPH_MAX_CAP entries the per-step bookkeeping runs in two
// one-CTA kernels around the draws (same results as the multi-kernel sequence above).
constexpr int BK_T = 1024;
constexpr int64_t BK_SMEM_PER_ENTRY = sizeof(uint64_t) + 3 * sizeof(uint32_t);   // bits, merged count, ones, zeros

// Exclusive scan of one value per thread across the CTA; *total receives the block sum.
__device__ int64_t bk_block_scan(int64_t v, int64_t* warp_sums, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = warp_sums[lane];
        int64_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        warp_sums[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const int64_t r = warp_sums[warp] + incl - v;
    __syncthreads();
    return r;
}

// After the draws: children positions (scans of the two flag arrays), merge into the spare
// buffers (nb, nc, npar), eviction or copy back into (cb, cc, par), the unique count, and the
// ancestor table of the next step (when the transformer cache is bound).
// first index in [0, U) whose key exceeds v, over bits staged in shared memory
__device__ __forceinline__ int upper_s(const uint64_t* sbits, int U, uint64_t orbit, uint64_t v) {
    int lo = 0, hi = U;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((sbits[mid] | orbit) <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(BK_T)
bk_finish_kernel(uint64_t* __restrict__ cb, int64_t* __restrict__ cc, int64_t* __restrict__ n1,
                 int64_t* __restrict__ pos0, int64_t* __restrict__ pos1, int64_t* __restrict__ Udev,
                 uint64_t qbit, uint64_t* __restrict__ nb, int64_t* __restrict__ nc,
                 int32_t* __restrict__ par, int32_t* __restrict__ npar, int64_t max_unique,
                 const int32_t* __restrict__ anc_old, int32_t* __restrict__ anc_new, int n, int k,
                 int64_t cap, int64_t* __restrict__ start_next) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t tot0, tot1;
    // dynamic shared memory: the U parent bit strings, cap merged counts, the parents' ones and
    // zeros counts (BK_SMEM_PER_ENTRY bytes per buffer entry)
    extern __shared__ uint64_t sbits[];
    pdl_wait();
    pdl_trigger();
    const int64_t U = *Udev;
    uint32_t* scnt = reinterpret_cast<uint32_t*>(sbits + cap);
    uint32_t* s1 = scnt + cap;
    uint32_t* s0 = s1 + cap;
    // flags and their scans; the parents' bits and child counts staged (counts < 2^31)
    int64_t c0 = 0, c1 = 0;
    for (int64_t base = 0; base < U; base += BK_T) {
        const int64_t s = base + threadIdx.x;
        int64_t m1 = 0, m0 = 0;
        if (s < U) {
            sbits[s] = cb[s];
            m1 = n1[s];
            m0 = cc[s] - m1;
            s1[s] = (uint32_t)m1;
            s0[s] = (uint32_t)m0;
        }
        const int64_t e0 = bk_block_scan(m0 > 0 ? 1 : 0, warp_sums, &tot0) + c0;
        const int64_t e1 = bk_block_scan(m1 > 0 ? 1 : 0, warp_sums, &tot1) + c1;
        if (s < U) { pos0[s] = e0; pos1[s] = e1; }
        c0 += tot0;
        c1 += tot1;
    }
    if (threadIdx.x == 0) { pos0[U] = c0; pos1[U] = c1; }
    __syncthreads();
    int64_t Un = c0 + c1;
    // merge (as merge_kernel), searching the staged bits: straight into the current buffers when
    // nothing is evicted (the parents' data is all staged), else into the spare ones
    const bool direct = Un <= max_unique;
    uint64_t* ob = direct ? cb : nb;
    int64_t* oc = direct ? cc : nc;
    int32_t* op = direct ? par : npar;
    for (int64_t s = threadIdx.x; s < U; s += BK_T) {
        const int64_t m1 = s1[s], m0 = s0[s];
        const uint64_t bs = sbits[s];
        if (m0 > 0) {
            const int64_t r = pos1[upper_s(sbits, (int)U, qbit, bs)];
            ob[pos0[s] + r] = bs;
            oc[pos0[s] + r] = m0;
            scnt[pos0[s] + r] = (uint32_t)m0;
            if (npar) op[pos0[s] + r] = (int32_t)s;
        }
        if (m1 > 0) {
            const uint64_t key = bs | qbit;
            const int64_t r = pos0[upper_s(sbits, (int)U, 0, key)];
            ob[pos1[s] + r] = key;
            oc[pos1[s] + r] = m1;
            scnt[pos1[s] + r] = (uint32_t)m1;
            if (npar) op[pos1[s] + r] = (int32_t)s;
        }
    }
    __syncthreads();
    if (!direct) {
        evict_block(nb, nc, npar, Un, max_unique, cb, cc, par, scnt);
        Un = max_unique;
    }
    __syncthreads();
    if (anc_new) {
        // every (prefix, step 0..k) entry by its own thread iteration: independent loads in flight
        const int kk = k + 1;
        const int tot = (int)Un * kk;                // Un <= SAMPLER_GRAPH_MAX_CAP, k < 64
#pragma unroll 4
        for (int e = threadIdx.x; e < tot; e += BK_T) {
            const int i = e / kk, j = e - i * kk;
            const int32_t p = par[i];
            anc_new[(int64_t)i * n + j] = j < k ? anc_old[(int64_t)p * n + j] : p;
        }
    }
    if (start_next) {
        // the next step's draw ranges (exclusive scan of the surviving counts, start[U] = their
        // sum) and zeroed ones counters
        __syncthreads();
        int64_t carry = 0;
        for (int64_t base = 0; base < Un; base += BK_T) {
            const int64_t i = base + threadIdx.x;
            const int64_t v = i < Un ? (direct ? (int64_t)scnt[i] : cc[i]) : 0;
            const int64_t ex = bk_block_scan(v, warp_sums, &tot0) + carry;
            if (i < Un) { start_next[i] = ex; n1[i] = 0; }
            carry += tot0;
        }
        if (threadIdx.x == 0) start_next[Un] = carry;
    }
    if (threadIdx.x == 0) *Udev = Un;
}

template <class BT>
__global__ void copy_back_kernel(const int32_t* __restrict__ did, const int64_t* __restrict__ Udev,
                                 const BT* __restrict__ sb, const int64_t* __restrict__ sc,
                                 BT* __restrict__ db, int64_t* __restrict__ dc,
                                 const int32_t* __restrict__ sp, int32_t* __restrict__ dp) {
    if (!*did) return;
    const int64_t U = *Udev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < U; i += (int64_t)gridDim.x * blockDim.x) {
        db[i] = sb[i];
        dc[i] = sc[i];
        if (sp) dp[i] = sp[i];
    }
}

// Ancestor table of the step-(k+1) prefixes: slot i (child of step-k slot par[i]) inherits its
// parent's ancestors at steps 0..k-1, and its ancestor at step k is the parent itself.
__global__ void anc_gather_kernel(const int32_t* __restrict__ par, const int32_t* __restrict__ anc_old,
                                  int32_t* __restrict__ anc_new, const int64_t* __restrict__ Udev, int n, int k) {
    const int64_t U = *Udev;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < U * (k + 1);
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / (k + 1);
        const int j = (int)(e % (k + 1));
        const int32_t p = par[i];
        anc_new[i * n + j] = j < k ? anc_old[(int64_t)p * n + j] : p;
    }
}

template <class BT>
__global__ void copy_out_kernel(const BT* __restrict__ sb, const int64_t* __restrict__ sc,
                                BT* __restrict__ db, int64_t* __restrict__ dc, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        db[i] = sb[i];
        dc[i] = sc[i];
    }
}

inline int grid_for(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)num_sms() * 16));
}

}  // namespace

int sampler_layout(Carver& c, int64_t n_samples, int64_t max_unique, SamplerBufs& b, int words) {
    b.cap = std::max<int64_t>(1, std::min<int64_t>(n_samples, 2 * max_unique));
    b.words = words;
    const int64_t cap = b.cap;
    b.bitsA = c.take<uint64_t>(cap * words);
    b.bitsB = c.take<uint64_t>(cap * words);
    b.cntA = c.take<int64_t>(cap);
    b.cntB = c.take<int64_t>(cap);
    b.start = c.take<int64_t>(cap + 1);
    b.n1 = c.take<int64_t>(cap);
    b.thr = c.take<uint64_t>(cap);
    b.p = c.take<float>(cap);
    b.flags0 = c.take<int64_t>(cap);
    b.flags1 = c.take<int64_t>(cap);
    b.pos0 = c.take<int64_t>(cap + 1);
    b.pos1 = c.take<int64_t>(cap + 1);
    b.U = c.take<int64_t>(4);
    return NQS_OK;
}

// Transformer conditional at step k over the first k+1 positions.  With fixed_rows the pass
// covers the whole buffer capacity (rows past the unique count are ignored later), so no host
// synchronisation is needed and the steps can be captured in a graph; otherwise the parent
// count is read back (one small synchronous copy per step) to size the passes exactly.
static int tf_cond(const ModelConst& mc, const float* P, int k, const uint64_t* bits,
                   const int64_t* Udev, SamplerBufs& b, float* trace, const TfCtx* tf,
                   bool fixed_rows, bool compose, cudaStream_t s) {
    int64_t U = b.cap;
    if (!fixed_rows) {
        NQS_CK(cudaMemcpyAsync(&U, Udev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
    }
    if (b.kv) {
        // incremental: position k only, earlier keys and values from the cache
        TfStepCache kc;
        kc.kv = b.kv; kc.cap = b.cap; kc.anc = b.ancA; kc.Udev = Udev;
        if (tf_step_fused_supported(mc)) {
            if (compose) { kc.par = b.par; kc.anc_new = b.ancB; }
            if (tf->tok_tables) { kc.tab_h = tf->b->tab_h; kc.tab_qkv = tf->b->tab_qkv; }
            return tf_step_fused(mc, P, *tf->w, bits, U, k, kc, b.p, b.thr, trace, s);
        }
        NQS_TRY(tf_step(mc, P, *tf->w, bits, U, k, kc, *tf->b, s));
        HeadArgsHost ha{};
        ha.mode = 2; ha.p_out = b.p; ha.thr = b.thr; ha.trace = trace; ha.step_pos = k;
        return tf_heads(mc, P, bits, U, 1, *tf->b, ha, s);
    }
    for (int64_t lo = 0; lo < U; lo += tf->b->R) {
        const int64_t R = std::min(tf->b->R, U - lo);
        NQS_TRY(tf_forward(mc, P, *tf->w, bits + lo, R, k + 1, *tf->b, s));
        HeadArgsHost ha{};
        ha.mode = 2; ha.p_out = b.p + lo; ha.thr = b.thr + lo; ha.trace = trace ? trace + lo : nullptr;
        NQS_TRY(tf_heads(mc, P, bits + lo, R, k + 1, *tf->b, ha, s));
    }
    return NQS_OK;
}

void sampler_bind_cache(SamplerBufs& b, const ModelConst& mc, void* mem) {
    Carver c(mem);
    b.kv = c.take<float>((int64_t)mc.n * mc.layers * b.cap * 3 * mc.hidden);
    b.ancA = c.take<int32_t>(b.cap * mc.n);
    b.ancB = c.take<int32_t>(b.cap * mc.n);
    b.par = c.take<int32_t>(b.cap);
    b.par2 = c.take<int32_t>(b.cap);
}

// Merge of the step-k children into the spare buffer, the unique count, and (when over
// max_unique) the eviction, on the multi-kernel path; (cb, cc) is current afterwards.
template <class BT>
static int merge_evict(const ModelConst& mc, int k, int64_t n_samples, int64_t max_unique, SamplerBufs& b,
                       uint64_t*& cb, int64_t*& cc, uint64_t*& nb, int64_t*& nc, int32_t* did, cudaStream_t s) {
    const int g = grid_for(b.cap);
    merge_kernel<BT><<<g, 256, 0, s>>>(reinterpret_cast<const BT*>(cb), cc, b.n1, b.pos0, b.pos1, b.U,
                                       with_bit(bits_zero<BT>(), mc.order[k]), reinterpret_cast<BT*>(nb), nc, b.par);
    NQS_LAUNCHED();
    set_u_kernel<<<1, 1, 0, s>>>(b.U, b.pos0, b.pos1);
    NQS_LAUNCHED();
    std::swap(cb, nb);
    std::swap(cc, nc);
    if (max_unique < n_samples) {
        // evict into the spare buffer, then copy back so (cb, cc) stays current
        evict_kernel<BT><<<1, 1024, 0, s>>>(reinterpret_cast<const BT*>(cb), cc, b.U, max_unique,
                                            reinterpret_cast<BT*>(nb), nc, did, b.par, b.par2);
        NQS_LAUNCHED();
        copy_back_kernel<BT><<<g, 256, 0, s>>>(did, b.U, reinterpret_cast<const BT*>(nb), nc,
                                               reinterpret_cast<BT*>(cb), cc, b.par2, b.par);
        NQS_LAUNCHED();
    }
    return NQS_OK;
}

int sampler_init(SamplerBufs& b, int64_t n_samples, uint64_t seed, cudaStream_t s) {
    if (b.words == 2)
        init_kernel<U128><<<1, 1, 0, s>>>(reinterpret_cast<U128*>(b.bitsA), b.cntA, b.U, n_samples, seed, b.start, b.n1);
    else
        init_kernel<uint64_t><<<1, 1, 0, s>>>(b.bitsA, b.cntA, b.U, n_samples, seed, b.start, b.n1);
    NQS_LAUNCHED();
    return NQS_OK;
}

int sampler_steps(const ModelConst& mc, const float* P, int64_t n_samples, int64_t max_unique,
                  SamplerBufs& b, float* trace, int64_t trace_stride, const TfCtx* tf,
                  bool fixed_rows, cudaStream_t s) {
    int32_t* did = reinterpret_cast<int32_t*>(b.U + 2);
    uint64_t* cb = b.bitsA; int64_t* cc = b.cntA;
    uint64_t* nb = b.bitsB; int64_t* nc = b.cntB;
    const int g = grid_for(b.cap);
    const bool one_cta = b.cap <= SAMPLER_GRAPH_MAX_CAP && b.words == 1;   // two-word bits: multi-kernel path
    if (one_cta) {
        // the parent bits and counts staged by bk_finish_kernel take up to 160 KB of shared
        // memory; the limit is raised once per device (before any captured launch: the first call
        // is an eager one)
        static int configured_device = -1;
        int dev = 0;
        NQS_CK(cudaGetDevice(&dev));
        if (configured_device != dev) {
            NQS_CK(cudaFuncSetAttribute(bk_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(SAMPLER_GRAPH_MAX_CAP * BK_SMEM_PER_ENTRY)));
            NQS_CK(cudaFuncSetAttribute(draw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((SAMPLER_GRAPH_MAX_CAP + 1) * sizeof(int64_t))));
            configured_device = dev;
        }
    }
    // the one-kernel transformer step composes each step's ancestor table itself (from the
    // parents the bookkeeping leaves), so the bookkeeping does not write it
    const bool compose = one_cta && mc.arch == NQS_ARCH_TRANSFORMER && b.kv && tf_step_fused_supported(mc);
    for (int k = 0; k < mc.n; ++k) {
        float* tr = trace ? trace + (int64_t)k * trace_stride : nullptr;
        if (mc.arch == NQS_ARCH_TRANSFORMER) NQS_TRY(tf_cond(mc, P, k, cb, b.U, b, tr, tf, fixed_rows, compose, s));
        else NQS_TRY(launch_cond_rows(mc, P, k, cb, b.U, b.cap, b.p, b.thr, tr, s));
        if (compose) std::swap(b.ancA, b.ancB);
        if (one_cta) {
            // two launches: draws, then flags / merge / eviction / ancestors and the next step's
            // draw ranges (the first step's come from init_kernel)
            // programmatic dependent launches: each kernel is resident before its predecessor ends
            NQS_CK(launch_pdl(draw_kernel, dim3(grid_for(n_samples)), dim3(256), (size_t)((b.cap + 1) * sizeof(int64_t)), s,
                              n_samples, (const int64_t*)b.start, (const int64_t*)b.U, (const uint64_t*)b.thr, b.n1, k,
                              (int64_t)(b.cap + 1)));
            count_launch();
            const bool anc = b.kv && k + 1 < mc.n && !compose;
            NQS_CK(launch_pdl(bk_finish_kernel, dim3(1), dim3(BK_T), (size_t)(b.cap * BK_SMEM_PER_ENTRY), s, cb, cc, b.n1,
                              b.pos0, b.pos1, b.U, (uint64_t)(1ull << mc.order[k]), nb, nc, b.kv ? b.par : nullptr,
                              b.kv ? b.par2 : nullptr, max_unique, (const int32_t*)(anc ? b.ancA : nullptr),
                              anc ? b.ancB : nullptr, (int)mc.n, k, b.cap, b.start));
            count_launch();
            if (anc) std::swap(b.ancA, b.ancB);
            continue;
        }
        NQS_TRY(launch_scan_i64(cc, b.cap, b.U, b.start, s));
        zero_kernel<<<g, 256, 0, s>>>(b.n1, b.U, b.cap);
        NQS_LAUNCHED();
        draw_kernel<<<grid_for(n_samples), 256, 0, s>>>(n_samples, b.start, b.U, b.thr, b.n1, k, 0);
        NQS_LAUNCHED();
        flags_kernel<<<g, 256, 0, s>>>(cc, b.n1, b.U, b.flags0, b.flags1);
        NQS_LAUNCHED();
        NQS_TRY(launch_scan_i64(b.flags0, b.cap, b.U, b.pos0, s));
        NQS_TRY(launch_scan_i64(b.flags1, b.cap, b.U, b.pos1, s));
        NQS_TRY(b.words == 2 ? merge_evict<U128>(mc, k, n_samples, max_unique, b, cb, cc, nb, nc, did, s)
                             : merge_evict<uint64_t>(mc, k, n_samples, max_unique, b, cb, cc, nb, nc, did, s));
        if (b.kv && k + 1 < mc.n) {
            anc_gather_kernel<<<grid_for(b.cap * (k + 1)), 256, 0, s>>>(b.par, b.ancA, b.ancB, b.U, mc.n, k);
            NQS_LAUNCHED();
            std::swap(b.ancA, b.ancB);
        }
    }
    if (cb != b.bitsA) {
        if (b.words == 2)
            copy_out_kernel<U128><<<g, 256, 0, s>>>(reinterpret_cast<const U128*>(cb), cc,
                                                    reinterpret_cast<U128*>(b.bitsA), b.cntA, b.cap);
        else
            copy_out_kernel<uint64_t><<<g, 256, 0, s>>>(cb, cc, b.bitsA, b.cntA, b.cap);
        NQS_LAUNCHED();
    }
    return NQS_OK;
}

int run_sampler(const ModelConst& mc, const float* P, int64_t n_samples, int64_t max_unique,
                uint64_t seed, SamplerBufs& b, float* trace, int64_t trace_stride,
                const TfCtx* tf, bool fixed_rows, cudaStream_t s) {
    ProfScope ps("sample", s);
    NQS_TRY(sampler_init(b, n_samples, seed, s));
    return sampler_steps(mc, P, n_samples, max_unique, b, trace, trace_stride, tf, fixed_rows, s);
}

int launch_copy_samples(const SamplerBufs& b, uint64_t* bits_out, int64_t* counts_out, int64_t n,
                        cudaStream_t s) {
    if (b.words == 2)
        copy_out_kernel<U128><<<grid_for(n), 256, 0, s>>>(reinterpret_cast<const U128*>(b.bitsA), b.cntA,
                                                          reinterpret_cast<U128*>(bits_out), counts_out, n);
    else
        copy_out_kernel<uint64_t><<<grid_for(n), 256, 0, s>>>(b.bitsA, b.cntA, bits_out, counts_out, n);
    NQS_LAUNCHED();
    return NQS_OK;
}

}  // namespace nqs
