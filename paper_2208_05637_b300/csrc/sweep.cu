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
#include "nqs_internal.h"

namespace nqs {
namespace {

__device__ __forceinline__ bool sector_ok(uint64_t x, uint64_t m, uint32_t meta, uint64_t A,
                                          uint64_t Bm) {
    const uint32_t na = meta & 0xffu, nb = (meta >> 8) & 0xffu;
    return 2u * (uint32_t)__popcll(x & m & A) == na && 2u * (uint32_t)__popcll(x & m & Bm) == nb;
}

// Knuth's TwoSum: s + e == a + b exactly, accumulated into the error term.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
}

__global__ void __launch_bounds__(SWEEP_GT)
sweep_count_kernel(HamDev h, uint64_t A, uint64_t Bm, const uint64_t* __restrict__ bits, int64_t B,
                   int32_t* __restrict__ cnt, int64_t ntiles) {
    __shared__ uint64_t xs[SWEEP_SB];
    __shared__ int32_t wcnt[SWEEP_SB][SWEEP_GT / 32];
    const int tile = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * SWEEP_SB;
    const int nb = (int)(B - s0 < SWEEP_SB ? B - s0 : SWEEP_SB);
    const int64_t g = (int64_t)tile * SWEEP_GT + threadIdx.x;
    const bool live = g < h.G;
    const uint64_t m = live ? h.grp_mask[g] : 0;
    const uint32_t meta = live ? h.grp_meta[g] : 0;
    if (threadIdx.x < nb) xs[threadIdx.x] = bits[s0 + threadIdx.x];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = 0; s < nb; ++s) {
        const bool v = live && sector_ok(xs[s], m, meta, A, Bm);
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == 0) wcnt[s][warp] = __popc(bal);
    }
    __syncthreads();
    if (threadIdx.x < nb) {
        int32_t c = 0;
#pragma unroll
        for (int w = 0; w < SWEEP_GT / 32; ++w) c += wcnt[threadIdx.x][w];
        cnt[(s0 + threadIdx.x) * ntiles + tile] = c;
    }
}

__global__ void __launch_bounds__(SWEEP_GT)
sweep_emit_kernel(HamDev h, uint64_t A, uint64_t Bm, int compensated,
                  const uint64_t* __restrict__ bits, int64_t B, const int64_t* __restrict__ off,
                  int64_t ntiles, uint64_t* __restrict__ xprime, float4* __restrict__ S) {
    constexpr int NW = SWEEP_GT / 32;
    __shared__ uint64_t xs[SWEEP_SB];
    __shared__ int32_t woff[SWEEP_SB * NW + 1];
    __shared__ uint16_t pairs[SWEEP_SB * SWEEP_GT];
    __shared__ int32_t sstart[SWEEP_SB + 1];
    __shared__ int64_t obase[SWEEP_SB];

    const int tile = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * SWEEP_SB;
    const int nb = (int)(B - s0 < SWEEP_SB ? B - s0 : SWEEP_SB);
    const int64_t g = (int64_t)tile * SWEEP_GT + threadIdx.x;
    const bool live = g < h.G;
    const uint64_t m = live ? h.grp_mask[g] : 0;
    const uint32_t meta = live ? h.grp_meta[g] : 0;
    if (threadIdx.x < nb) {
        xs[threadIdx.x] = bits[s0 + threadIdx.x];
        obase[threadIdx.x] = off[(s0 + threadIdx.x) * ntiles + tile];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;

    // validity bits of this thread's group for every sample of the batch
    uint32_t vmask = 0;
    for (int s = 0; s < nb; ++s)
        if (live && sector_ok(xs[s], m, meta, A, Bm)) vmask |= 1u << s;
    for (int s = 0; s < SWEEP_SB; ++s) {
        const unsigned bal = __ballot_sync(0xffffffffu, (vmask >> s) & 1u);
        if (lane == 0) woff[s * NW + warp] = __popc(bal);
    }
    __syncthreads();
    // exclusive scan of the SB*NW warp counts (sample-major, warp-minor) by one warp
    if (warp == 0) {
        constexpr int PER = (SWEEP_SB * NW + 31) / 32;
        int32_t loc[PER];
        int32_t run = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = lane * PER + i;
            loc[i] = idx < SWEEP_SB * NW ? woff[idx] : 0;
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
            if (idx < SWEEP_SB * NW) woff[idx] = excl;
            excl += loc[i];
        }
        if (lane == 31) woff[SWEEP_SB * NW] = incl;
    }
    __syncthreads();
    for (int s = 0; s < SWEEP_SB; ++s) {
        const unsigned bal = __ballot_sync(0xffffffffu, (vmask >> s) & 1u);
        if ((vmask >> s) & 1u) pairs[woff[s * NW + warp] + __popc(bal & lt)] = (uint16_t)((s << 8) | threadIdx.x);
    }
    if (threadIdx.x <= SWEEP_SB) sstart[threadIdx.x] = woff[min((int)threadIdx.x, SWEEP_SB) * NW];
    __syncthreads();

    const int total = woff[SWEEP_SB * NW];
    for (int p = threadIdx.x; p < total; p += SWEEP_GT) {
        const int s = pairs[p] >> 8;
        const int gl = pairs[p] & 0xff;
        const int64_t gg = (int64_t)tile * SWEEP_GT + gl;
        const uint64_t x = xs[s];
        const uint64_t mg = h.grp_mask[gg];
        const bool has_imag = (h.grp_meta[gg] & META_HAS_IMAG) != 0;
        const uint32_t k0 = h.grp_off[gg], k1 = h.grp_off[gg + 1];
        float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
        for (uint32_t k = k0; k < k1; ++k) {
            const uint64_t z = __ldg(h.term_z + k);
            const float2 c = __ldg(h.term_c + k);
            // (-1)^{popcount(x & z)}: flip the float sign bits by the parity
            const uint32_t flip = ((uint32_t)__popcll(x & z) & 1u) << 31;
            const float hi = __uint_as_float(__float_as_uint(c.x) ^ flip);
            const float lo = __uint_as_float(__float_as_uint(c.y) ^ flip);
            const bool imag = has_imag && (__popcll(mg & z) & 1);
            if (compensated) {
                if (imag) { two_sum_acc(im, im_e, hi); im_e += lo; }
                else      { two_sum_acc(re, re_e, hi); re_e += lo; }
            } else {
                if (imag) im += hi; else re += hi;
            }
        }
        const int64_t row = obase[s] + (p - sstart[s]);
        xprime[row] = x ^ mg;
        S[row] = make_float4(re, re_e, im, im_e);
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

int launch_sweep_count(const HamDev& h, uint64_t A, uint64_t Bm, int, int, const uint64_t* bits,
                       int64_t B, int32_t* cnt, cudaStream_t s) {
    if (B <= 0) return NQS_OK;
    const int64_t T = sweep_tiles(h);
    dim3 grid((unsigned)((B + SWEEP_SB - 1) / SWEEP_SB), (unsigned)T);
    sweep_count_kernel<<<grid, SWEEP_GT, 0, s>>>(h, A, Bm, bits, B, cnt, T);
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_sweep_emit(const HamDev& h, uint64_t A, uint64_t Bm, int, int, int compensated,
                      const uint64_t* bits, int64_t B, const int64_t* off, uint64_t* xprime,
                      float4* S, cudaStream_t s) {
    if (B <= 0) return NQS_OK;
    const int64_t T = sweep_tiles(h);
    dim3 grid((unsigned)((B + SWEEP_SB - 1) / SWEEP_SB), (unsigned)T);
    sweep_emit_kernel<<<grid, SWEEP_GT, 0, s>>>(h, A, Bm, compensated, bits, B, off, T, xprime, S);
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
