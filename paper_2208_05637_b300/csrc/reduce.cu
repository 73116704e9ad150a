// Scans, FP64 energy statistics (paper Eq. total_energy_sum), Adam (Section 5.1) and the
// deterministic outer-product reduction used by the backward pass (Eq. grad).
#include "nqs_internal.h"

namespace nqs {
namespace {

constexpr int SCAN_T = 1024;   // threads of the single-CTA scans
constexpr int SCAN_V = 4;      // elements per thread per tile

// Block-wide exclusive scan of one int64 per thread; returns the block total in *total.
__device__ int64_t block_excl_scan(int64_t v, int64_t* warp_sums, int64_t* total) {
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
        const int nw = blockDim.x >> 5;
        int64_t w = lane < nw ? warp_sums[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const int64_t r = warp_sums[warp] + incl - v;
    __syncthreads();
    return r;
}

template <class T>
__global__ void __launch_bounds__(SCAN_T)
scan_kernel(const T* __restrict__ in, int64_t n_max, const int64_t* __restrict__ n_dev,
            int64_t* __restrict__ out) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t tot;
    const int64_t n = n_dev ? min(*n_dev, n_max) : n_max;
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += (int64_t)SCAN_T * SCAN_V) {
        int64_t v[SCAN_V];
        int64_t sum = 0;
#pragma unroll
        for (int i = 0; i < SCAN_V; ++i) {
            const int64_t idx = base + (int64_t)threadIdx.x * SCAN_V + i;
            v[i] = idx < n ? (int64_t)in[idx] : 0;
            sum += v[i];
        }
        int64_t ex = block_excl_scan(sum, warp_sums, &tot) + carry;
#pragma unroll
        for (int i = 0; i < SCAN_V; ++i) {
            const int64_t idx = base + (int64_t)threadIdx.x * SCAN_V + i;
            if (idx < n) out[idx] = ex;
            ex += v[i];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// ---------------------------------------------------------------- energy statistics
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 block sums of up to three values per thread: warp shuffles, then warp 0 over the warp sums.
__device__ __forceinline__ void block_sum3_f64(double (&v)[3], int nv, double (*red)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = 0; q < nv; ++q) v[q] = warp_sum_f64(v[q]);
    if (lane == 0)
        for (int q = 0; q < nv; ++q) red[q][warp] = v[q];
    __syncthreads();
    if (warp == 0) {
        for (int q = 0; q < nv; ++q) {
            const double t = lane < nw ? red[q][lane] : 0.0;
            red[q][lane] = warp_sum_f64(t);
        }
    }
    __syncthreads();
    for (int q = 0; q < nv; ++q) v[q] = red[q][0];
    __syncthreads();
}

__global__ void __launch_bounds__(1024)
stats_kernel(const float* __restrict__ eloc, const int64_t* __restrict__ counts, int64_t B,
             double* __restrict__ stats, float* __restrict__ g_abs, float* __restrict__ g_phase) {
    __shared__ double red[3][32];
    double a[3] = {0.0, 0.0, 0.0};          // W, sum w Re E, sum w Im E
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
        const double c = (double)counts[i];
        a[0] += c;
        a[1] += c * (double)eloc[2 * i];
        a[2] += c * (double)eloc[2 * i + 1];
    }
    block_sum3_f64(a, 3, red);
    // one FP64 division (the reciprocal of W), products elsewhere
    const double W = a[0], invW = 1.0 / W, mr = a[1] * invW, mi = a[2] * invW;
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
        const double c = (double)counts[i];
        const double dr = (double)eloc[2 * i] - mr, di = (double)eloc[2 * i + 1] - mi;
        v[0] += c * (dr * dr + di * di);
        if (g_abs) {
            const double cw = 2.0 * c * invW;
            g_abs[i] = (float)(cw * dr);
            g_phase[i] = (float)(cw * (double)eloc[2 * i + 1]);
        }
    }
    block_sum3_f64(v, 1, red);
    if (threadIdx.x == 0) {
        stats[0] = mr; stats[1] = mi; stats[2] = v[0] * invW; stats[3] = W;
    }
}

// Per-rank pieces of the data-parallel VMC gradient: FP64 sums [sum w Re E, sum w Im E,
// sum w |E|^2, W] and the two sets of upstream gradients whose backward passes give the
// unnormalised gradient sums (2 w Re E, 2 w Im E) and (w, 0).
__global__ void __launch_bounds__(1024)
sums_kernel(const float* __restrict__ eloc, const int64_t* __restrict__ counts, int64_t B, double* __restrict__ sums,
            float* __restrict__ ga_e, float* __restrict__ gp_e, float* __restrict__ ga_w) {
    __shared__ double red[3][32];
    double a[3] = {0.0, 0.0, 0.0};
    double q[3] = {0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
        const double c = (double)counts[i];
        const double er = (double)eloc[2 * i], ei = (double)eloc[2 * i + 1];
        a[0] += c * er;
        a[1] += c * ei;
        a[2] += c * (er * er + ei * ei);
        q[0] += c;
        if (ga_e) {
            ga_e[i] = (float)(2.0 * c * er);
            gp_e[i] = (float)(2.0 * c * ei);
            ga_w[i] = (float)c;
        }
    }
    block_sum3_f64(a, 3, red);
    block_sum3_f64(q, 1, red);
    if (threadIdx.x == 0) { sums[0] = a[0]; sums[1] = a[1]; sums[2] = a[2]; sums[3] = q[0]; }
}

// ---------------------------------------------------------------- Adam
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi; v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// ---------------------------------------------------------------- outer-product gradients
__device__ __forceinline__ bool made_mask(int kind, int o, int i, int n) {
    if (kind == 0) return true;
    const int dn = n - 1;
    if (kind == 1) return i < (o % dn) + 1;              // input t feeds hidden o iff t < deg(o)
    if (kind == 2) return (i % dn) <= (o % dn);           // deg(i) <= deg(o)
    return (i % dn) + 1 < o + 1;                          // output o <- hidden i iff deg(i) < o+1
}

constexpr int OG_T = 32;   // output/input tile
__global__ void __launch_bounds__(256)
outer_grad_kernel(const float* __restrict__ delta, int64_t ld_d, const float* __restrict__ act,
                  int64_t ld_a, int64_t B, int out_dim, int in_dim, int mask_kind, int n_mask,
                  float* __restrict__ dW, float* __restrict__ db) {
    __shared__ float sd[OG_T][OG_T + 1];
    __shared__ float sa[OG_T][OG_T + 1];
    const int o0 = blockIdx.y * OG_T, i0 = blockIdx.x * OG_T;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // ty: 0..7
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float bacc = 0.f;
    for (int64_t b0 = 0; b0 < B; b0 += OG_T) {
        for (int r = ty; r < OG_T; r += 8) {
            const int64_t b = b0 + r;
            sd[r][tx] = (b < B && o0 + tx < out_dim) ? delta[b * ld_d + o0 + tx] : 0.f;
            sa[r][tx] = (b < B && i0 + tx < in_dim) ? act[b * ld_a + i0 + tx] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < OG_T; ++r) {
            const float a = sa[r][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += sd[r][ty * 4 + q] * a;
            if (ty == 0 && blockIdx.x == 0) bacc += sd[r][tx];
        }
        __syncthreads();
    }
    const int i = i0 + tx;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int o = o0 + ty * 4 + q;
        if (o < out_dim && i < in_dim && made_mask(mask_kind, o, i, n_mask))
            dW[(int64_t)o * in_dim + i] += acc[q];
    }
    if (db && ty == 0 && blockIdx.x == 0 && o0 + tx < out_dim) db[o0 + tx] += bacc;
}

}  // namespace

int launch_scan_i32(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
    scan_kernel<int32_t><<<1, SCAN_T, 0, s>>>(in, n, nullptr, out);
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_scan_i64(const int64_t* in, int64_t n_max, const int64_t* n_dev, int64_t* out,
                    cudaStream_t s) {
    scan_kernel<int64_t><<<1, SCAN_T, 0, s>>>(in, n_max, n_dev, out);
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_energy_stats(const float* eloc, const int64_t* counts, int64_t B, double* stats,
                        float* g_abs, float* g_phase, cudaStream_t s) {
    ProfScope ps("energy_stats", s);
    stats_kernel<<<1, 1024, 0, s>>>(eloc, counts, B, stats, g_abs, g_phase);
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_energy_sums(const float* eloc, const int64_t* counts, int64_t B, double* sums, float* ga_e,
                       float* gp_e, float* ga_w, cudaStream_t s) {
    sums_kernel<<<1, 1024, 0, s>>>(eloc, counts, B, sums, ga_e, gp_e, ga_w);
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int step, float lr,
                float b1, float b2, float eps, cudaStream_t s) {
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, step)));
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
    ProfScope ps("adam", s);
    adam_kernel<<<grid, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    NQS_LAUNCHED();
    return NQS_OK;
}

int launch_outer_grad(const float* delta, int64_t ld_d, const float* act, int64_t ld_a,
                      int64_t B, int out_dim, int in_dim, int mask_kind, int n_mask, float* dW,
                      float* db, cudaStream_t s) {
    if (out_dim <= 0) return NQS_OK;
    dim3 grid((unsigned)std::max(1, (in_dim + OG_T - 1) / OG_T), (unsigned)((out_dim + OG_T - 1) / OG_T));
    outer_grad_kernel<<<grid, 256, 0, s>>>(delta, ld_d, act, ld_a, B, out_dim, in_dim, mask_kind,
                                           n_mask, dW, db);
    NQS_LAUNCHED();
    return NQS_OK;
}

}  // namespace nqs
