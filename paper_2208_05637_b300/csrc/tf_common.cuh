// Device helpers shared by the transformer forward (transformer.cu) and backward
// (tf_backward.cu): LayerNorm, the FP32 SIMT GEMM, causal attention and small math helpers.
// Everything sits in an unnamed namespace, so each translation unit gets its own copy.
#pragma once

#include <cuda_bf16.h>

#include "nqs_internal.h"

namespace nqs {
namespace {

constexpr float LN_EPS = 1e-5f;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
}

__device__ __forceinline__ float logsig(float v) { return fminf(v, 0.f) - log1pf(expf(-fabsf(v))); }

__device__ __forceinline__ float gelu_tanh(float x) {
    const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
    return 0.5f * x * (1.f + tanhf(u));
}

template <class T>
__device__ __forceinline__ void store_act(T* p, float v);
template <>
__device__ __forceinline__ void store_act<float>(float* p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_act<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Storage of a GEMM input activation (row `row` of a matrix of `width` columns):
//   ACT_F32     fp32
//   ACT_BF16    bf16 (round to nearest even)
//   ACT_BF16X2  two bf16 numbers hi = bf16(v), lo = bf16(v - hi): row stride 2*width, hi in
//               columns [0, width), lo in [width, 2*width) -- the compensated tensor-core form
//   ACT_F32_Q1  fp32 holding bf16(v)            (backward recompute of ACT_BF16 models)
//   ACT_F32_Q2  fp32 holding hi + lo            (backward recompute of ACT_BF16X2 models)
enum { ACT_F32 = 0, ACT_BF16 = 1, ACT_BF16X2 = 2, ACT_F32_Q1 = 3, ACT_F32_Q2 = 4 };

template <int MODE>
__device__ __forceinline__ void store_mode(void* base, int64_t row, int width, int col, float v) {
    if (MODE == ACT_F32) {
        reinterpret_cast<float*>(base)[row * width + col] = v;
    } else if (MODE == ACT_BF16) {
        reinterpret_cast<__nv_bfloat16*>(base)[row * width + col] = __float2bfloat16_rn(v);
    } else if (MODE == ACT_BF16X2) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(base) + row * 2 * width;
        b[col] = hi;
        b[width + col] = lo;
    } else if (MODE == ACT_F32_Q1) {
        reinterpret_cast<float*>(base)[row * width + col] = __bfloat162float(__float2bfloat16_rn(v));
    } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const float h = __bfloat162float(hi);
        reinterpret_cast<float*>(base)[row * width + col] = h + __bfloat162float(__float2bfloat16_rn(v - h));
    }
}

// ---------------------------------------------------------------- embedding + first LayerNorm
// One warp per row (sequence r, position t).  Writes h (fp32) and a = LN1_0(h) (T_ACT).
template <int MODE, int DPL>   // DPL = d / 32 values per lane
__global__ void __launch_bounds__(256)
embed_ln_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
                int64_t R, int T, float* __restrict__ h, void* __restrict__ a) {
    const int d = mc.hidden;
    const int lane = threadIdx.x & 31;
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= R * T) return;
    const int64_t r = row / T;
    const int t = (int)(row % T);
    const int tok = t == 0 ? 2 : (int)((bits[r] >> mc.order[t - 1]) & 1ull);
    float v[DPL];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        v[i] = P[mc.tok_emb + tok * d + j] + P[mc.pos_emb + t * d + j];
        s += v[i];
    }
    const float mu = warp_sum(s) / d;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) { const float c = v[i] - mu; q += c * c; }
    const float rstd = rsqrtf(warp_sum(q) / d + LN_EPS);
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        h[row * d + j] = v[i];
        store_mode<MODE>(a, row, d, j, (v[i] - mu) * rstd * P[mc.ln1_g[0] + j] + P[mc.ln1_b[0] + j]);
    }
}

// LayerNorm of h rows into a (T_ACT), one warp per row.
template <int MODE, int DPL>
__global__ void __launch_bounds__(256)
layernorm_kernel(const float* __restrict__ h, int64_t M, int d, const float* __restrict__ g,
                 const float* __restrict__ b, void* __restrict__ a) {
    const int lane = threadIdx.x & 31;
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    float v[DPL];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) { v[i] = h[row * d + lane + 32 * i]; s += v[i]; }
    const float mu = warp_sum(s) / d;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) { const float c = v[i] - mu; q += c * c; }
    const float rstd = rsqrtf(warp_sum(q) / d + LN_EPS);
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        store_mode<MODE>(a, row, d, j, (v[i] - mu) * rstd * g[j] + b[j]);
    }
}

// ---------------------------------------------------------------- FP32 SIMT GEMM
// C[M,N] (epilogue) A[M,K] . B^T with B = W[N][K] (NT) or B = W[K][N] (NN, for dX = dY . W).
// 64x64 tile, K step 16, 256 threads with 4x4 outputs each.
constexpr int SG_BM = 64, SG_BN = 64, SG_BK = 16;

template <class T_A, bool NN, int EPI, class T_C>
__global__ void __launch_bounds__(256)
sgemm_kernel(const T_A* __restrict__ A, const float* __restrict__ W, const float* __restrict__ bias,
             T_C* __restrict__ C, int64_t M, int N, int K) {
    __shared__ float As[SG_BK][SG_BM + 4];
    __shared__ float Bs[SG_BK][SG_BN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * SG_BM;
    const int n0 = blockIdx.x * SG_BN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += SG_BK) {
        // A tile: 64 rows x 16 k
        for (int i = threadIdx.x; i < SG_BM * SG_BK; i += 256) {
            const int mm = i / SG_BK, kk = i % SG_BK;
            const int64_t gm = m0 + mm;
            const int gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? (float)A[gm * K + gk] : 0.f;
        }
        for (int i = threadIdx.x; i < SG_BN * SG_BK; i += 256) {
            int nn, kk;
            if (NN) { kk = i / SG_BN; nn = i % SG_BN; }
            else    { nn = i / SG_BK; kk = i % SG_BK; }
            const int gn = n0 + nn, gk = k0 + kk;
            float w = 0.f;
            if (gn < N && gk < K) w = NN ? W[(int64_t)gk * N + gn] : W[(int64_t)gn * K + gk];
            Bs[kk][nn] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SG_BK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { av[i] = As[kk][ty * 4 + i]; bv[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx * 4 + j;
            if (gn >= N) continue;
            float v = acc[i][j] + (bias ? bias[gn] : 0.f);
            T_C* dst = C + gm * N + gn;
            if (EPI == TF_EPI_GELU) store_act(dst, gelu_tanh(v));
            else if (EPI == TF_EPI_RESID) store_act(dst, (float)*dst + v);
            else if (EPI == TF_EPI_ACCUM) store_act(dst, (float)*dst + acc[i][j]);
            else store_act(dst, v);
        }
    }
}

// ---------------------------------------------------------------- causal attention
// One CTA per (sequence, head): scores S = Q K^T / sqrt(dh) with the causal mask, row softmax,
// O = P V.  qkv rows hold [q | k | v] (3d floats).  T <= 64, dh in {16, 32}.
template <int MODE>
__global__ void __launch_bounds__(128)
attention_kernel(const float* __restrict__ qkv, int T, int d, int dh, void* __restrict__ o) {
    __shared__ float q[64][33], k[64][33], v[64][33];
    __shared__ float p[64][65];
    const int64_t r = blockIdx.x;
    const int hd = blockIdx.y;
    const float scale = rsqrtf((float)dh);
    for (int i = threadIdx.x; i < T * dh; i += blockDim.x) {
        const int t = i / dh, j = i % dh;
        const float* row = qkv + (r * T + t) * (int64_t)(3 * d);
        q[t][j] = row[hd * dh + j];
        k[t][j] = row[d + hd * dh + j];
        v[t][j] = row[2 * d + hd * dh + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
        const int t = i / T, u = i % T;
        float s = -INFINITY;
        if (u <= t) {
            s = 0.f;
            for (int j = 0; j < dh; ++j) s = fmaf(q[t][j], k[u][j], s);
            s *= scale;
        }
        p[t][u] = s;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = warp; t < T; t += blockDim.x >> 5) {
        float mx = -INFINITY;
        for (int u = lane; u <= t; u += 32) mx = fmaxf(mx, p[t][u]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        float s = 0.f;
        for (int u = lane; u <= t; u += 32) { const float e = expf(p[t][u] - mx); p[t][u] = e; s += e; }
        s = warp_sum(s);
        const float inv = 1.f / s;
        for (int u = lane; u <= t; u += 32) p[t][u] *= inv;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * dh; i += blockDim.x) {
        const int t = i / dh, j = i % dh;
        float acc = 0.f;
        for (int u = 0; u <= t; ++u) acc = fmaf(p[t][u], v[u][j], acc);
        store_mode<MODE>(o, r * T + t, d, hd * dh + j, acc);
    }
}

// Causal attention, one CTA per sequence (looping over sequences) with one warp per head.  The
// sequence's whole [T x 3d] q|k|v block is copied row by row with coalesced loads into shared
// memory (row stride 3d + 4 floats: 16-byte aligned rows, so keys and values are read as
// float4 broadcasts); lane l of warp h owns query rows l and l + 32 of head h and runs an online
// (streaming) softmax over keys 0..t, accumulating P V in registers; the [T x d] output is staged
// in shared memory and written back as whole rows.  DH = head size.
template <int MODE, int DH>
__global__ void __launch_bounds__(256)
attention_seq_kernel(const float* __restrict__ qkv, int64_t R, int T, int d, int H, void* __restrict__ o) {
    extern __shared__ __align__(16) float att_sm[];
    const int ldq = 3 * d + 4, ldo = d + 1;
    float* X = att_sm;                 // [T][3d+4]
    float* O = att_sm + T * ldq;       // [T][d+1]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const float scale = rsqrtf((float)DH);
    for (int64_t r = blockIdx.x; r < R; r += gridDim.x) {
        const float* src = qkv + r * T * (int64_t)(3 * d);
        for (int t = warp; t < T; t += nw)
            for (int c = lane; c < 3 * d; c += 32) X[t * ldq + c] = src[(int64_t)t * 3 * d + c];
        __syncthreads();
        const int hd = warp;
        for (int t = lane; t < T; t += 32) {
            float q[DH], acc[DH];
#pragma unroll
            for (int j = 0; j < DH; ++j) { q[j] = X[t * ldq + hd * DH + j] * scale; acc[j] = 0.f; }
            float m = -INFINITY, ssum = 0.f;
            for (int u = 0; u <= t; ++u) {
                const float4* kr = reinterpret_cast<const float4*>(X + u * ldq + d + hd * DH);
                const float4* vr = reinterpret_cast<const float4*>(X + u * ldq + 2 * d + hd * DH);
                float sc = 0.f;
#pragma unroll
                for (int j4 = 0; j4 < DH / 4; ++j4) {
                    const float4 k4 = kr[j4];
                    sc = fmaf(q[4 * j4 + 0], k4.x, sc);
                    sc = fmaf(q[4 * j4 + 1], k4.y, sc);
                    sc = fmaf(q[4 * j4 + 2], k4.z, sc);
                    sc = fmaf(q[4 * j4 + 3], k4.w, sc);
                }
                const float mn = fmaxf(m, sc);
                const float corr = expf(m - mn);      // 0 on the first key (m = -inf)
                const float e = expf(sc - mn);
                ssum = ssum * corr + e;
#pragma unroll
                for (int j4 = 0; j4 < DH / 4; ++j4) {
                    const float4 v4 = vr[j4];
                    acc[4 * j4 + 0] = fmaf(e, v4.x, acc[4 * j4 + 0] * corr);
                    acc[4 * j4 + 1] = fmaf(e, v4.y, acc[4 * j4 + 1] * corr);
                    acc[4 * j4 + 2] = fmaf(e, v4.z, acc[4 * j4 + 2] * corr);
                    acc[4 * j4 + 3] = fmaf(e, v4.w, acc[4 * j4 + 3] * corr);
                }
                m = mn;
            }
            const float inv = 1.f / ssum;
#pragma unroll
            for (int j = 0; j < DH; ++j) O[t * ldo + hd * DH + j] = acc[j] * inv;
        }
        __syncthreads();
        for (int t = warp; t < T; t += nw)
            for (int c = lane; c < d; c += 32) store_mode<MODE>(o, r * T + t, d, c, O[t * ldo + c]);
        __syncthreads();
    }
}

template <int MODE>
inline cudaError_t launch_attention(const float* qkv, int64_t R, int T, int d, int H, void* o, cudaStream_t s) {
    const int dh = d / H;
    const size_t smem = (size_t)(T * (3 * d + 4) + T * (d + 1)) * sizeof(float);
    const unsigned grid = (unsigned)std::min<int64_t>(R, (int64_t)num_sms() * 8);
    if (dh == 16) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(attention_seq_kernel<MODE, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attention_seq_kernel<MODE, 16><<<grid, H * 32, smem, s>>>(qkv, R, T, d, H, o);
    } else {
        if (smem > 48 * 1024) cudaFuncSetAttribute(attention_seq_kernel<MODE, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attention_seq_kernel<MODE, 32><<<grid, H * 32, smem, s>>>(qkv, R, T, d, H, o);
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace nqs
