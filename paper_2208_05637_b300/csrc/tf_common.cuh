// Device helpers shared by the transformer forward (transformer.cu) and backward
// (tf_backward.cu): LayerNorm, the FP32 SIMT GEMM, causal attention and small math helpers.
// Everything sits in an unnamed namespace, so each translation unit gets its own copy.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

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

// GELU, tanh form: 0.5 x (1 + tanh(u)), u = sqrt(2/pi) (x + 0.044715 x^3).  Evaluated through
// tanh(u) = 2 sigmoid(2u) - 1 as x / (1 + exp(-2u)), with exp(-2u) = exp2(x (c1 + c2 x^2)),
// c1 = -2 sqrt(2/pi) log2(e), c2 = 0.044715 c1, on the hardware approximations ex2.approx and
// rcp.approx (PTX ISA: ~2 ulp each).  Limits: for large x the exponential flushes to 0 and the
// result is x; for very negative x it is +inf and the result is (-)0.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_tanh(float x) {
    constexpr float c1 = -2.f * 0.7978845608028654f * 1.4426950408889634f;
    constexpr float c2 = c1 * 0.044715f;
    const float e = ex2_approx(x * fmaf(c2, x * x, c1));
    return x * rcp_approx(1.f + e);
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

// ---------------------------------------------------------------- LayerNorm kernels
// One warp per LN_ROWS rows (their loads issued together), lane l holding the DPL = d / 32
// contiguous columns [l * DPL, (l + 1) * DPL); eight warps per CTA.
constexpr int LN_ROWS = 4;
constexpr int LN_ROWS_PER_CTA = 8 * LN_ROWS;
inline int ln_grid(int64_t rows) { return (int)((rows + LN_ROWS_PER_CTA - 1) / LN_ROWS_PER_CTA); }

template <int DPL>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[DPL]) {
    if (DPL == 1) {
        v[0] = p[0];
    } else if (DPL == 2) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        v[0] = x.x; v[1] = x.y;
    } else {
#pragma unroll
        for (int i = 0; i < DPL; i += 4) {
            const float4 x = *reinterpret_cast<const float4*>(p + i);
            v[i] = x.x; v[i + 1] = x.y; v[i + 2] = x.z; v[i + 3] = x.w;
        }
    }
}

template <int N>
__device__ __forceinline__ void store_floats(float* p, const float* v) {
    if (N == 1) {
        p[0] = v[0];
    } else if (N == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 4) *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
}

template <int N>
__device__ __forceinline__ void store_bf16s(__nv_bfloat16* p, const __nv_bfloat16* v) {
    if (N == 1) {
        p[0] = v[0];
    } else if (N == 2) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __halves2bfloat162(v[0], v[1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            uint2 u;
            u.x = (uint32_t)__bfloat16_as_ushort(v[i]) | ((uint32_t)__bfloat16_as_ushort(v[i + 1]) << 16);
            u.y = (uint32_t)__bfloat16_as_ushort(v[i + 2]) | ((uint32_t)__bfloat16_as_ushort(v[i + 3]) << 16);
            *reinterpret_cast<uint2*>(p + i) = u;
        }
    }
}

// N consecutive columns [col0, col0 + N) of row `row` in the storage form of MODE (store_mode).
template <int MODE, int N>
__device__ __forceinline__ void store_mode_vec(void* base, int64_t row, int width, int col0, const float* v) {
    if (MODE == ACT_F32 || MODE == ACT_F32_Q1 || MODE == ACT_F32_Q2) {
        float w[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (MODE == ACT_F32) {
                w[j] = v[j];
            } else if (MODE == ACT_F32_Q1) {
                w[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
            } else {
                const float hv = __bfloat162float(__float2bfloat16_rn(v[j]));
                w[j] = hv + __bfloat162float(__float2bfloat16_rn(v[j] - hv));
            }
        }
        store_floats<N>(reinterpret_cast<float*>(base) + row * width + col0, w);
    } else {
        __nv_bfloat16 hi[N], lo[N];
        if (N >= 2) {
#pragma unroll
            for (int j = 0; j < N; j += 2) {   // packed conversions, two columns at a time
                const __nv_bfloat162 hh = __floats2bfloat162_rn(v[j], v[j + 1]);
                hi[j] = hh.x; hi[j + 1] = hh.y;
                if (MODE == ACT_BF16X2) {
                    const float2 hf = __bfloat1622float2(hh);
                    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[j] - hf.x, v[j + 1] - hf.y);
                    lo[j] = ll.x; lo[j + 1] = ll.y;
                }
            }
        } else {
            hi[0] = __float2bfloat16_rn(v[0]);
            if (MODE == ACT_BF16X2) lo[0] = __float2bfloat16_rn(v[0] - __bfloat162float(hi[0]));
        }
        const int64_t stride = MODE == ACT_BF16X2 ? 2 * (int64_t)width : width;
        __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(base) + row * stride + col0;
        store_bf16s<N>(b, hi);
        if (MODE == ACT_BF16X2) store_bf16s<N>(b + width, lo);
    }
}

// LayerNorm of LN_ROWS rows held by one warp (v[r] = row r's DPL values of this lane):
// two-pass mean and variance, then a = (v - mean) * rstd * g + b stored in MODE's form.
template <int MODE, int DPL>
__device__ __forceinline__ void ln_rows_store(float (&v)[LN_ROWS][DPL], const int64_t (&rows)[LN_ROWS], int64_t M,
                                              int d, int col0, const float* __restrict__ g,
                                              const float* __restrict__ b, void* __restrict__ a) {
    float gg[DPL], bb[DPL];
    load_row<DPL>(g + col0, gg);
    load_row<DPL>(b + col0, bb);
    float mu[LN_ROWS], q[LN_ROWS];
#pragma unroll
    for (int r = 0; r < LN_ROWS; ++r) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) s += v[r][i];
        mu[r] = s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < LN_ROWS; ++r) mu[r] += __shfl_xor_sync(0xffffffffu, mu[r], o);
    const float inv_d = 1.f / (float)d;   // d is a power of two: exact
#pragma unroll
    for (int r = 0; r < LN_ROWS; ++r) {
        mu[r] *= inv_d;
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) { const float c = v[r][i] - mu[r]; t += c * c; }
        q[r] = t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < LN_ROWS; ++r) q[r] += __shfl_xor_sync(0xffffffffu, q[r], o);
#pragma unroll
    for (int r = 0; r < LN_ROWS; ++r) {
        if (rows[r] >= M) continue;
        const float rstd = rsqrtf(fmaf(q[r], inv_d, LN_EPS));
        float y[DPL];
#pragma unroll
        for (int i = 0; i < DPL; ++i) y[i] = (v[r][i] - mu[r]) * rstd * gg[i] + bb[i];
        store_mode_vec<MODE, DPL>(a, rows[r], d, col0, y);
    }
}

// Embedding + first LayerNorm: rows (sequence r, position t = t0 + row % T) get
// h = tok_emb[token] + pos_emb[t] (fp32) and a = LN1_0(h) (MODE).
template <int MODE, int DPL>   // DPL = d / 32 values per lane
__global__ void __launch_bounds__(256)
embed_ln_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
                int64_t R, int T, int t0, float* __restrict__ h, void* __restrict__ a) {
    const int d = mc.hidden;
    const int lane = threadIdx.x & 31, col0 = lane * DPL;
    const int64_t M = R * T;
    const int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * LN_ROWS;
    if (base >= M) return;
    float v[LN_ROWS][DPL];
    int64_t rows[LN_ROWS];
    // (sequence, position) of the first row, then advanced row by row (rows < 2^31)
    int sq = (int)(base / T), tp = (int)(base - (int64_t)sq * T);
#pragma unroll
    for (int r = 0; r < LN_ROWS; ++r) {
        rows[r] = base + r;
        if (r > 0 && ++tp == T) { tp = 0; ++sq; }
        const int sqc = rows[r] < M ? sq : (int)((M - 1) / T);
        const int t = t0 + (rows[r] < M ? tp : (int)((M - 1) % T));
        const int tok = t == 0 ? 2 : (int)((bits[sqc] >> mc.order[t - 1]) & 1ull);
        float e[DPL], p[DPL];
        load_row<DPL>(P + mc.tok_emb + tok * d + col0, e);
        load_row<DPL>(P + mc.pos_emb + t * d + col0, p);
#pragma unroll
        for (int i = 0; i < DPL; ++i) v[r][i] = e[i] + p[i];
        if (rows[r] < M) store_floats<DPL>(h + rows[r] * d + col0, v[r]);
    }
    ln_rows_store<MODE, DPL>(v, rows, M, d, col0, P + mc.ln1_g[0], P + mc.ln1_b[0], a);
}

// LayerNorm of h rows into a (MODE).
template <int MODE, int DPL>
__global__ void __launch_bounds__(256)
layernorm_kernel(const float* __restrict__ h, int64_t M, int d, const float* __restrict__ g,
                 const float* __restrict__ b, void* __restrict__ a) {
    const int lane = threadIdx.x & 31, col0 = lane * DPL;
    const int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * LN_ROWS;
    if (base >= M) return;
    float v[LN_ROWS][DPL];
    int64_t rows[LN_ROWS];
#pragma unroll
    for (int r = 0; r < LN_ROWS; ++r) {
        rows[r] = base + r;
        load_row<DPL>(h + (rows[r] < M ? rows[r] : M - 1) * d + col0, v[r]);
    }
    ln_rows_store<MODE, DPL>(v, rows, M, d, col0, g, b, a);
}

// ---------------------------------------------------------------- FP32 SIMT GEMM
// FP32 SIMT GEMM  C[M, N] (epilogue) = A[M, K] . W^T + bias  (W [N, K]; NN: A . W with W [K, N]).
// 128 x 64 output tile per CTA, 16-deep k-slices double-buffered in shared memory (the next
// slice is fetched into registers while the current one is multiplied); 256 threads, each with
// an 8 x 4 block of outputs fed by float4 shared-memory loads.
constexpr int SG_BM = 128, SG_BN = 64, SG_BK = 16;

template <class T_A, bool NN, int EPI, class T_C>
__global__ void __launch_bounds__(256)
sgemm_kernel(const T_A* __restrict__ A, const float* __restrict__ W, const float* __restrict__ bias,
             T_C* __restrict__ C, int64_t M, int N, int K) {
    __shared__ __align__(16) float As[2][SG_BK][SG_BM + 4];
    __shared__ __align__(16) float Bs[2][SG_BK][SG_BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;          // outputs: rows ty*8.., columns tx*4..
    const int64_t m0 = (int64_t)blockIdx.y * SG_BM;
    const int n0 = blockIdx.x * SG_BN;
    // global fetch roles: A rows (tid >> 2) and (tid >> 2) + 64, k quad (tid & 3);
    // W (NT) row tid >> 2, k quad tid & 3;  W (NN) k row tid >> 4, n quad tid & 15
    const int ar = tid >> 2, aq = tid & 3;
    float ra[2][4], rb[4];
    // four consecutive elements, as one float4 when in range and aligned (vec)
    auto load4 = [&](const auto* p, bool in0, bool all_in, bool vec_ok, float (&r)[4], int64_t stride_in) {
        if (all_in && vec_ok) {
            const float4 v = *reinterpret_cast<const float4*>(p);
            r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) r[j] = 0.f;
            if (in0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) r[j] = (j < stride_in) ? (float)p[j] : 0.f;
            }
        }
    };
    const bool avec = std::is_same<T_A, float>::value && (K & 3) == 0 && ((uintptr_t)A & 15) == 0;
    const bool wvec = NN ? ((N & 3) == 0 && ((uintptr_t)W & 15) == 0) : ((K & 3) == 0 && ((uintptr_t)W & 15) == 0);
    auto fetch = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gm = m0 + ar + 64 * h;
            const int gk = k0 + 4 * aq;
            load4(A + gm * K + gk, gm < M && gk < K, gm < M && gk + 3 < K, avec, ra[h], (int64_t)K - gk);
        }
        if (NN) {
            const int gk = k0 + (tid >> 4), gn = n0 + 4 * (tid & 15);
            load4(W + (int64_t)gk * N + gn, gk < K && gn < N, gk < K && gn + 3 < N, wvec, rb, (int64_t)N - gn);
        } else {
            const int gn = n0 + ar, gk = k0 + 4 * aq;
            load4(W + (int64_t)gn * K + gk, gn < N && gk < K, gn < N && gk + 3 < K, wvec, rb, (int64_t)K - gk);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) As[buf][4 * aq + j][ar + 64 * h] = ra[h][j];
        if (NN) {
            *reinterpret_cast<float4*>(&Bs[buf][tid >> 4][4 * (tid & 15)]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) Bs[buf][4 * aq + j][ar] = rb[j];
        }
    };
    float acc[8][4] = {};
    fetch(0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += SG_BK) {
        const bool more = k0 + SG_BK < K;
        if (more) fetch(k0 + SG_BK);
#pragma unroll
        for (int kk = 0; kk < SG_BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
            const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) {
            stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    const bool cvec = std::is_same<T_C, float>::value && (N & 3) == 0 && ((uintptr_t)C & 15) == 0;
    const int gn0 = n0 + tx * 4;
    float bj[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) bj[j] = (bias && gn0 + j < N) ? bias[gn0 + j] : 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gm = m0 + ty * 8 + i;
        if (gm >= M) continue;
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (EPI == TF_EPI_ACCUM) ? acc[i][j] : acc[i][j] + bj[j];
        T_C* dst = C + gm * N + gn0;
        if (cvec && gn0 + 3 < N) {
            float4* d4 = reinterpret_cast<float4*>(dst);
            float4 o = make_float4(v[0], v[1], v[2], v[3]);
            if (EPI == TF_EPI_RESID || EPI == TF_EPI_ACCUM) {
                const float4 y = *d4;
                o.x += y.x; o.y += y.y; o.z += y.z; o.w += y.w;
            } else if (EPI == TF_EPI_GELU) {
                o = make_float4(gelu_tanh(v[0]), gelu_tanh(v[1]), gelu_tanh(v[2]), gelu_tanh(v[3]));
            }
            *d4 = o;
            continue;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (gn0 + j >= N) continue;
            if (EPI == TF_EPI_GELU) store_act(dst + j, gelu_tanh(v[j]));
            else if (EPI == TF_EPI_RESID || EPI == TF_EPI_ACCUM) store_act(dst + j, (float)dst[j] + v[j]);
            else store_act(dst + j, v[j]);
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

// Sixteen consecutive columns [col0, col0 + 16) of row `row` in the storage form of MODE
// (see store_mode); col0 and width are multiples of 16.
template <int MODE>
__device__ __forceinline__ void store_mode16(void* base, int64_t row, int width, int col0, const float* v) {
    if (MODE == ACT_F32 || MODE == ACT_F32_Q1 || MODE == ACT_F32_Q2) {
        float w[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (MODE == ACT_F32) {
                w[j] = v[j];
            } else if (MODE == ACT_F32_Q1) {
                w[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
            } else {
                const float h = __bfloat162float(__float2bfloat16_rn(v[j]));
                w[j] = h + __bfloat162float(__float2bfloat16_rn(v[j] - h));
            }
        }
        float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(base) + row * width + col0);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_float4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    } else {
        __align__(16) __nv_bfloat16 hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            hi[j] = __float2bfloat16_rn(v[j]);
            if (MODE == ACT_BF16X2) lo[j] = __float2bfloat16_rn(v[j] - __bfloat162float(hi[j]));
        }
        const int64_t stride = MODE == ACT_BF16X2 ? 2 * (int64_t)width : width;
        uint4* dh = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(base) + row * stride + col0);
        dh[0] = reinterpret_cast<const uint4*>(hi)[0];
        dh[1] = reinterpret_cast<const uint4*>(hi)[1];
        if (MODE == ACT_BF16X2) {
            uint4* dl = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(base) + row * stride + width + col0);
            dl[0] = reinterpret_cast<const uint4*>(lo)[0];
            dl[1] = reinterpret_cast<const uint4*>(lo)[1];
        }
    }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Dot product of a query row with a key row from shared memory, as two interleaved partial
// sums (even and odd float4 pieces) for instruction-level parallelism.
template <int DH>
__device__ __forceinline__ float att_dot(const float (&q)[DH], const float4* __restrict__ k) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int j4 = 0; j4 < DH / 4; ++j4) {
        const float4 k4 = k[j4];
        float& sp = (j4 & 1) ? s1 : s0;
        sp = fmaf(q[4 * j4 + 0], k4.x, sp);
        sp = fmaf(q[4 * j4 + 1], k4.y, sp);
        sp = fmaf(q[4 * j4 + 2], k4.z, sp);
        sp = fmaf(q[4 * j4 + 3], k4.w, sp);
    }
    return s0 + s1;
}

// Online-softmax update of one row (reference max m, normaliser l, unnormalised output acc) by
// keys u and u+1 (scores s0, s1 in the log2 domain; value rows v0, v1), or by key u alone.  The
// reference moves only when some lane of the warp sees a score more than 2^8 above it (the
// weights exp2(s - m) then stay below 256 and the quotient acc / l is unchanged), so the
// rescaling of acc is skipped on most keys; all lanes of the warp call this together.
template <int DH, bool PAIR>
__device__ __forceinline__ void att_update(float s0, float s1, const float4* __restrict__ v0,
                                           const float4* __restrict__ v1, float (&acc)[DH], float& m, float& l) {
    const float smax = PAIR ? fmaxf(s0, s1) : s0;
    if (__any_sync(0xffffffffu, smax > m + 8.f)) {
        const float mn = fmaxf(m, smax);
        const float c = ex2_approx(m - mn);        // 0 on the first key (m = -inf)
        l *= c;
#pragma unroll
        for (int j = 0; j < DH; ++j) acc[j] *= c;
        m = mn;
    }
    const float e0 = ex2_approx(s0 - m);
    const float e1 = PAIR ? ex2_approx(s1 - m) : 0.f;
    l += PAIR ? e0 + e1 : e0;
#pragma unroll
    for (int j4 = 0; j4 < DH / 4; ++j4) {
        const float4 a = v0[j4];
        float x0 = fmaf(e0, a.x, acc[4 * j4 + 0]), x1 = fmaf(e0, a.y, acc[4 * j4 + 1]);
        float x2 = fmaf(e0, a.z, acc[4 * j4 + 2]), x3 = fmaf(e0, a.w, acc[4 * j4 + 3]);
        if (PAIR) {
            const float4 b = v1[j4];
            x0 = fmaf(e1, b.x, x0); x1 = fmaf(e1, b.y, x1); x2 = fmaf(e1, b.z, x2); x3 = fmaf(e1, b.w, x3);
        }
        acc[4 * j4 + 0] = x0; acc[4 * j4 + 1] = x1; acc[4 * j4 + 2] = x2; acc[4 * j4 + 3] = x3;
    }
}

// Keys [u0, u1) of the online softmax for query row qa, or for rows qa and qb sharing the key
// and value loads.
template <int DH, bool TWO>
__device__ __forceinline__ void attend_keys(const float* __restrict__ kv, int LU, int VOFF, int u0, int u1,
                                            const float (&qa)[DH], float (&aa)[DH], float& ma, float& la,
                                            const float (&qb)[DH], float (&ab)[DH], float& mb, float& lb) {
    int u = u0;
    // two keys per step for a single row; the two-row form keeps one key per step (registers)
    for (; !TWO && u + 1 < u1; u += 2) {
        const float4* k0 = reinterpret_cast<const float4*>(kv + u * LU);
        const float4* k1 = reinterpret_cast<const float4*>(kv + (u + 1) * LU);
        const float4* v0 = reinterpret_cast<const float4*>(kv + u * LU + VOFF);
        const float4* v1 = reinterpret_cast<const float4*>(kv + (u + 1) * LU + VOFF);
        att_update<DH, true>(att_dot<DH>(qa, k0), att_dot<DH>(qa, k1), v0, v1, aa, ma, la);
    }
    for (; u < u1; ++u) {
        const float4* k0 = reinterpret_cast<const float4*>(kv + u * LU);
        const float4* v0 = reinterpret_cast<const float4*>(kv + u * LU + VOFF);
        const float sa0 = att_dot<DH>(qa, k0);
        if (TWO) att_update<DH, false>(att_dot<DH>(qb, k0), 0.f, v0, v0, ab, mb, lb);
        att_update<DH, false>(sa0, 0.f, v0, v0, aa, ma, la);
    }
}

// Query row (scaled) into q and a zeroed accumulator, for attention_grp_kernel.
template <int DH>
__device__ __forceinline__ void att_load_q(const float* __restrict__ src, bool act, float scale, float (&q)[DH],
                                           float (&acc)[DH]) {
#pragma unroll
    for (int j4 = 0; j4 < DH / 4; ++j4) {
        const float4 x = act ? __ldg(reinterpret_cast<const float4*>(src) + j4) : make_float4(0.f, 0.f, 0.f, 0.f);
        q[4 * j4 + 0] = x.x * scale;
        q[4 * j4 + 1] = x.y * scale;
        q[4 * j4 + 2] = x.z * scale;
        q[4 * j4 + 3] = x.w * scale;
    }
#pragma unroll
    for (int j = 0; j < DH; ++j) acc[j] = 0.f;
}

// Normalised output row acc / l into columns [col0, col0 + DH) of row `row`.
template <int MODE, int DH>
__device__ __forceinline__ void att_store_row(float (&acc)[DH], float l, void* o, int64_t row, int d, int col0) {
    const float inv = 1.f / l;
#pragma unroll
    for (int j = 0; j < DH; ++j) acc[j] *= inv;
#pragma unroll
    for (int j0 = 0; j0 < DH; j0 += 16) store_mode16<MODE>(o, row, d, col0 + j0, acc + j0);
}

// Causal attention with lanes over (sequence, head) groups: a CTA stages the keys and values of
// S sequences in shared memory (cp.async), lane l of every warp serves group (s = l / H,
// h = l % H), and warp w takes the query-row pairs (p, T-1-p), p = w, w + warps, ...: the two
// rows cost T + 1 key steps together, so every warp does the same work and every loop is
// warp-uniform.  With DH = 16 the pair shares the key/value loads of keys 0..p.
// Shared layout per sequence (floats): row u at u*LU, K of head h at h*LH, V at H*LH + h*LH,
// LH = DH + 4, LU = 2*H*LH; sequence stride SS (padded by the host so that the eight lanes of a
// quarter-warp read distinct 16-byte bank groups).
constexpr int ATT_GRP_MAX_WARPS = 10;   // 320 threads, two CTAs per SM

template <int MODE, int DH>
__global__ void __launch_bounds__(ATT_GRP_MAX_WARPS * 32, 2)
attention_grp_kernel(const float* __restrict__ qkv, int64_t R, int T, int d, int H, int S, int SS,
                     void* __restrict__ o) {
    extern __shared__ __align__(16) float att_sm[];
    constexpr int LH = DH + 4;
    const int LU = 2 * H * LH, VOFF = H * LH;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    // scores in the log2 domain: q is scaled by log2(e) / sqrt(DH), weights are exp2(s - max)
    const float scale = rsqrtf((float)DH) * 1.4426950408889634f;
    const int ld = 3 * d;
    // staging: thread i copies float4 chunk cc = i % chunks_row of positions q = i / chunks_row,
    // q + rows_step, ... (q = s*T + u); the chunk's offsets are fixed per thread
    const int chunks_row = d / 2;                  // float4 chunks of K|V per position
    const int rows_step = blockDim.x / chunks_row;
    const int cc = threadIdx.x % chunks_row, q0 = threadIdx.x / chunks_row;
    const int kv = cc / (d / 4), wch = cc % (d / 4);
    const int soff = kv * VOFF + (wch / (DH / 4)) * LH + 4 * (wch % (DH / 4));
    const bool lane_ok = lane < S * H;
    const int ls = lane_ok ? lane / H : 0, lh = lane % H;
    const int64_t nbatch = (R + S - 1) / S;
    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x) {
        const int64_t r0 = b * S;
        const int sv = (int)((R - r0) < S ? (R - r0) : S);
        if (q0 < rows_step) {
            const float* src = qkv + (r0 * T) * (int64_t)ld + d + 4 * cc;
            int s_ = q0 / T, u = q0 % T;
            for (int q = q0; q < sv * T; q += rows_step) {
                cp_async16(att_sm + s_ * SS + u * LU + soff, src + (int64_t)q * ld);
                u += rows_step;
                while (u >= T) { u -= T; ++s_; }
            }
        }
        const bool act = lane_ok && ls < sv;
        const int64_t r = r0 + (act ? ls : 0);
        const float* kvs = att_sm + ls * SS + lh * LH;
        const int npairs = (T + 1) / 2;
        const bool share = DH <= 16;               // the pair shares its key/value loads
        float qa[DH], qb[DH], aa[DH], ab[DH];
        // the query rows of the warp's first pair load while the keys and values are staged
        if (warp < npairs) {
            att_load_q<DH>(qkv + (r * T + warp) * (int64_t)ld + lh * DH, act, scale, qa, aa);
            if (share) att_load_q<DH>(qkv + (r * T + T - 1 - warp) * (int64_t)ld + lh * DH, act, scale, qb, ab);
        }
        cp_async_wait_all();
        __syncthreads();
        for (int p = warp; p < npairs; p += nw) {
            const int ta = p, tb = T - 1 - p;
            if (p != warp) {
                att_load_q<DH>(qkv + (r * T + ta) * (int64_t)ld + lh * DH, act, scale, qa, aa);
                if (share) att_load_q<DH>(qkv + (r * T + tb) * (int64_t)ld + lh * DH, act, scale, qb, ab);
            }
            float ma = -INFINITY, la = 0.f, mb = -INFINITY, lb = 0.f;
            if (share && tb != ta) {
                // keys 0..ta serve both rows, then row tb runs on alone
                attend_keys<DH, true>(kvs, LU, VOFF, 0, ta + 1, qa, aa, ma, la, qb, ab, mb, lb);
                if (act) att_store_row<MODE, DH>(aa, la, o, r * T + ta, d, lh * DH);
                attend_keys<DH, false>(kvs, LU, VOFF, ta + 1, tb + 1, qb, ab, mb, lb, qa, aa, ma, la);
                if (act) att_store_row<MODE, DH>(ab, lb, o, r * T + tb, d, lh * DH);
            } else {
                attend_keys<DH, false>(kvs, LU, VOFF, 0, ta + 1, qa, aa, ma, la, qb, ab, mb, lb);
                if (act) att_store_row<MODE, DH>(aa, la, o, r * T + ta, d, lh * DH);
                if (tb != ta) {
                    att_load_q<DH>(qkv + (r * T + tb) * (int64_t)ld + lh * DH, act, scale, qa, aa);
                    ma = -INFINITY; la = 0.f;
                    attend_keys<DH, false>(kvs, LU, VOFF, 0, tb + 1, qa, aa, ma, la, qb, ab, mb, lb);
                    if (act) att_store_row<MODE, DH>(aa, la, o, r * T + tb, d, lh * DH);
                }
            }
        }
        __syncthreads();
    }
}

// Sequence stride (floats) of a grouped-attention shared layout whose sequences hold `base`
// floats: the padding (a multiple of four floats) that spreads the eight lanes of each
// quarter-warp over the most 16-byte bank groups when lanes l = (sequence l / H, head l % H)
// read the same position (head stride LH floats).
inline int grp_seq_stride(int base, int H, int LH, int S) {
    int best = base, best_cost = 1 << 30;
    for (int pad = 0; pad < 32; pad += 4) {
        int cost = 0;
        for (int q = 0; q < 4; ++q) {
            int used[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int worst = 0;
            for (int l = 8 * q; l < 8 * q + 8 && l < S * H; ++l) {
                const int addr = (l / H) * (base + pad) + (l % H) * LH;
                const int slot = (addr / 4) & 7;
                worst = std::max(worst, ++used[slot]);
            }
            cost += worst;
        }
        if (cost < best_cost) { best_cost = cost; best = base + pad; }
    }
    return best;
}
inline int attention_grp_stride(int T, int H, int DH, int S) { return grp_seq_stride(T * 2 * H * (DH + 4), H, DH + 4, S); }

template <int MODE>
inline cudaError_t launch_attention(const float* qkv, int64_t R, int T, int d, int H, void* o, cudaStream_t s) {
    const int dh = d / H;
    if (R <= 0) return cudaSuccess;
    // grouped kernel: as many sequences per CTA as fill the 32 lanes (or ~110 KB of shared
    // memory), when that keeps at least half of the lanes busy
    if (32 % H == 0) {
        const size_t seq_bytes = (size_t)T * 2 * H * (dh + 4) * sizeof(float) + 32 * sizeof(float);
        const int S = std::min<int>(32 / H, (int)((110 * 1024) / seq_bytes));
        if (S * H >= 16 && d / 2 <= ATT_GRP_MAX_WARPS * 32) {
            // the dynamic shared-memory limit is raised once per kernel and device (outside any
            // stream capture: the first launch of a shape is an eager one)
            static int configured16 = -1, configured32 = -1;
            int dev = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return e;
            int& cfg = dh == 16 ? configured16 : configured32;
            if (cfg != dev) {
                e = dh == 16 ? cudaFuncSetAttribute(attention_grp_kernel<MODE, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
                             : cudaFuncSetAttribute(attention_grp_kernel<MODE, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (e != cudaSuccess) return e;
                cfg = dev;
            }
            const int SS = attention_grp_stride(T, H, dh, S);
            const size_t smem = (size_t)S * SS * sizeof(float);
            // one warp per query-row pair, and at least one thread per float4 of a position's K|V
            const int warps = std::max(std::min((T + 1) / 2, ATT_GRP_MAX_WARPS), (d / 2 + 31) / 32);
            const int per_sm = std::max(1, (int)((228 * 1024) / (smem + 1024)));
            const int64_t nbatch = (R + S - 1) / S;
            const unsigned grid = (unsigned)std::min<int64_t>(nbatch, (int64_t)num_sms() * per_sm);
            if (dh == 16) attention_grp_kernel<MODE, 16><<<grid, warps * 32, smem, s>>>(qkv, R, T, d, H, S, SS, o);
            else attention_grp_kernel<MODE, 32><<<grid, warps * 32, smem, s>>>(qkv, R, T, d, H, S, SS, o);
            return cudaGetLastError();
        }
    }
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

// Weight conversions of every block in one launch: job j takes the rows x cols fp32 matrix at
// src and writes its bf16 values (dup: the [W | W] rows of the compensated GEMM) or, with
// f32_out, their bf16-rounded fp32 values; jobs are laid end to end in the element index.
struct WconvJob {
    const float* src;
    void* dst;
    int64_t start;      // first element index of the job
    int cols;
};
struct WconvList {
    WconvJob job[4 * TF_MAX_LAYERS];
    int njobs;
    int dup, f32_out;
    int64_t total;
};

__global__ void wconv_kernel(const __grid_constant__ WconvList L) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L.total; i += (int64_t)gridDim.x * blockDim.x) {
        int j = 0;
        while (j + 1 < L.njobs && L.job[j + 1].start <= i) ++j;
        const WconvJob& J = L.job[j];
        const int64_t e = i - J.start;
        const int64_t r = e / J.cols;
        const int k = (int)(e - r * J.cols);
        const __nv_bfloat16 v = __float2bfloat16_rn(J.src[e]);
        if (L.f32_out) {
            reinterpret_cast<float*>(J.dst)[e] = __bfloat162float(v);
        } else {
            __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(J.dst);
            const int64_t kk = L.dup ? 2 * (int64_t)J.cols : J.cols;
            dst[r * kk + k] = v;
            if (L.dup) dst[r * kk + J.cols + k] = v;
        }
    }
}

}  // namespace
}  // namespace nqs
