// Decoder-only transformer wavefunction (used by the larger workloads; not in the paper) in
// layer-wise kernels over a compact activation buffer of R sequences x T positions.
//
//   tokens     [BOS, x_order[0], ..., x_order[T-2]]        (token ids 2, then bits 0/1)
//   h          tok_emb[token] + pos_emb[t]
//   block l    h += Wo . attn(LN1(h))  ;  h += W2 . gelu(W1 . LN2(h))      (pre-LayerNorm)
//   heads      logit_t = LNf(h_t) . head_w + head_b[t];  phase = LNf(h_{n-2}) . phase_w + phase_b
//   log f      1/2 sum_t log pihat_t(x_t) (Hamming-weight constraint as for MADE) + i phase[sel]
//
// Every GEMM is C[M, N] = A[M, K] . W[N, K]^T (+ bias, + epilogue) with M = R*T rows; the four
// block GEMMs run in FP32 on CUDA cores (this file) or in BF16 on the tensor cores
// (tc_gemm.cu, precision NQS_PREC_BF16).  Attention (T <= 64, head size 16/32) runs per
// (sequence, head) on CUDA cores in FP32.  The last kernel applies LNf, the heads and the
// constraint and, for the local energy, multiplies the row's coefficient sum S by
// exp(log|f(x')| - log|f(x)|) e^{i (phi(x') - phi(x))} -- the ratio-weighted reduction is fused
// into the network's epilogue; a per-sample TwoSum pass adds the rows of each sample.
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

// ---------------------------------------------------------------- embedding + first LayerNorm
// One warp per row (sequence r, position t).  Writes h (fp32) and a = LN1_0(h) (T_ACT).
template <class T_ACT, int DPL>   // DPL = d / 32 values per lane
__global__ void __launch_bounds__(256)
embed_ln_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
                int64_t R, int T, float* __restrict__ h, T_ACT* __restrict__ a) {
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
        store_act(a + row * d + j, (v[i] - mu) * rstd * P[mc.ln1_g[0] + j] + P[mc.ln1_b[0] + j]);
    }
}

// LayerNorm of h rows into a (T_ACT), one warp per row.
template <class T_ACT, int DPL>
__global__ void __launch_bounds__(256)
layernorm_kernel(const float* __restrict__ h, int64_t M, int d, const float* __restrict__ g,
                 const float* __restrict__ b, T_ACT* __restrict__ a) {
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
        store_act(a + row * d + j, (v[i] - mu) * rstd * g[j] + b[j]);
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
template <class T_ACT>
__global__ void __launch_bounds__(128)
attention_kernel(const float* __restrict__ qkv, int T, int d, int dh, T_ACT* __restrict__ o) {
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
        store_act(o + (r * T + t) * (int64_t)d + hd * dh + j, acc);
    }
}

// ---------------------------------------------------------------- heads and constraint
// One warp per sequence.  mode 0: (log|f|, phi) per sequence; mode 1: local-energy
// contribution of an x' row; mode 2: sampler conditional at position k = T-1.
struct HeadArgs {
    int mode;
    float* la;                 // mode 0
    float* ph;
    const uint64_t* xsample;   // mode 1: the samples of the chunk
    const float* la_x;
    const float* ph_x;
    const int64_t* seg;        // mode 1: row offsets per sample (stride seg_stride), nseg samples
    int64_t seg_stride, nseg, row0;
    const float4* S;
    float2* contrib;
    float* p_out;              // mode 2
    uint64_t* thr;
    float* trace;
};

template <int DPL>
__global__ void __launch_bounds__(256)
heads_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
             const float* __restrict__ h, int64_t R, int T, HeadArgs args) {
    const int d = mc.hidden;
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= R) return;
    const uint64_t x = bits[r];
    float hw[DPL], g[DPL], bb[DPL];
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        hw[i] = P[mc.head_w + j]; g[i] = P[mc.lnf_g + j]; bb[i] = P[mc.lnf_b + j];
    }
    auto lnf_row = [&](int t, float (&y)[DPL]) {
        const float* row = h + (r * T + t) * (int64_t)d;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) { y[i] = row[lane + 32 * i]; s += y[i]; }
        const float mu = warp_sum(s) / d;
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) { const float c = y[i] - mu; q += c * c; }
        const float rstd = rsqrtf(warp_sum(q) / d + LN_EPS);
#pragma unroll
        for (int i = 0; i < DPL; ++i) y[i] = (y[i] - mu) * rstd * g[i] + bb[i];
    };
    if (args.mode == 2) {
        const int k = T - 1;
        int ones0 = 0, ones1 = 0;
        for (int t = 0; t < k; ++t) {
            const int b = (int)((x >> mc.order[t]) & 1ull);
            if (mc.order[t] & 1) ones1 += b; else ones0 += b;
        }
        const int sp = mc.order[k] & 1;
        const int c = sp ? ones1 : ones0;
        const int need = sp ? mc.n_dn : mc.n_up;
        float p;
        if (c + mc.after[k] < need) p = 1.f;
        else if (c >= need) p = 0.f;
        else {
            float y[DPL];
            lnf_row(k, y);
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < DPL; ++i) a = fmaf(y[i], hw[i], a);
            a = warp_sum(a) + P[mc.head_b + k];
            p = 1.f / (1.f + expf(-a));
        }
        if (lane == 0) {
            args.p_out[r] = p;
            args.thr[r] = (uint64_t)(p * 4294967296.0f);
            if (args.trace) args.trace[r] = p;
        }
        return;
    }
    // full log psi over all n positions
    float acc = 0.f, err = 0.f;
    int ones0 = 0, ones1 = 0;
    bool bad = false;
    float phase = 0.f;
    for (int t = 0; t < mc.n; ++t) {
        const int sp = mc.order[t] & 1;
        const int b = (int)((x >> mc.order[t]) & 1ull);
        const int c = sp ? ones1 : ones0;
        const int need = sp ? mc.n_dn : mc.n_up;
        const bool f1 = c + mc.after[t] < need, f0 = c >= need;
        if (f1) bad |= (b == 0);
        else if (f0) bad |= (b == 1);
        if (!(f1 || f0) || t == mc.n - 2) {
            float y[DPL];
            lnf_row(t, y);
            if (!(f1 || f0)) {
                float a = 0.f;
#pragma unroll
                for (int i = 0; i < DPL; ++i) a = fmaf(y[i], hw[i], a);
                a = warp_sum(a) + P[mc.head_b + t];
                const float lp = logsig(b ? a : -a);
                if (mc.compensated) two_sum_acc(acc, err, lp); else acc += lp;
            }
            if (t == mc.n - 2) {
                const int sel = (int)(((x >> mc.order[mc.n - 2]) & 1ull) * 2 + ((x >> mc.order[mc.n - 1]) & 1ull));
                float a = 0.f;
#pragma unroll
                for (int i = 0; i < DPL; ++i) a = fmaf(y[i], P[mc.phase_w + sel * d + lane + 32 * i], a);
                phase = warp_sum(a) + P[mc.phase_b + sel];
            }
        }
        if (sp) ones1 += b; else ones0 += b;
    }
    const float la = bad ? -INFINITY : 0.5f * (acc + err);
    if (lane != 0) return;
    if (args.mode == 0) {
        args.la[r] = la;
        args.ph[r] = phase;
        return;
    }
    // mode 1: row r of the chunk belongs to the sample whose segment contains row0 + r
    const int64_t grow = args.row0 + r;
    int64_t lo = 0, hi = args.nseg - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (args.seg[mid * args.seg_stride] <= grow) lo = mid; else hi = mid - 1;
    }
    const float4 s4 = args.S[grow];
    const float sre = s4.x + s4.y, sim = s4.z + s4.w;
    float cr = sre, ci = sim;
    if (x != args.xsample[lo]) {
        const float mag = expf(la - args.la_x[lo]);
        float sn, cs;
        sincosf(phase - args.ph_x[lo], &sn, &cs);
        const float rr = mag * cs, ri = mag * sn;
        cr = sre * rr - sim * ri;
        ci = sre * ri + sim * rr;
    }
    args.contrib[grow] = make_float2(cr, ci);
}

// Per-sample sum of the row contributions (TwoSum), one CTA per sample.
__global__ void __launch_bounds__(128)
segment_sum_kernel(const int64_t* __restrict__ seg, int64_t seg_stride, int64_t nseg,
                   const float2* __restrict__ contrib, int compensated, float* __restrict__ eloc) {
    __shared__ float red[4][128];
    for (int64_t i = blockIdx.x; i < nseg; i += gridDim.x) {
        const int64_t r0 = seg[i * seg_stride], r1 = seg[(i + 1) * seg_stride];
        float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const float2 c = contrib[r];
            if (compensated) { two_sum_acc(re, re_e, c.x); two_sum_acc(im, im_e, c.y); }
            else { re += c.x; im += c.y; }
        }
        red[0][threadIdx.x] = re; red[1][threadIdx.x] = re_e;
        red[2][threadIdx.x] = im; red[3][threadIdx.x] = im_e;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) {
                float a = red[0][threadIdx.x], ae = red[1][threadIdx.x] + red[1][threadIdx.x + st];
                two_sum_acc(a, ae, red[0][threadIdx.x + st]);
                red[0][threadIdx.x] = a; red[1][threadIdx.x] = ae;
                float b = red[2][threadIdx.x], be = red[3][threadIdx.x] + red[3][threadIdx.x + st];
                two_sum_acc(b, be, red[2][threadIdx.x + st]);
                red[2][threadIdx.x] = b; red[3][threadIdx.x] = be;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            eloc[2 * i] = red[0][0] + red[1][0];
            eloc[2 * i + 1] = red[2][0] + red[3][0];
        }
        __syncthreads();
    }
}

// fp32 master weights -> bf16 working copies of the four block GEMM matrices
__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

inline int blocks_for(int64_t rows, int per) { return (int)((rows + per - 1) / per); }

template <class F>
int with_dpl(int d, F&& f) {
    switch (d / 32) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 8: return f(std::integral_constant<int, 8>{});
        default:
            set_error("transformer d_model must be 32, 64, 128 or 256");
            return NQS_ERR_UNSUPPORTED;
    }
}

}  // namespace

// ====================================================================== host side
int64_t tf_seq_capacity(const ModelConst& mc) {
    // about 256 MB of activations: h, a, qkv, o (fp32) and the 4d MLP buffer
    const int64_t per_seq = (int64_t)mc.n * mc.hidden * 10 * 4;
    int64_t R = 64;
    while (R * 2 * per_seq <= (256ll << 20) && R < 8192) R *= 2;
    return R;
}

void tf_layout(Carver& c, const ModelConst& mc, int64_t R, TfBufs& b) {
    const int64_t M = R * mc.n, d = mc.hidden;
    b.R = R;
    b.h = c.take<float>(M * d);
    b.a = c.take<float>(M * d);          // fp32 or bf16 view
    b.qkv = c.take<float>(M * 3 * d);
    b.o = c.take<float>(M * d);          // fp32 or bf16 view
    b.mid = c.take<float>(M * 4 * d);    // fp32 or bf16 view
}

int tf_gemm(const ModelConst& mc, const TfWeights& w, int which, int layer, const void* A,
            void* C, int64_t M, int N, int K, int epi, const float* bias, cudaStream_t s) {
    if (mc.precision == NQS_PREC_BF16)
        return tc_gemm_bf16((const __nv_bfloat16*)A, w.bf16 + w.bf16_off[layer][which], bias, C,
                            M, N, K, epi, s);
    const float* W = w.fp32 + w.fp32_off[layer][which];
    dim3 grid((unsigned)((N + SG_BN - 1) / SG_BN), (unsigned)((M + SG_BM - 1) / SG_BM));
    const float* Af = (const float*)A;
    float* Cf = (float*)C;
    switch (epi) {
        case TF_EPI_STORE: sgemm_kernel<float, false, TF_EPI_STORE, float><<<grid, 256, 0, s>>>(Af, W, bias, Cf, M, N, K); break;
        case TF_EPI_GELU: sgemm_kernel<float, false, TF_EPI_GELU, float><<<grid, 256, 0, s>>>(Af, W, bias, Cf, M, N, K); break;
        case TF_EPI_RESID: sgemm_kernel<float, false, TF_EPI_RESID, float><<<grid, 256, 0, s>>>(Af, W, bias, Cf, M, N, K); break;
        default: set_error("bad GEMM epilogue"); return NQS_ERR_INVALID_ARG;
    }
    NQS_LAUNCHED();
    return NQS_OK;
}

int tf_prepare_weights(const ModelConst& mc, const float* P, TfWeights& w, cudaStream_t s) {
    w.fp32 = P;
    for (int l = 0; l < mc.layers; ++l) {
        w.fp32_off[l][TF_WQKV] = mc.wqkv[l];
        w.fp32_off[l][TF_WO] = mc.wo[l];
        w.fp32_off[l][TF_W1] = mc.w1[l];
        w.fp32_off[l][TF_W2] = mc.w2[l];
    }
    if (mc.precision != NQS_PREC_BF16) return NQS_OK;
    if (!w.bf16) { set_error("bf16 weight buffer missing"); return NQS_ERR_INVALID_ARG; }
    const int64_t d = mc.hidden;
    int64_t off = 0;
    const int64_t sizes[4] = {3 * d * d, d * d, 4 * d * d, 4 * d * d};
    for (int l = 0; l < mc.layers; ++l) {
        for (int q = 0; q < 4; ++q) {
            w.bf16_off[l][q] = off;
            const int64_t n = sizes[q];
            const int grid = (int)std::min<int64_t>((n + 255) / 256, 1024);
            to_bf16_kernel<<<grid, 256, 0, s>>>(P + w.fp32_off[l][q], reinterpret_cast<__nv_bfloat16*>(w.bf16) + off, n);
            NQS_LAUNCHED();
            off += (n + 127) & ~int64_t(127);   // 256-byte aligned matrices
        }
    }
    return NQS_OK;
}

int64_t tf_bf16_weight_elems(const ModelConst& mc) {
    const int64_t d = mc.hidden;
    int64_t total = 0;
    const int64_t sizes[4] = {3 * d * d, d * d, 4 * d * d, 4 * d * d};
    for (int l = 0; l < mc.layers; ++l)
        for (int q = 0; q < 4; ++q) total += (sizes[q] + 127) & ~int64_t(127);
    return total;
}

// Forward of R sequences over their first T positions, leaving the final residual stream in
// b.h.  `bits` are the R configurations.
int tf_forward(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
               int64_t R, int T, TfBufs& b, cudaStream_t s) {
    const int d = mc.hidden, dh = d / mc.heads;
    const int64_t M = R * T;
    const bool bf = mc.precision == NQS_PREC_BF16;
    return with_dpl(d, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        const int rows_per_cta = 8;
        if (bf) embed_ln_kernel<__nv_bfloat16, DPL><<<blocks_for(M, rows_per_cta), 256, 0, s>>>(mc, P, bits, R, T, b.h, (__nv_bfloat16*)b.a);
        else embed_ln_kernel<float, DPL><<<blocks_for(M, rows_per_cta), 256, 0, s>>>(mc, P, bits, R, T, b.h, b.a);
        NQS_LAUNCHED();
        for (int l = 0; l < mc.layers; ++l) {
            {
                ProfScope ps("tf_gemm", s);
                NQS_TRY(tf_gemm(mc, w, TF_WQKV, l, b.a, b.qkv, M, 3 * d, d, TF_EPI_STORE, P + mc.bqkv[l], s));
            }
            {
                ProfScope ps("tf_attention", s);
                dim3 g((unsigned)R, (unsigned)mc.heads);
                if (bf) attention_kernel<__nv_bfloat16><<<g, 128, 0, s>>>(b.qkv, T, d, dh, (__nv_bfloat16*)b.o);
                else attention_kernel<float><<<g, 128, 0, s>>>(b.qkv, T, d, dh, b.o);
                NQS_LAUNCHED();
            }
            {
                ProfScope ps("tf_gemm", s);
                NQS_TRY(tf_gemm(mc, w, TF_WO, l, b.o, b.h, M, d, d, TF_EPI_RESID, P + mc.bo[l], s));
            }
            if (bf) layernorm_kernel<__nv_bfloat16, DPL><<<blocks_for(M, 8), 256, 0, s>>>(b.h, M, d, P + mc.ln2_g[l], P + mc.ln2_b[l], (__nv_bfloat16*)b.a);
            else layernorm_kernel<float, DPL><<<blocks_for(M, 8), 256, 0, s>>>(b.h, M, d, P + mc.ln2_g[l], P + mc.ln2_b[l], b.a);
            NQS_LAUNCHED();
            {
                ProfScope ps("tf_gemm", s);
                NQS_TRY(tf_gemm(mc, w, TF_W1, l, b.a, b.mid, M, 4 * d, d, TF_EPI_GELU, P + mc.b1[l], s));
                NQS_TRY(tf_gemm(mc, w, TF_W2, l, b.mid, b.h, M, d, 4 * d, TF_EPI_RESID, P + mc.b2[l], s));
            }
            if (l + 1 < mc.layers) {
                if (bf) layernorm_kernel<__nv_bfloat16, DPL><<<blocks_for(M, 8), 256, 0, s>>>(b.h, M, d, P + mc.ln1_g[l + 1], P + mc.ln1_b[l + 1], (__nv_bfloat16*)b.a);
                else layernorm_kernel<float, DPL><<<blocks_for(M, 8), 256, 0, s>>>(b.h, M, d, P + mc.ln1_g[l + 1], P + mc.ln1_b[l + 1], b.a);
                NQS_LAUNCHED();
            }
        }
        return NQS_OK;
    });
}

int tf_heads(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t R, int T,
             const TfBufs& b, const HeadArgsHost& ha, cudaStream_t s) {
    HeadArgs a{};
    a.mode = ha.mode; a.la = ha.la; a.ph = ha.ph; a.xsample = ha.xsample; a.la_x = ha.la_x;
    a.ph_x = ha.ph_x; a.seg = ha.seg; a.seg_stride = ha.seg_stride; a.nseg = ha.nseg;
    a.row0 = ha.row0; a.S = ha.S; a.contrib = ha.contrib; a.p_out = ha.p_out; a.thr = ha.thr;
    a.trace = ha.trace;
    return with_dpl(mc.hidden, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        ProfScope ps("tf_heads", s);
        heads_kernel<DPL><<<blocks_for(R, 8), 256, 0, s>>>(mc, P, bits, b.h, R, T, a);
        NQS_LAUNCHED();
        return NQS_OK;
    });
}

int tf_segment_sum(const int64_t* seg, int64_t seg_stride, int64_t nseg, const float2* contrib,
                   int compensated, float* eloc, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>(nseg, (int64_t)num_sms() * 8);
    segment_sum_kernel<<<grid, 128, 0, s>>>(seg, seg_stride, nseg, contrib, compensated, eloc);
    NQS_LAUNCHED();
    return NQS_OK;
}

int tf_logpsi(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
              int64_t B, float* la, float* ph, TfBufs& b, cudaStream_t s) {
    for (int64_t lo = 0; lo < B; lo += b.R) {
        const int64_t R = std::min(b.R, B - lo);
        NQS_TRY(tf_forward(mc, P, w, bits + lo, R, mc.n, b, s));
        HeadArgsHost ha{};
        ha.mode = 0; ha.la = la + lo; ha.ph = ph + lo;
        NQS_TRY(tf_heads(mc, P, bits + lo, R, mc.n, b, ha, s));
    }
    return NQS_OK;
}

}  // namespace nqs
