// Fused incremental step of the transformer sampler (Sec. 3.2: the conditional of position k
// given the prefix x_<k, with the keys and values of earlier positions cached) for the d_model-64,
// four-head models in the bf16 tensor-core forms.  One CTA takes 16 prefixes through the whole
// step: embedding and LayerNorm, per block the QKV projection (stored into the cache slab of
// step k), causal attention over the cached keys of the prefix's ancestors, output projection
// and residual, LayerNorm, GELU MLP and residual, then the final LayerNorm, the output head and
// the Hamming-weight constraint, leaving p(x_k = 1 | x_<k), the draw threshold and the trace.
//
// The four GEMMs run on mma.sync m16n8k16 (bf16 in, fp32 accumulate) with the operand forms of
// the batched forward: activations as bf16 (ACT_BF16) or as hi | lo bf16 pairs against the
// duplicated [W | W] weights (ACT_BF16X2), so the arithmetic is that of the multi-kernel step
// up to the fp32 summation order.  The weights stream from L2 straight into B fragments.
#include "tf_common.cuh"

namespace nqs {
namespace {

constexpr int FS_RB = 16;                       // prefixes per CTA: one m16 row tile
constexpr int FS_WARPS = 16;
constexpr int FS_THREADS = FS_WARPS * 32;
constexpr int FS_D = 64, FS_H = 4, FS_DH = 16, FS_F = 4 * FS_D;
// shared-memory layout; padded row strides keep the m16n8 fragment accesses conflict-free
constexpr int FS_LDH = FS_D + 8;                // fp32: residual stream h, split-K partials
constexpr int FS_LDQ = 3 * FS_D + 8;            // fp32: q | k | v of position k
constexpr int FS_LDA = 2 * FS_D + 8;            // bf16: GEMM operand of width d (hi | lo)
constexpr int FS_LDG = 2 * FS_F + 8;            // bf16: MLP hidden operand (hi | lo)
constexpr int FS_MAXK = 64;                     // positions (n <= 64)
constexpr int FS_OFF_H = 0;
constexpr int FS_OFF_RED = FS_OFF_H + FS_RB * FS_LDH * 4;
constexpr int FS_OFF_Q = FS_OFF_RED + FS_RB * FS_LDH * 4;
constexpr int FS_OFF_A = FS_OFF_Q + FS_RB * FS_LDQ * 4;
constexpr int FS_OFF_G = FS_OFF_A + FS_RB * FS_LDA * 2;
constexpr int FS_OFF_E = FS_OFF_G + FS_RB * FS_LDG * 2;          // per warp: e[head][key]
constexpr int FS_OFF_S = FS_OFF_E + FS_WARPS * FS_H * FS_MAXK * 4;   // per warp: key slots
constexpr int FS_SMEM = FS_OFF_S + FS_WARPS * FS_MAXK * 4;

struct FsArgs {
    const float* P;
    const __nv_bfloat16* wb;                    // bf16 weights (duplicated rows when compensated)
    int64_t woff[TF_MAX_LAYERS][4];             // element offsets of Wqkv, Wo, W1, W2 in wb
    const uint64_t* bits;
    int64_t R;                                  // rows of the pass (the kernel stops at *Udev)
    int k;                                      // position
    float* kv;                                  // QKV slabs of every layer and step
    int64_t cap;
    const int32_t* anc;                         // anc[r * n + j]: slot of r's ancestor at step j
    const int64_t* Udev;
    float* p_out;
    uint64_t* thr;
    float* trace;
};

__device__ __forceinline__ void fs_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t fs_lds32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// C (16 x 8) += A[:, k0:k1] . W[n0:n0+8, k0:k1]^T: A in shared memory (bf16, row stride lda), W
// row-major in global memory (bf16, row stride ldw).  Fragment layouts of m16n8k16: A rows g and
// g + 8, columns 2q, 2q + 1 and 2q + 8, 2q + 9 of the k-step; B column g, the same k; C rows g,
// g + 8, columns 2q, 2q + 1 (g = lane / 4, q = lane % 4).
template <int KSTEPS>
__device__ __forceinline__ void fs_tile(const __nv_bfloat16* sA, int lda, const __nv_bfloat16* W, int64_t ldw,
                                        int n0, int k0, float (&c)[4], int lane) {
    const int g = lane >> 2, q = lane & 3;
    const uint32_t* wr = reinterpret_cast<const uint32_t*>(W + (int64_t)(n0 + g) * ldw + k0 + 2 * q);
    const __nv_bfloat16* a0 = sA + g * lda + k0 + 2 * q;
    const __nv_bfloat16* a1 = a0 + 8 * lda;
    uint32_t b[KSTEPS][2];
#pragma unroll
    for (int s = 0; s < KSTEPS; ++s) { b[s][0] = __ldg(wr + 8 * s); b[s][1] = __ldg(wr + 8 * s + 4); }
#pragma unroll
    for (int s = 0; s < KSTEPS; ++s) {
        const uint32_t a[4] = {fs_lds32(a0 + 16 * s), fs_lds32(a1 + 16 * s), fs_lds32(a0 + 16 * s + 8),
                               fs_lds32(a1 + 16 * s + 8)};
        fs_mma(c, a, b[s][0], b[s][1]);
    }
}

// (v0, v1) into columns c, c + 1 of row r of a GEMM operand of width K: bf16, or hi at c and
// lo = bf16(v - hi) at K + c.
template <int MODE>
__device__ __forceinline__ void fs_put2(__nv_bfloat16* A, int lda, int K, int r, int c, float v0, float v1) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v0, v1);
    *reinterpret_cast<__nv_bfloat162*>(A + r * lda + c) = hh;
    if (MODE == ACT_BF16X2) {
        const float2 hf = __bfloat1622float2(hh);
        *reinterpret_cast<__nv_bfloat162*>(A + r * lda + K + c) = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    }
}

// LayerNorm of row r of h (warp-wide, two columns a lane) as in the batched kernels.
__device__ __forceinline__ float2 fs_ln(const float* sH, int r, const float* __restrict__ g,
                                        const float* __restrict__ b, int lane) {
    const int c0 = 2 * lane;
    const float2 x = *reinterpret_cast<const float2*>(sH + r * FS_LDH + c0);
    const float inv_d = 1.f / (float)FS_D;
    const float mu = warp_sum(x.x + x.y) * inv_d;
    const float d0 = x.x - mu, d1 = x.y - mu;
    float t = d0 * d0;
    t += d1 * d1;
    const float rstd = rsqrtf(fmaf(warp_sum(t), inv_d, LN_EPS));
    const float2 gg = *reinterpret_cast<const float2*>(g + c0), bb = *reinterpret_cast<const float2*>(b + c0);
    return make_float2(d0 * rstd * gg.x + bb.x, d1 * rstd * gg.y + bb.y);
}

template <int MODE>
__global__ void __launch_bounds__(FS_THREADS, 1)
tf_step_fused_kernel(ModelConst mc, FsArgs A) {
    extern __shared__ __align__(16) uint8_t fs_smem[];
    float* sH = reinterpret_cast<float*>(fs_smem + FS_OFF_H);
    float* sRed = reinterpret_cast<float*>(fs_smem + FS_OFF_RED);
    float* sQ = reinterpret_cast<float*>(fs_smem + FS_OFF_Q);
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(fs_smem + FS_OFF_A);
    __nv_bfloat16* sG = reinterpret_cast<__nv_bfloat16*>(fs_smem + FS_OFF_G);
    float* sE = reinterpret_cast<float*>(fs_smem + FS_OFF_E);
    int32_t* sS = reinterpret_cast<int32_t*>(fs_smem + FS_OFF_S);
    constexpr int KX = MODE == ACT_BF16X2 ? 2 : 1;       // operand width factor (hi | lo)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, q4 = lane & 3;
    const int64_t U = min(*A.Udev, A.R);
    const int64_t row0 = (int64_t)blockIdx.x * FS_RB;
    if (row0 >= U) return;
    const int n = mc.n, k = A.k;
    const float* P = A.P;
    const int64_t slab_stride = A.cap * 3 * FS_D;
    const int r = warp;                                  // the row of the row-wise phases
    const int64_t grow = row0 + r;
    const bool live = grow < U;
    const uint64_t x = A.bits[live ? grow : U - 1];

    // ---- embedding and LayerNorm 1 of block 0
    {
        const int tok = k == 0 ? 2 : (int)((x >> mc.order[k - 1]) & 1ull);
        const int c0 = 2 * lane;
        const float2 e = *reinterpret_cast<const float2*>(P + mc.tok_emb + tok * FS_D + c0);
        const float2 p = *reinterpret_cast<const float2*>(P + mc.pos_emb + k * FS_D + c0);
        *reinterpret_cast<float2*>(sH + r * FS_LDH + c0) = make_float2(e.x + p.x, e.y + p.y);
        __syncwarp();
        const float2 y = fs_ln(sH, r, P + mc.ln1_g[0], P + mc.ln1_b[0], lane);
        fs_put2<MODE>(sA, FS_LDA, FS_D, r, c0, y.x, y.y);
    }
    __syncthreads();

    for (int l = 0; l < mc.layers; ++l) {
        float* slab0 = A.kv + (int64_t)l * n * slab_stride;   // step-0 slab of this layer
        // ---- qkv = a . Wqkv^T + bqkv: 24 n-tiles over the 16 warps
        {
            const __nv_bfloat16* W = A.wb + A.woff[l][TF_WQKV];
            const float* bq = P + mc.bqkv[l];
            for (int t = warp; t < 3 * FS_D / 8; t += FS_WARPS) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                fs_tile<KX * FS_D / 16>(sA, FS_LDA, W, KX * FS_D, 8 * t, 0, c, lane);
                const int col = 8 * t + 2 * q4;
                const float2 bb = *reinterpret_cast<const float2*>(bq + col);
                *reinterpret_cast<float2*>(sQ + g * FS_LDQ + col) = make_float2(c[0] + bb.x, c[1] + bb.y);
                *reinterpret_cast<float2*>(sQ + (g + 8) * FS_LDQ + col) = make_float2(c[2] + bb.x, c[3] + bb.y);
            }
        }
        __syncthreads();
        // the step-k slab rows of the live prefixes (coalesced float4 copies)
        {
            float* dst = slab0 + (int64_t)k * slab_stride + row0 * (3 * FS_D);
            const int nrow = (int)min((int64_t)FS_RB, U - row0);
            for (int i = threadIdx.x; i < nrow * (3 * FS_D / 4); i += FS_THREADS) {
                const int rr = i / (3 * FS_D / 4), c4 = i - rr * (3 * FS_D / 4);
                reinterpret_cast<float4*>(dst + rr * 3 * FS_D)[c4] = reinterpret_cast<const float4*>(sQ + rr * FS_LDQ)[c4];
            }
        }
        // ---- attention of row r over keys j = 0..k (ancestor slots for j < k, own row at k)
        {
            float* e_s = sE + warp * FS_H * FS_MAXK;
            int32_t* s_s = sS + warp * FS_MAXK;
            const float scale = rsqrtf((float)FS_DH) * 1.4426950408889634f;   // log2 domain
            float sc[2][FS_H];
            const float* kr[2] = {nullptr, nullptr};
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int j = lane + 32 * h2;
                if (j > k) continue;
                if (j < k) {
                    int64_t slot = live ? A.anc[grow * n + j] : 0;
                    slot = slot < 0 ? 0 : (slot >= A.cap ? A.cap - 1 : slot);
                    s_s[j] = (int32_t)slot;
                    kr[h2] = slab0 + (int64_t)j * slab_stride + slot * (3 * FS_D) + FS_D;
                } else {
                    kr[h2] = sQ + r * FS_LDQ + FS_D;
                }
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll
                for (int hd = 0; hd < FS_H; ++hd) {
                    if (!kr[h2]) { sc[h2][hd] = -INFINITY; continue; }
                    const float4* k4 = reinterpret_cast<const float4*>(kr[h2] + hd * FS_DH);
                    const float4* q4p = reinterpret_cast<const float4*>(sQ + r * FS_LDQ + hd * FS_DH);
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int j4 = 0; j4 < FS_DH / 4; ++j4) {
                        const float4 kk = k4[j4], qq = q4p[j4];
                        float& sp = (j4 & 1) ? s1 : s0;
                        sp = fmaf(qq.x * scale, kk.x, sp);
                        sp = fmaf(qq.y * scale, kk.y, sp);
                        sp = fmaf(qq.z * scale, kk.z, sp);
                        sp = fmaf(qq.w * scale, kk.w, sp);
                    }
                    sc[h2][hd] = s0 + s1;
                }
            }
            float inv_l[FS_H];
#pragma unroll
            for (int hd = 0; hd < FS_H; ++hd) {
                float m = fmaxf(sc[0][hd], sc[1][hd]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                const float e0 = kr[0] ? exp2f(sc[0][hd] - m) : 0.f;
                const float e1 = kr[1] ? exp2f(sc[1][hd] - m) : 0.f;
                if (kr[0]) e_s[hd * FS_MAXK + lane] = e0;
                if (kr[1]) e_s[hd * FS_MAXK + lane + 32] = e1;
                inv_l[hd] = 1.f / warp_sum(e0 + e1);
            }
            __syncwarp();
            // weighted values: lane takes output columns 2 lane, 2 lane + 1 (head lane / 8)
            const int c0 = 2 * lane, hd = lane >> 3;
            const float* ev = e_s + hd * FS_MAXK;
            float ox = 0.f, oy = 0.f;
            int j = 0;
            for (; j + 4 <= k; j += 4) {
                float2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    v[u] = *reinterpret_cast<const float2*>(slab0 + (int64_t)(j + u) * slab_stride +
                                                            (int64_t)s_s[j + u] * (3 * FS_D) + 2 * FS_D + c0);
#pragma unroll
                for (int u = 0; u < 4; ++u) { ox = fmaf(ev[j + u], v[u].x, ox); oy = fmaf(ev[j + u], v[u].y, oy); }
            }
            for (; j < k; ++j) {
                const float2 v = *reinterpret_cast<const float2*>(slab0 + (int64_t)j * slab_stride +
                                                                  (int64_t)s_s[j] * (3 * FS_D) + 2 * FS_D + c0);
                ox = fmaf(ev[j], v.x, ox);
                oy = fmaf(ev[j], v.y, oy);
            }
            {
                const float2 v = *reinterpret_cast<const float2*>(sQ + r * FS_LDQ + 2 * FS_D + c0);
                ox = fmaf(ev[k], v.x, ox);
                oy = fmaf(ev[k], v.y, oy);
            }
            float il = inv_l[0];
#pragma unroll
            for (int h2 = 1; h2 < FS_H; ++h2) il = hd == h2 ? inv_l[h2] : il;
            fs_put2<MODE>(sA, FS_LDA, FS_D, r, c0, ox * il, oy * il);
        }
        __syncthreads();
        // ---- h += o . Wo^T + bo: 8 n-tiles, K split over two warp halves
        {
            const __nv_bfloat16* W = A.wb + A.woff[l][TF_WO];
            const int t = warp & 7, kh = warp >> 3;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            fs_tile<KX * FS_D / 32>(sA, FS_LDA, W, KX * FS_D, 8 * t, kh * (KX * FS_D / 2), c, lane);
            const int col = 8 * t + 2 * q4;
            if (kh) {
                *reinterpret_cast<float2*>(sRed + g * FS_LDH + col) = make_float2(c[0], c[1]);
                *reinterpret_cast<float2*>(sRed + (g + 8) * FS_LDH + col) = make_float2(c[2], c[3]);
            }
            __syncthreads();
            if (!kh) {
                const float2 bb = *reinterpret_cast<const float2*>(P + mc.bo[l] + col);
                const float2 p0 = *reinterpret_cast<const float2*>(sRed + g * FS_LDH + col);
                const float2 p1 = *reinterpret_cast<const float2*>(sRed + (g + 8) * FS_LDH + col);
                float2* h0 = reinterpret_cast<float2*>(sH + g * FS_LDH + col);
                float2* h1 = reinterpret_cast<float2*>(sH + (g + 8) * FS_LDH + col);
                h0->x += (c[0] + p0.x) + bb.x; h0->y += (c[1] + p0.y) + bb.y;
                h1->x += (c[2] + p1.x) + bb.x; h1->y += (c[3] + p1.y) + bb.y;
            }
        }
        __syncthreads();
        // ---- LayerNorm 2
        {
            const float2 y = fs_ln(sH, r, P + mc.ln2_g[l], P + mc.ln2_b[l], lane);
            fs_put2<MODE>(sA, FS_LDA, FS_D, r, 2 * lane, y.x, y.y);
        }
        __syncthreads();
        // ---- hidden = GELU(a . W1^T + b1): 32 n-tiles, two per warp
        {
            const __nv_bfloat16* W = A.wb + A.woff[l][TF_W1];
            const float* b1 = P + mc.b1[l];
#pragma unroll
            for (int tt = 0; tt < 2; ++tt) {
                const int t = warp + FS_WARPS * tt;
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                fs_tile<KX * FS_D / 16>(sA, FS_LDA, W, KX * FS_D, 8 * t, 0, c, lane);
                const int col = 8 * t + 2 * q4;
                const float2 bb = *reinterpret_cast<const float2*>(b1 + col);
                fs_put2<MODE>(sG, FS_LDG, FS_F, g, col, gelu_tanh(c[0] + bb.x), gelu_tanh(c[1] + bb.y));
                fs_put2<MODE>(sG, FS_LDG, FS_F, g + 8, col, gelu_tanh(c[2] + bb.x), gelu_tanh(c[3] + bb.y));
            }
        }
        __syncthreads();
        // ---- h += hidden . W2^T + b2: 8 n-tiles, K split over two warp halves
        {
            const __nv_bfloat16* W = A.wb + A.woff[l][TF_W2];
            const int t = warp & 7, kh = warp >> 3;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            fs_tile<KX * FS_F / 32>(sG, FS_LDG, W, KX * FS_F, 8 * t, kh * (KX * FS_F / 2), c, lane);
            const int col = 8 * t + 2 * q4;
            if (kh) {
                *reinterpret_cast<float2*>(sRed + g * FS_LDH + col) = make_float2(c[0], c[1]);
                *reinterpret_cast<float2*>(sRed + (g + 8) * FS_LDH + col) = make_float2(c[2], c[3]);
            }
            __syncthreads();
            if (!kh) {
                const float2 bb = *reinterpret_cast<const float2*>(P + mc.b2[l] + col);
                const float2 p0 = *reinterpret_cast<const float2*>(sRed + g * FS_LDH + col);
                const float2 p1 = *reinterpret_cast<const float2*>(sRed + (g + 8) * FS_LDH + col);
                float2* h0 = reinterpret_cast<float2*>(sH + g * FS_LDH + col);
                float2* h1 = reinterpret_cast<float2*>(sH + (g + 8) * FS_LDH + col);
                h0->x += (c[0] + p0.x) + bb.x; h0->y += (c[1] + p0.y) + bb.y;
                h1->x += (c[2] + p1.x) + bb.x; h1->y += (c[3] + p1.y) + bb.y;
            }
        }
        __syncthreads();
        if (l + 1 < mc.layers) {
            const float2 y = fs_ln(sH, r, P + mc.ln1_g[l + 1], P + mc.ln1_b[l + 1], lane);
            fs_put2<MODE>(sA, FS_LDA, FS_D, r, 2 * lane, y.x, y.y);
            __syncthreads();
        }
    }

    // ---- output head: p(x_k = 1 | x_<k) under the Hamming-weight constraint
    int ones0 = 0, ones1 = 0;
    for (int t = 0; t < k; ++t) {
        const int b = (int)((x >> mc.order[t]) & 1ull);
        if (mc.order[t] & 1) ones1 += b; else ones0 += b;
    }
    const int sp = mc.order[k] & 1;
    const int cnt = sp ? ones1 : ones0;
    const int need = sp ? mc.n_dn : mc.n_up;
    float p;
    if (cnt + mc.after[k] < need) {
        p = 1.f;
    } else if (cnt >= need) {
        p = 0.f;
    } else {
        const float2 y = fs_ln(sH, r, P + mc.lnf_g, P + mc.lnf_b, lane);
        const float2 hw = *reinterpret_cast<const float2*>(P + mc.head_w + 2 * lane);
        const float a = warp_sum(fmaf(y.x, hw.x, y.y * hw.y)) + P[mc.head_b + k];
        p = 1.f / (1.f + expf(-a));
    }
    if (lane == 0 && live) {
        A.p_out[grow] = p;
        A.thr[grow] = (uint64_t)(p * 4294967296.0f);
        if (A.trace) A.trace[grow] = p;
    }
}

}  // namespace

bool tf_step_fused_supported(const ModelConst& mc) {
    return mc.precision == NQS_PREC_BF16 && mc.hidden == FS_D && mc.heads == FS_H && mc.n <= FS_MAXK &&
           mc.layers <= TF_MAX_LAYERS;
}

int tf_step_fused(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits, int64_t R,
                  int k, const TfStepCache& kc, float* p_out, uint64_t* thr, float* trace, cudaStream_t s) {
    if (!tf_step_fused_supported(mc)) { set_error("fused sampler step: unsupported model shape"); return NQS_ERR_UNSUPPORTED; }
    if (R > kc.cap) { set_error("sampler step: more prefixes than the cache holds"); return NQS_ERR_CAPACITY; }
    if (R <= 0) return NQS_OK;
    // the dynamic shared memory limit is raised once per device (the first call is an eager one,
    // before any captured launch)
    static int configured_device = -1;
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (configured_device != dev) {
        NQS_CK(cudaFuncSetAttribute(tf_step_fused_kernel<ACT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, FS_SMEM));
        NQS_CK(cudaFuncSetAttribute(tf_step_fused_kernel<ACT_BF16X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, FS_SMEM));
        configured_device = dev;
    }
    FsArgs a{};
    a.P = P;
    a.wb = reinterpret_cast<const __nv_bfloat16*>(w.bf16);
    for (int l = 0; l < mc.layers; ++l)
        for (int m = 0; m < 4; ++m) a.woff[l][m] = w.bf16_off[l][m];
    a.bits = bits; a.R = R; a.k = k;
    a.kv = kc.kv; a.cap = kc.cap; a.anc = kc.anc; a.Udev = kc.Udev;
    a.p_out = p_out; a.thr = thr; a.trace = trace;
    const unsigned grid = (unsigned)((R + FS_RB - 1) / FS_RB);
    const int64_t M = R;
    const double flops = 2.0 * M * mc.layers * (double)FS_D * (3 * FS_D + FS_D + 2 * FS_F) * (mc.compensated ? 2 : 1);
    ProfScope ps("tf_step_fused", s, flops, 0.0);
    if (mc.compensated) tf_step_fused_kernel<ACT_BF16X2><<<grid, FS_THREADS, FS_SMEM, s>>>(mc, a);
    else tf_step_fused_kernel<ACT_BF16><<<grid, FS_THREADS, FS_SMEM, s>>>(mc, a);
    NQS_LAUNCHED();
    return NQS_OK;
}

}  // namespace nqs
