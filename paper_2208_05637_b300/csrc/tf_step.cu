// Fused incremental step of the transformer sampler (Section 4, Sampling: the conditional of
// position k given the prefix x_<k, with the keys and values of earlier positions cached) for the d_model-64,
// four-head models in the bf16 tensor-core forms.  One CTA takes 16 prefixes through the whole
// step: embedding and LayerNorm, per block the QKV projection (stored into the cache slab of
// step k), causal attention over the cached keys of the prefix's ancestors, output projection
// and residual, LayerNorm, GELU MLP and residual, then the final LayerNorm, the output head and
// the Hamming-weight constraint, leaving p(x_k = 1 | x_<k), the draw threshold and the trace.
//
// The four GEMMs run on mma.sync m16n8k16 (bf16 in, fp32 accumulate) with the operand forms of
// the batched forward: activations as bf16 (ACT_BF16) or as hi | lo bf16 pairs against the
// duplicated [W | W] weights (ACT_BF16X2), so the arithmetic is that of the multi-kernel step
// up to the fp32 summation order.  Each block's weights are staged in shared memory one group
// (Wqkv | Wo, W1 | W2) ahead of their use by asynchronous copies.
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
constexpr int FS_VB = 6;                        // value rows in flight per lane
constexpr int FS_LDW = FS_D + 8;                // bf16: staged Wqkv, Wo, W1 rows (K = d)
constexpr int FS_LDW2 = FS_F + 8;               // bf16: staged W2 rows (K = 4d)
constexpr int FS_OFF_WQKV = 0;                  // block weights staged in shared memory: Wqkv | Wo
constexpr int FS_OFF_WO = FS_OFF_WQKV + 3 * FS_D * FS_LDW * 2;            // (group A), W1 | W2
constexpr int FS_OFF_W1 = FS_OFF_WO + FS_D * FS_LDW * 2;                  // (group B)
constexpr int FS_OFF_W2 = FS_OFF_W1 + FS_F * FS_LDW * 2;
constexpr int FS_OFF_H = FS_OFF_W2 + FS_D * FS_LDW2 * 2;
constexpr int FS_OFF_RED = FS_OFF_H + FS_RB * FS_LDH * 4;
constexpr int FS_OFF_Q = FS_OFF_RED + FS_RB * FS_LDH * 4;
constexpr int FS_OFF_A = FS_OFF_Q + FS_RB * FS_LDQ * 4;
constexpr int FS_OFF_G = FS_OFF_A + FS_RB * FS_LDA * 2;
constexpr int FS_OFF_E = FS_OFF_G + FS_RB * FS_LDG * 2;          // per warp: e[head][key]
constexpr int FS_OFF_S = FS_OFF_E + FS_WARPS * FS_H * FS_MAXK * 4;   // per warp: key slots
constexpr int FS_OFF_PV = FS_OFF_S + FS_WARPS * FS_MAXK * 4;     // small parameter vectors
// per block: bqkv | bo | ln2_g | ln2_b | b1 | b2 | ln1_g | ln1_b, then lnf_g | lnf_b | head_w | head_b[k]
constexpr int FS_PV_NF = 8;
__host__ __device__ constexpr int fs_pv_start(int f) {
    return f == 0 ? 0 : f == 1 ? 3 * FS_D : f == 2 ? 4 * FS_D : f == 3 ? 5 * FS_D : f == 4 ? 6 * FS_D
         : f == 5 ? 6 * FS_D + FS_F : f == 6 ? 7 * FS_D + FS_F : f == 7 ? 8 * FS_D + FS_F : 9 * FS_D + FS_F;
}
constexpr int FS_PV = fs_pv_start(FS_PV_NF);   // floats per block
constexpr int FS_PG = 3 * FS_D + 4;            // the head's vectors (padded)
inline int fs_smem_bytes(int layers) { return FS_OFF_PV + (layers * FS_PV + FS_PG) * 4; }

struct FsArgs {
    const float* P;
    int64_t pv[TF_MAX_LAYERS][FS_PV_NF];        // offsets in P of each block's small vectors
    int64_t pg[4];                              // offsets of lnf_g, lnf_b, head_w, head_b
    const __nv_bfloat16* wb;                    // bf16 weights (duplicated rows when compensated)
    int64_t woff[TF_MAX_LAYERS][4];             // element offsets of Wqkv, Wo, W1, W2 in wb
    const uint64_t* bits;
    int64_t R;                                  // rows of the pass (the kernel stops at *Udev)
    int k;                                      // position
    float* kv;                                  // QKV slabs of every layer and step
    int64_t cap;
    const int32_t* anc;                         // anc[r * n + j]: slot of r's ancestor at step j
    const int32_t* par;                         // set: anc is the previous step's table (compose)
    int32_t* anc_new;                           //   and this step's table is written here
    const float* tab_h;                         // optional first-block tables over (token, position):
    const float* tab_qkv;                       //   h0 [3n][64] and q|k|v without bias [3n][192]
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

__device__ __forceinline__ void fs_ldm4(uint32_t (&r)[4], const __nv_bfloat16* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
}
__device__ __forceinline__ void fs_ldm2(uint32_t& r0, uint32_t& r1, const __nv_bfloat16* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
}

// C (16 x 8) += A . W[n0 : n0 + 8]^T over the logical columns kb .. kb + 16 KS of W (width K):
// A and W in shared memory (bf16, row strides lda and ldw); a compensated A holds its lo halves
// K columns after the hi ones and both meet the same W fragment, on two accumulators (the plain
// form alternates its k-steps between them), joined at the end.  Fragments by ldmatrix: A as four
// 8 x 8 pieces (rows 0-7 / 8-15, columns 0-7 / 8-15 of the k-step), W as two (its 8 rows,
// columns 0-7 / 8-15), which are the m16n8k16 operand layouts.
template <int MODE, int KS>
__device__ __forceinline__ void fs_tile(const __nv_bfloat16* sA, int lda, int K, const __nv_bfloat16* W, int ldw,
                                        int n0, int kb, float (&c)[4], int lane) {
    const __nv_bfloat16* pa = sA + (lane & 15) * lda + kb + 8 * (lane >> 4);
    const __nv_bfloat16* pb = W + (n0 + (lane & 7)) * ldw + kb + 8 * ((lane >> 3) & 1);
    float c2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < KS; ++s) {
        uint32_t b0, b1, a[4];
        fs_ldm2(b0, b1, pb + 16 * s);
        fs_ldm4(a, pa + 16 * s);
        if (MODE == ACT_BF16X2) {
            uint32_t al[4];
            fs_ldm4(al, pa + K + 16 * s);
            fs_mma(c, a, b0, b1);
            fs_mma(c2, al, b0, b1);
        } else if (s & 1) {
            fs_mma(c2, a, b0, b1);
        } else {
            fs_mma(c, a, b0, b1);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] += c2[i];
}

__device__ __forceinline__ void fs_cp16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void fs_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void fs_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Rows [0, N) of a weight matrix (the first K columns of each global row, row stride ldw) into
// shared memory with row stride lds, by 16-byte asynchronous copies spread over the CTA.
template <int N, int K>
__device__ __forceinline__ void fs_stage(__nv_bfloat16* dst, int lds, const __nv_bfloat16* src, int64_t ldw) {
    constexpr int CPR = K / 8;                         // 16-byte pieces per row
    for (int i = threadIdx.x; i < N * CPR; i += FS_THREADS) {
        const int r = i / CPR, c = i - r * CPR;
        fs_cp16(dst + r * lds + 8 * c, src + r * ldw + 8 * c);
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

// split-K pair of a 64-column GEMM: warps 8..15 leave their partial sums in sRed, warps 0..7 add
// them, the bias and the residual into h
__device__ __forceinline__ void fs_resid_join(float* sH, float* sRed, const float* __restrict__ bias,
                                              const float (&c)[4], int kh, int col, int g) {
    if (kh) {
        *reinterpret_cast<float2*>(sRed + g * FS_LDH + col) = make_float2(c[0], c[1]);
        *reinterpret_cast<float2*>(sRed + (g + 8) * FS_LDH + col) = make_float2(c[2], c[3]);
    }
    __syncthreads();
    if (!kh) {
        const float2 bb = *reinterpret_cast<const float2*>(bias + col);
        const float2 p0 = *reinterpret_cast<const float2*>(sRed + g * FS_LDH + col);
        const float2 p1 = *reinterpret_cast<const float2*>(sRed + (g + 8) * FS_LDH + col);
        float2* h0 = reinterpret_cast<float2*>(sH + g * FS_LDH + col);
        float2* h1 = reinterpret_cast<float2*>(sH + (g + 8) * FS_LDH + col);
        h0->x += (c[0] + p0.x) + bb.x; h0->y += (c[1] + p0.y) + bb.y;
        h1->x += (c[2] + p1.x) + bb.x; h1->y += (c[3] + p1.y) + bb.y;
    }
}

template <int MODE>
__global__ void __launch_bounds__(FS_THREADS, 1)
tf_step_fused_kernel(const __grid_constant__ ModelConst mc, const __grid_constant__ FsArgs A) {
    extern __shared__ __align__(16) uint8_t fs_smem[];
    __nv_bfloat16* sWqkv = reinterpret_cast<__nv_bfloat16*>(fs_smem + FS_OFF_WQKV);
    __nv_bfloat16* sWo = reinterpret_cast<__nv_bfloat16*>(fs_smem + FS_OFF_WO);
    __nv_bfloat16* sW1 = reinterpret_cast<__nv_bfloat16*>(fs_smem + FS_OFF_W1);
    __nv_bfloat16* sW2 = reinterpret_cast<__nv_bfloat16*>(fs_smem + FS_OFF_W2);
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
    pdl_wait();                                          // the previous step's bookkeeping is complete
    pdl_trigger();
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
    // block weights: Wqkv | Wo of block l in group A, W1 | W2 in group B, staged one group ahead
    const bool tables = A.tab_qkv != nullptr;             // block 0's h and q|k|v from the tables
    auto stage_a = [&](int l) {
        if (l > 0 || !tables) fs_stage<3 * FS_D, FS_D>(sWqkv, FS_LDW, A.wb + A.woff[l][TF_WQKV], KX * FS_D);
        fs_stage<FS_D, FS_D>(sWo, FS_LDW, A.wb + A.woff[l][TF_WO], KX * FS_D);
        fs_cp_commit();
    };
    auto stage_b = [&](int l) {
        fs_stage<FS_F, FS_D>(sW1, FS_LDW, A.wb + A.woff[l][TF_W1], KX * FS_D);
        fs_stage<FS_D, FS_F>(sW2, FS_LDW2, A.wb + A.woff[l][TF_W2], KX * FS_F);
        fs_cp_commit();
    };
    stage_a(0);
    stage_b(0);
    // the blocks' biases and LayerNorm vectors and the head's vectors into shared memory
    float* sPv = reinterpret_cast<float*>(fs_smem + FS_OFF_PV);
    const int L = mc.layers;
    const int npv = L * FS_PV + FS_PG;
    for (int base = 0; base < npv; base += 4 * FS_THREADS) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + u * FS_THREADS + threadIdx.x;
            int64_t src = -1;
            if (i < L * FS_PV) {
                const int l = i / FS_PV, o = i - l * FS_PV;
                int f = 0;
                while (o >= fs_pv_start(f + 1)) ++f;
                src = A.pv[l][f] + (o - fs_pv_start(f));
            } else if (i < npv) {
                const int o = i - L * FS_PV;
                if (o < 3 * FS_D) src = A.pg[o / FS_D] + (o % FS_D);
                else if (o == 3 * FS_D) src = A.pg[3] + k;
            }
            v[u] = src >= 0 ? __ldg(P + src) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = base + u * FS_THREADS + threadIdx.x;
            if (i < npv) sPv[i] = v[u];
        }
    }
    const float* sHead = sPv + L * FS_PV;                // lnf_g | lnf_b | head_w | head_b[k]
    // this row's ancestor slots (the same for every block)
    int32_t* s_s = sS + warp * FS_MAXK;
    if (A.par) {
        // compose this step's table from the parent's row of the previous one and keep it
        int64_t p = live ? A.par[grow] : 0;
        p = p < 0 ? 0 : (p >= A.cap ? A.cap - 1 : p);
        for (int j = lane; j < k; j += 32) {
            int64_t slot = j + 1 < k ? (int64_t)A.anc[p * n + j] : p;
            slot = slot < 0 ? 0 : (slot >= A.cap ? A.cap - 1 : slot);
            s_s[j] = (int32_t)slot;
            if (live) A.anc_new[grow * n + j] = (int32_t)slot;
        }
    } else {
        for (int j = lane; j < k; j += 32) {
            int64_t slot = live ? A.anc[grow * n + j] : 0;
            slot = slot < 0 ? 0 : (slot >= A.cap ? A.cap - 1 : slot);
            s_s[j] = (int32_t)slot;
        }
    }

    // ---- embedding and LayerNorm 1 of block 0, or block 0's h and q|k|v from the tables
    if (tables) {
        const int tok = k == 0 ? 2 : (int)((x >> mc.order[k - 1]) & 1ull);
        const int64_t trow = (int64_t)tok * n + k;
        const int c0 = 2 * lane;
        *reinterpret_cast<float2*>(sH + r * FS_LDH + c0) = *reinterpret_cast<const float2*>(A.tab_h + trow * FS_D + c0);
        __syncthreads();                                 // the staged bias of block 0
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int c = FS_D * i + c0;
            const float2 v = *reinterpret_cast<const float2*>(A.tab_qkv + trow * 3 * FS_D + c);
            const float2 bb = *reinterpret_cast<const float2*>(sPv + fs_pv_start(0) + c);
            *reinterpret_cast<float2*>(sQ + r * FS_LDQ + c) = make_float2(v.x + bb.x, v.y + bb.y);
        }
    } else {
        const int tok = k == 0 ? 2 : (int)((x >> mc.order[k - 1]) & 1ull);
        const int c0 = 2 * lane;
        const float2 e = *reinterpret_cast<const float2*>(P + mc.tok_emb + tok * FS_D + c0);
        const float2 p = *reinterpret_cast<const float2*>(P + mc.pos_emb + k * FS_D + c0);
        *reinterpret_cast<float2*>(sH + r * FS_LDH + c0) = make_float2(e.x + p.x, e.y + p.y);
        __syncthreads();
        const float2 y = fs_ln(sH, r, sPv + fs_pv_start(6), sPv + fs_pv_start(7), lane);
        fs_put2<MODE>(sA, FS_LDA, FS_D, r, c0, y.x, y.y);
    }

    for (int l = 0; l < mc.layers; ++l) {
        const bool next = l + 1 < mc.layers;
        float* slab0 = A.kv + (int64_t)l * n * slab_stride;   // step-0 slab of this layer
        const float* pv = sPv + l * FS_PV;
        fs_cp_wait<1>();                                     // group A of this block has landed
        __syncthreads();
        // ---- qkv = a . Wqkv^T + bqkv: 24 n-tiles over the 16 warps (block 0 with tables: done)
        if (l > 0 || !tables) {
            const float* bq = pv + fs_pv_start(0);
            for (int t = warp; t < 3 * FS_D / 8; t += FS_WARPS) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                fs_tile<MODE, FS_D / 16>(sA, FS_LDA, FS_D, sWqkv, FS_LDW, 8 * t, 0, c, lane);
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
            const float scale = rsqrtf((float)FS_DH) * 1.4426950408889634f;   // log2 domain
            const float4* qrow = reinterpret_cast<const float4*>(sQ + r * FS_LDQ);   // the query row
            // scores: lane takes keys j = lane and j = lane + 32 (the second only when k >= 32)
            float sc[2][FS_H];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int j = lane + 32 * h2;
                if (h2 == 1 && k < 32) {
#pragma unroll
                    for (int hd = 0; hd < FS_H; ++hd) sc[1][hd] = -INFINITY;
                    break;
                }
                const float* kr = j < k ? slab0 + (int64_t)j * slab_stride + (int64_t)s_s[j] * (3 * FS_D) + FS_D
                                        : sQ + r * FS_LDQ + FS_D;
#pragma unroll
                for (int hd = 0; hd < FS_H; ++hd) {
                    float4 kk[FS_DH / 4];
#pragma unroll
                    for (int j4 = 0; j4 < FS_DH / 4; ++j4)
                        kk[j4] = j <= k ? reinterpret_cast<const float4*>(kr)[hd * (FS_DH / 4) + j4] : make_float4(0.f, 0.f, 0.f, 0.f);
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int j4 = 0; j4 < FS_DH / 4; ++j4) {
                        const float4 k4 = kk[j4];
                        const float4 qh = qrow[hd * (FS_DH / 4) + j4];
                        float& sp = (j4 & 1) ? s1 : s0;
                        sp = fmaf(qh.x * scale, k4.x, sp);
                        sp = fmaf(qh.y * scale, k4.y, sp);
                        sp = fmaf(qh.z * scale, k4.z, sp);
                        sp = fmaf(qh.w * scale, k4.w, sp);
                    }
                    sc[h2][hd] = j <= k ? s0 + s1 : -INFINITY;
                }
            }
            float inv_l[FS_H];
#pragma unroll
            for (int hd = 0; hd < FS_H; ++hd) {
                float m = fmaxf(sc[0][hd], sc[1][hd]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                const float e0 = lane <= k ? exp2f(sc[0][hd] - m) : 0.f;
                const float e1 = lane + 32 <= k ? exp2f(sc[1][hd] - m) : 0.f;
                if (lane <= k) e_s[hd * FS_MAXK + lane] = e0;
                if (lane + 32 <= k) e_s[hd * FS_MAXK + lane + 32] = e1;
                inv_l[hd] = 1.f / warp_sum(e0 + e1);
            }
            __syncwarp();
            // weighted values: lane (half, dq) takes columns 4 dq .. 4 dq + 3 (head dq / 4) over the
            // keys j = half, half + 2, ...; the two halves are joined by one shuffle
            const int half = lane >> 4, dq = lane & 15, hd = dq >> 2;
            const float* ev = e_s + hd * FS_MAXK;
            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int jb = half; jb < k; jb += 2 * FS_VB) {
                float4 v[FS_VB];
                float e[FS_VB];
#pragma unroll
                for (int u = 0; u < FS_VB; ++u) {
                    const int j = jb + 2 * u;
                    e[u] = j < k ? ev[j] : 0.f;
                    v[u] = j < k ? *reinterpret_cast<const float4*>(slab0 + (int64_t)j * slab_stride +
                                                                     (int64_t)s_s[j] * (3 * FS_D) + 2 * FS_D + 4 * dq)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < FS_VB; ++u) {
                    o.x = fmaf(e[u], v[u].x, o.x); o.y = fmaf(e[u], v[u].y, o.y);
                    o.z = fmaf(e[u], v[u].z, o.z); o.w = fmaf(e[u], v[u].w, o.w);
                }
            }
            if (half == (k & 1)) {                           // the own value row, once
                const float4 v = *reinterpret_cast<const float4*>(sQ + r * FS_LDQ + 2 * FS_D + 4 * dq);
                o.x = fmaf(ev[k], v.x, o.x); o.y = fmaf(ev[k], v.y, o.y);
                o.z = fmaf(ev[k], v.z, o.z); o.w = fmaf(ev[k], v.w, o.w);
            }
            o.x += __shfl_xor_sync(0xffffffffu, o.x, 16);
            o.y += __shfl_xor_sync(0xffffffffu, o.y, 16);
            o.z += __shfl_xor_sync(0xffffffffu, o.z, 16);
            o.w += __shfl_xor_sync(0xffffffffu, o.w, 16);
            float il = inv_l[0];
#pragma unroll
            for (int h2 = 1; h2 < FS_H; ++h2) il = hd == h2 ? inv_l[h2] : il;
            if (half == 0) {
                fs_put2<MODE>(sA, FS_LDA, FS_D, r, 4 * dq, o.x * il, o.y * il);
                fs_put2<MODE>(sA, FS_LDA, FS_D, r, 4 * dq + 2, o.z * il, o.w * il);
            }
        }
        __syncthreads();
        // ---- h += o . Wo^T + bo: 8 n-tiles, K split over two warp halves
        {
            const int t = warp & 7, kh = warp >> 3;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            fs_tile<MODE, FS_D / 32>(sA, FS_LDA, FS_D, sWo, FS_LDW, 8 * t, kh * (FS_D / 2), c, lane);
            fs_resid_join(sH, sRed, pv + fs_pv_start(1), c, kh, 8 * t + 2 * q4, g);
        }
        __syncthreads();
        if (next) stage_a(l + 1);                            // Wqkv and Wo are free
        // ---- LayerNorm 2
        {
            const float2 y = fs_ln(sH, r, pv + fs_pv_start(2), pv + fs_pv_start(3), lane);
            fs_put2<MODE>(sA, FS_LDA, FS_D, r, 2 * lane, y.x, y.y);
        }
        if (next) fs_cp_wait<1>(); else fs_cp_wait<0>();     // group B of this block has landed
        __syncthreads();
        // ---- hidden = GELU(a . W1^T + b1): 32 n-tiles, two per warp
        {
            const float* b1 = pv + fs_pv_start(4);
#pragma unroll
            for (int tt = 0; tt < 2; ++tt) {
                const int t = warp + FS_WARPS * tt;
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                fs_tile<MODE, FS_D / 16>(sA, FS_LDA, FS_D, sW1, FS_LDW, 8 * t, 0, c, lane);
                const int col = 8 * t + 2 * q4;
                const float2 bb = *reinterpret_cast<const float2*>(b1 + col);
                fs_put2<MODE>(sG, FS_LDG, FS_F, g, col, gelu_tanh(c[0] + bb.x), gelu_tanh(c[1] + bb.y));
                fs_put2<MODE>(sG, FS_LDG, FS_F, g + 8, col, gelu_tanh(c[2] + bb.x), gelu_tanh(c[3] + bb.y));
            }
        }
        __syncthreads();
        // ---- h += hidden . W2^T + b2: 8 n-tiles, K split over two warp halves
        {
            const int t = warp & 7, kh = warp >> 3;
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            fs_tile<MODE, FS_F / 32>(sG, FS_LDG, FS_F, sW2, FS_LDW2, 8 * t, kh * (FS_F / 2), c, lane);
            fs_resid_join(sH, sRed, pv + fs_pv_start(5), c, kh, 8 * t + 2 * q4, g);
        }
        __syncthreads();
        if (next) {
            stage_b(l + 1);                                  // W1 and W2 are free
            const float2 y = fs_ln(sH, r, pv + FS_PV + fs_pv_start(6), pv + FS_PV + fs_pv_start(7), lane);
            fs_put2<MODE>(sA, FS_LDA, FS_D, r, 2 * lane, y.x, y.y);
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
        const float2 y = fs_ln(sH, r, sHead, sHead + FS_D, lane);
        const float2 hw = *reinterpret_cast<const float2*>(sHead + 2 * FS_D + 2 * lane);
        const float a = warp_sum(fmaf(y.x, hw.x, y.y * hw.y)) + sHead[3 * FS_D];
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
        const int most = fs_smem_bytes(TF_MAX_LAYERS);
        NQS_CK(cudaFuncSetAttribute(tf_step_fused_kernel<ACT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
        NQS_CK(cudaFuncSetAttribute(tf_step_fused_kernel<ACT_BF16X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, most));
        configured_device = dev;
    }
    FsArgs a{};
    a.P = P;
    for (int l = 0; l < mc.layers; ++l) {
        const int64_t f[FS_PV_NF] = {mc.bqkv[l], mc.bo[l], mc.ln2_g[l], mc.ln2_b[l], mc.b1[l], mc.b2[l], mc.ln1_g[l], mc.ln1_b[l]};
        for (int i = 0; i < FS_PV_NF; ++i) a.pv[l][i] = f[i];
    }
    a.pg[0] = mc.lnf_g; a.pg[1] = mc.lnf_b; a.pg[2] = mc.head_w; a.pg[3] = mc.head_b;
    a.wb = reinterpret_cast<const __nv_bfloat16*>(w.bf16);
    for (int l = 0; l < mc.layers; ++l)
        for (int m = 0; m < 4; ++m) a.woff[l][m] = w.bf16_off[l][m];
    a.bits = bits; a.R = R; a.k = k;
    a.kv = kc.kv; a.cap = kc.cap; a.anc = kc.anc; a.Udev = kc.Udev;
    a.par = kc.par; a.anc_new = kc.anc_new;
    a.tab_h = kc.tab_h; a.tab_qkv = kc.tab_qkv;
    a.p_out = p_out; a.thr = thr; a.trace = trace;
    const unsigned grid = (unsigned)((R + FS_RB - 1) / FS_RB);
    const int64_t M = R;
    const double flops = 2.0 * M * mc.layers * (double)FS_D * (3 * FS_D + FS_D + 2 * FS_F) * (mc.compensated ? 2 : 1);
    ProfScope ps("tf_step_fused", s, flops, 0.0);
    const int smem = fs_smem_bytes(mc.layers);
    // a programmatic dependent launch: resident before the previous step's bookkeeping ends
    if (mc.compensated) NQS_CK(launch_pdl(tf_step_fused_kernel<ACT_BF16X2>, dim3(grid), dim3(FS_THREADS), (size_t)smem, s, mc, a));
    else NQS_CK(launch_pdl(tf_step_fused_kernel<ACT_BF16>, dim3(grid), dim3(FS_THREADS), (size_t)smem, s, mc, a));
    count_launch();
    return NQS_OK;
}

}  // namespace nqs
