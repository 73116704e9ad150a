// Tensor-core GEMMs of the transformer backward for the bf16 models (the recompute forward, the
// input gradients and the weight gradients of the VMC gradient's log psi backward, Eq. grad):
// fp32 operands split into bf16 pairs v = hi + lo on mma.sync m16n8k16 with fp32 accumulation.
//   NT  C[M][N] = A[M][K] . W[N][K]^T (+ bias, or += for the residual)   recompute forward
//   NN  C[M][N] = A[M][K] . W[K][N]                                       input gradients
//   TN  part[z][M][N] = sum over rows k of A[k][M] B[k][N] in split z    weight gradients
// Products: A_hi B_hi + A_lo B_hi, plus A_hi B_lo when B is not bf16-exact (TN: B is the
// recomputed activation, a sum of two bf16 numbers; W is bf16-rounded in these models).  The
// dropped terms are below 2^-16 of the product.  Each output's k-sum runs in a fixed order, so
// the results do not depend on the schedule.
#include "tf_common.cuh"

namespace nqs {
namespace {

constexpr int TB_M = 64, TB_N = 64, TB_K = 32;   // CTA tile, k-stage
constexpr int TB_LD = TB_M + 4;                  // fp32 smem row stride of [k][m] / [k][n] tiles
constexpr int TB_LDK = TB_K + 8;                 // fp32 smem row stride of [m][k] / [n][k] tiles (float2 reads conflict-free)
constexpr int TB_TILE = TB_K * TB_LD > TB_M * TB_LDK ? TB_K * TB_LD : TB_M * TB_LDK;
constexpr int TB_THREADS = 128;                  // 2 x 2 warps of 32 x 32 outputs

__device__ __forceinline__ void tb_mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                       uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// (x, y) -> packed bf16 hi pair and lo pair (lo = bf16(v - hi))
__device__ __forceinline__ void tb_split(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// One k-stage's fp32 tile into shared memory in the layout of global memory: [k][m] rows (stride
// TB_LD) from global [K][M], or [m][k] rows (stride TB_LDK) from global [M][K]; float4 loads with
// consecutive lanes on consecutive 16-byte pieces of a row.  Out-of-range elements are 0.
template <bool KM>
struct TbLoader {
    float4 r[4];
    __device__ __forceinline__ void fetch(const float* __restrict__ g, int64_t ld, int64_t m0, int64_t mlim, int64_t k0,
                                          int64_t klim) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int f = threadIdx.x + TB_THREADS * i;
            if (KM) {   // rows k (32) x 16 float4 of m
                const int k = f >> 4, mq = f & 15;
                const int64_t gk = k0 + k, gm = m0 + 4 * mq;
                r[i] = (gk < klim && gm < mlim) ? __ldg(reinterpret_cast<const float4*>(g + gk * ld + gm))
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {    // rows m (64) x 8 float4 of k
                const int m = f >> 3, kq = f & 7;
                const int64_t gm = m0 + m, gk = k0 + 4 * kq;
                r[i] = (gm < mlim && gk < klim) ? __ldg(reinterpret_cast<const float4*>(g + gm * ld + gk))
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    __device__ __forceinline__ void stash(float* s) const {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int f = threadIdx.x + TB_THREADS * i;
            if (KM) {
                const int k = f >> 4, mq = f & 15;
                *reinterpret_cast<float4*>(s + k * TB_LD + 4 * mq) = r[i];
            } else {
                const int m = f >> 3, kq = f & 7;
                *reinterpret_cast<float4*>(s + m * TB_LDK + 4 * kq) = r[i];
            }
        }
    }
};

// Element (m, k) of a staged tile and the bf16 hi | lo pair of elements (m, k), (m, k + 1).
template <bool KM>
__device__ __forceinline__ float tb_at(const float* s, int m, int k) {
    return KM ? s[k * TB_LD + m] : s[m * TB_LDK + k];
}
template <bool KM>
__device__ __forceinline__ void tb_pair(const float* s, int m, int k, uint32_t& hi, uint32_t& lo) {
    if (KM) {
        tb_split(s[k * TB_LD + m], s[(k + 1) * TB_LD + m], hi, lo);
    } else {
        const float2 v = *reinterpret_cast<const float2*>(s + m * TB_LDK + k);
        tb_split(v.x, v.y, hi, lo);
    }
}

// EPI: 0 store (C = acc + bias), 1 residual (C += acc + bias), 2 split-K partial (TN)
template <bool A_KM, bool B_KN, bool B_EXACT, int EPI>
__global__ void __launch_bounds__(TB_THREADS)
tb_gemm_kernel(const float* __restrict__ A, int64_t lda, const float* __restrict__ B, int64_t ldb,
               const float* __restrict__ bias, float* __restrict__ C, int64_t ldc, int64_t M, int N, int64_t K,
               int64_t k_split, float* __restrict__ part, int with_colsum) {
    __shared__ __align__(16) float sA[TB_TILE];
    __shared__ __align__(16) float sB[TB_TILE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
    const int64_t m0 = (int64_t)blockIdx.y * TB_M;
    const int n0 = blockIdx.x * TB_N;
    const int64_t kb = EPI == 2 ? (int64_t)blockIdx.z * k_split : 0;
    const int64_t ke = EPI == 2 ? min(K, kb + k_split) : K;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
    float csum = 0.f;                          // TN: column sums of A (the bias gradient)
    TbLoader<A_KM> la;
    TbLoader<B_KN> lb;
    la.fetch(A, lda, m0, M, kb, ke);
    lb.fetch(B, ldb, n0, N, kb, ke);
    for (int64_t k0 = kb; k0 < ke; k0 += TB_K) {
        __syncthreads();                       // the previous stage's reads are done
        la.stash(sA);
        lb.stash(sB);
        __syncthreads();
        if (k0 + TB_K < ke) {                  // the next stage's loads fly during the MMAs
            la.fetch(A, lda, m0, M, k0 + TB_K, ke);
            lb.fetch(B, ldb, n0, N, k0 + TB_K, ke);
        }
        if (EPI == 2 && with_colsum && blockIdx.x == 0 && threadIdx.x < TB_M) {
#pragma unroll 8
            for (int k = 0; k < TB_K; ++k) csum += tb_at<A_KM>(sA, threadIdx.x, k);
        }
#pragma unroll
        for (int ks = 0; ks < TB_K; ks += 16) {
            uint32_t bh[4][2], bl[4][2];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int nn = wn + 8 * j + g;
                tb_pair<B_KN>(sB, nn, ks + 2 * q, bh[j][0], bl[j][0]);
                tb_pair<B_KN>(sB, nn, ks + 2 * q + 8, bh[j][1], bl[j][1]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int mm = wm + 16 * i + g;
                uint32_t ah[4], al[4];
                tb_pair<A_KM>(sA, mm, ks + 2 * q, ah[0], al[0]);            // row g, k 2q..
                tb_pair<A_KM>(sA, mm + 8, ks + 2 * q, ah[1], al[1]);        // row g + 8
                tb_pair<A_KM>(sA, mm, ks + 2 * q + 8, ah[2], al[2]);        // row g, k 2q + 8..
                tb_pair<A_KM>(sA, mm + 8, ks + 2 * q + 8, ah[3], al[3]);    // row g + 8
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    tb_mma(acc[i][j], ah[0], ah[1], ah[2], ah[3], bh[j][0], bh[j][1]);
                    tb_mma(acc[i][j], al[0], al[1], al[2], al[3], bh[j][0], bh[j][1]);
                    if (!B_EXACT) tb_mma(acc[i][j], ah[0], ah[1], ah[2], ah[3], bl[j][0], bl[j][1]);
                }
            }
        }
    }
    // epilogue
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = n0 + wn + 8 * j + 2 * q;
            if (col >= N) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t row = m0 + wm + 16 * i + g + 8 * h;
                if (row >= M) continue;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if (EPI == 2) {
                    float* pz = part + (int64_t)blockIdx.z * ((int64_t)M * N + M);
                    *reinterpret_cast<float2*>(pz + row * N + col) = make_float2(v0, v1);
                } else {
                    if (bias) { v0 += bias[col]; v1 += bias[col + 1]; }
                    float2* cp = reinterpret_cast<float2*>(C + row * ldc + col);
                    if (EPI == 1) { const float2 o = *cp; v0 += o.x; v1 += o.y; }
                    *cp = make_float2(v0, v1);
                }
            }
        }
    if (EPI == 2 && with_colsum && blockIdx.x == 0 && threadIdx.x < TB_M && m0 + threadIdx.x < M)
        part[(int64_t)blockIdx.z * ((int64_t)M * N + M) + (int64_t)M * N + m0 + threadIdx.x] = csum;
}

bool tb_aligned(const void* p, int64_t ld) { return ((uintptr_t)p & 15) == 0 && (ld & 3) == 0; }

}  // namespace

bool tc_bwd_ok(const void* A, int64_t lda, const void* B, int64_t ldb) {
    return tb_aligned(A, lda) && tb_aligned(B, ldb);
}

int tc_bwd_gemm_nt(const float* A, int64_t lda, const float* W, int64_t ldw, const float* bias, float* C, int64_t ldc,
                   int64_t M, int N, int K, bool resid, cudaStream_t s) {
    if (M <= 0) return NQS_OK;
    if (N % 2 || K % 4 || !tc_bwd_ok(A, lda, W, ldw) || (ldc & 1) || ((uintptr_t)C & 7)) {
        set_error("tensor-core backward GEMM: bad layout");
        return NQS_ERR_INVALID_ARG;
    }
    dim3 grid((unsigned)((N + TB_N - 1) / TB_N), (unsigned)((M + TB_M - 1) / TB_M), 1);
    if (resid) tb_gemm_kernel<false, false, true, 1><<<grid, TB_THREADS, 0, s>>>(A, lda, W, ldw, bias, C, ldc, M, N, K, 0, nullptr, 0);
    else tb_gemm_kernel<false, false, true, 0><<<grid, TB_THREADS, 0, s>>>(A, lda, W, ldw, bias, C, ldc, M, N, K, 0, nullptr, 0);
    NQS_LAUNCHED();
    return NQS_OK;
}

int tc_bwd_gemm_nn(const float* A, int64_t lda, const float* W, int64_t ldw, float* C, int64_t ldc, int64_t M, int N,
                   int K, cudaStream_t s) {
    if (M <= 0) return NQS_OK;
    if (N % 4 || K % 4 || !tc_bwd_ok(A, lda, W, ldw) || (ldc & 1) || ((uintptr_t)C & 7)) {
        set_error("tensor-core backward GEMM: bad layout");
        return NQS_ERR_INVALID_ARG;
    }
    dim3 grid((unsigned)((N + TB_N - 1) / TB_N), (unsigned)((M + TB_M - 1) / TB_M), 1);
    tb_gemm_kernel<false, true, true, 0><<<grid, TB_THREADS, 0, s>>>(A, lda, W, ldw, nullptr, C, ldc, M, N, K, 0, nullptr, 0);
    NQS_LAUNCHED();
    return NQS_OK;
}

int tc_bwd_outer_partial(const float* delta, int64_t ld_d, const float* act, int64_t ld_a, int64_t rows, int out_dim,
                         int in_dim, int64_t nsplit, int64_t per, bool with_bias, float* part, cudaStream_t s) {
    if (rows <= 0) return NQS_OK;
    if (out_dim % 4 || in_dim % 4 || !tc_bwd_ok(delta, ld_d, act, ld_a)) {
        set_error("tensor-core weight gradient: bad layout");
        return NQS_ERR_INVALID_ARG;
    }
    dim3 grid((unsigned)((in_dim + TB_N - 1) / TB_N), (unsigned)((out_dim + TB_M - 1) / TB_M), (unsigned)nsplit);
    tb_gemm_kernel<true, true, false, 2><<<grid, TB_THREADS, 0, s>>>(delta, ld_d, act, ld_a, nullptr, nullptr, 0, out_dim,
                                                                     in_dim, rows, per, part, with_bias ? 1 : 0);
    NQS_LAUNCHED();
    return NQS_OK;
}

}  // namespace nqs
