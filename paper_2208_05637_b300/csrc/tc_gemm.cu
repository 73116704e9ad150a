// BF16 GEMM on the fifth-generation tensor cores for the transformer's block contractions:
//   C[M, N] (epilogue) = A[M, K] . W[N, K]^T + bias,   A, W bf16 K-contiguous, fp32 accumulate.
//
// One CTA computes a 128 x BN tile (BN = N, or N/2 when N > 256).  TMA copies 128 x 64 and
// BN x 64 bf16 boxes (128-byte rows, 128-byte swizzle) into a ring of shared-memory stages
// completing on mbarriers; one thread issues tcgen05.mma (M = 128, N = BN, K = 16 per
// instruction, four per 64-wide k-block) into a TMEM accumulator of BN fp32 columns and
// commits each stage back to an mbarrier so the stage can be refilled; after the last k-block a
// final commit releases the four warps, which read their 32 TMEM lanes (= rows) with
// tcgen05.ld and apply the epilogue: fp32 store (QKV), fp32 residual add (h += ...), or GELU to
// bf16 (MLP hidden).  Shared-memory descriptors use the K-major 128B-swizzle canonical layout
// (8-row x 128-byte atoms, stride 1024 bytes); moving 16 elements along K adds 32 bytes to the
// start address.
//
// Every wait on an mbarrier is bounded by a clock budget; a timeout records a nonzero status
// in g_tc_status, skips the epilogue, waits (bounded) for the CTA's own copies in flight,
// frees the TMEM it holds and returns.  The host reads the status with tc_status_take().
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "tf_common.cuh"

namespace nqs {

static __device__ int g_tc_status;

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;                  // 64 bf16 = one 128-byte swizzle row
constexpr long long TC_WAIT_CYCLES = 4ll * 1000 * 1000 * 1000;   // ~2 s at the boost clock

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false after the clock budget.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try(bar, phase)) {
        if (clock64() - t0 > TC_WAIT_CYCLES) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(su32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// K-major, 128-byte swizzle shared-memory matrix descriptor (sm_100 family layout).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address >> 4        bits [0, 14)
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // SWIZZLE_128B
    return d;
}

// kind::f16 instruction descriptor: fp32 accumulator, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int TC_THREADS = 256;   // 8 warps: warps w and w+4 share TMEM lanes 32(w%4).., split columns

template <int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const float* __restrict__ bias, void* __restrict__ Cv, int64_t M, int N, int K, int BN,
               int tmem_cols, int stages) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nkb = (K + TC_BK - 1) / TC_BK;
    const uint32_t a_bytes = TC_BM * 128;
    const uint32_t b_bytes = (uint32_t)BN * 128;
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)stages * a_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + (size_t)stages * b_bytes);
    uint64_t* empty = full + stages;
    uint64_t* done = empty + stages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.y * TC_BM;
    const int n0 = blockIdx.x * BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        bool ok = true;
        const uint32_t idesc = idesc_bf16(TC_BM, BN);
        int issued = 0;
        int waited_full = 0;   // k-blocks whose data arrived (for the timeout drain)
        for (; issued < stages && issued < nkb; ++issued) {
            mbar_expect_tx(&full[issued], a_bytes + b_bytes);
            tma_load_2d(sA + (size_t)issued * a_bytes, &tmA, &full[issued], issued * TC_BK, (int)m0);
            tma_load_2d(sB + (size_t)issued * b_bytes, &tmB, &full[issued], issued * TC_BK, n0);
        }
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % stages;
            if (!mbar_wait(&full[s], (uint32_t)((kb / stages) & 1))) { ok = false; break; }
            waited_full = kb + 1;
            tc_fence_after();
            const uint32_t a0 = su32(sA + (size_t)s * a_bytes), b0 = su32(sB + (size_t)s * b_bytes);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
                umma_bf16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (kb | kk) != 0);
            umma_commit(&empty[s]);
            // refill the stage the previous k-block used, once its MMAs are done
            if (kb >= 1 && issued < nkb) {
                const int ps = (kb - 1) % stages;
                if (!mbar_wait(&empty[ps], (uint32_t)(((kb - 1) / stages) & 1))) { ok = false; break; }
                mbar_expect_tx(&full[ps], a_bytes + b_bytes);
                tma_load_2d(sA + (size_t)ps * a_bytes, &tmA, &full[ps], issued * TC_BK, (int)m0);
                tma_load_2d(sB + (size_t)ps * b_bytes, &tmB, &full[ps], issued * TC_BK, n0);
                ++issued;
            }
        }
        umma_commit(done);
        if (!ok) {
            atomicExch(&g_tc_status, 1);
            // drain: wait (bounded) for every copy still in flight before the CTA exits
            for (int kb = waited_full; kb < issued; ++kb)
                mbar_wait(&full[kb % stages], (uint32_t)((kb / stages) & 1));
        }
        s_ok = ok ? 1 : 0;
    }
    const bool got = __syncthreads_and(mbar_wait(done, 0)) != 0;   // block-uniform
    if (!got && threadIdx.x == 0) atomicExch(&g_tc_status, 2);
    if (got && s_ok) {
        tc_fence_after();
        const int quad = warp & 3, half_w = warp >> 2;
        const int64_t row = m0 + quad * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16);
        for (int c = half_w * 16; c < BN; c += 32) {
            float v16[16];
            tmem_ld16(tbase + (uint32_t)c, v16);
            if (row < M) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int col = n0 + c + 8 * half;
                    float v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = v16[8 * half + j] + (bias ? bias[col + j] : 0.f);
                    if (EPI == TF_EPI_GELU) {
                        __nv_bfloat16* C = reinterpret_cast<__nv_bfloat16*>(Cv) + row * N + col;
                        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(gelu_tanh(v[j]));
                        *reinterpret_cast<uint4*>(C) = *reinterpret_cast<const uint4*>(o);
                    } else if (EPI == TF_EPI_GELU2) {
                        // compensated output: hi in columns [0, N), lo = bf16(g - hi) in [N, 2N)
                        __nv_bfloat16* C = reinterpret_cast<__nv_bfloat16*>(Cv) + row * 2 * N + col;
                        __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float g = gelu_tanh(v[j]);
                            hi[j] = __float2bfloat16_rn(g);
                            lo[j] = __float2bfloat16_rn(g - __bfloat162float(hi[j]));
                        }
                        *reinterpret_cast<uint4*>(C) = *reinterpret_cast<const uint4*>(hi);
                        *reinterpret_cast<uint4*>(C + N) = *reinterpret_cast<const uint4*>(lo);
                    } else {
                        float4* C = reinterpret_cast<float4*>(reinterpret_cast<float*>(Cv) + row * N + col);
                        float4 x0 = make_float4(v[0], v[1], v[2], v[3]), x1 = make_float4(v[4], v[5], v[6], v[7]);
                        if (EPI == TF_EPI_RESID) {
                            const float4 y0 = C[0], y1 = C[1];
                            x0.x += y0.x; x0.y += y0.y; x0.z += y0.z; x0.w += y0.w;
                            x1.x += y1.x; x1.y += y1.y; x1.z += y1.z; x1.w += y1.w;
                        }
                        C[0] = x0;
                        C[1] = x1;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---------------------------------------------------------------- host: tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// rows x cols bf16 row-major matrix, box of box_rows x 64
int make_map(CUtensorMap* map, const void* base, int64_t rows, int cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled is unavailable"); return NQS_ERR_CUDA; }
    if (((uintptr_t)base & 15) || ((cols * 2) & 15)) { set_error("TMA operand must be 16-byte aligned"); return NQS_ERR_INVALID_ARG; }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"); return NQS_ERR_CUDA; }
    return NQS_OK;
}

}  // namespace

int tc_gemm_bf16(const void* A, const uint16_t* W, const float* bias, void* C, int64_t M, int N, int K, int epi,
                 cudaStream_t s) {
    if (M <= 0) return NQS_OK;
    if (N % 16 || N < 16 || K % 8 || K <= 0) { set_error("tensor-core GEMM needs N % 16 == 0 and K % 8 == 0"); return NQS_ERR_UNSUPPORTED; }
    // N tile: N itself up to 128 columns, else the largest multiple of 16 <= 128 dividing N, so
    // that a 128-column TMEM accumulator lets four CTAs share an SM
    int BN = N;
    if (N > 128) {
        BN = 0;
        for (int b = 128; b >= 16; b -= 16)
            if (N % b == 0) { BN = b; break; }
    }
    if (BN == 0 || BN % 16 || N % BN) { set_error("tensor-core GEMM: unsupported N"); return NQS_ERR_UNSUPPORTED; }
    if ((M + TC_BM - 1) / TC_BM > 65535) { set_error("tensor-core GEMM: M too large"); return NQS_ERR_UNSUPPORTED; }
    const int nkb = (K + TC_BK - 1) / TC_BK;
    const int stages = std::min(nkb, 2);
    int tcols = 32;
    while (tcols < BN) tcols <<= 1;
    size_t smem = 1024 + (size_t)stages * (TC_BM * 128 + (size_t)BN * 128) + (2 * stages + 1) * 8 + 16;
    // keep (resident CTAs) x (TMEM columns) within the 512 columns of an SM: with 228 KB of
    // shared memory per SM and 1 KB reserved per CTA, at most 512/tcols CTAs may fit
    const size_t sm_bytes = 228 * 1024;
    const size_t max_ctas = 512 / (size_t)tcols;
    smem = std::max(smem, sm_bytes / (max_ctas + 1) - 1024 + 1);
    if (smem > 220 * 1024) { set_error("tensor-core GEMM: shared-memory plan too large"); return NQS_ERR_UNSUPPORTED; }
    CUtensorMap ma, mb;
    NQS_TRY(make_map(&ma, A, M, K, TC_BM));
    NQS_TRY(make_map(&mb, W, N, K, BN));
    dim3 grid((unsigned)(N / BN), (unsigned)((M + TC_BM - 1) / TC_BM));
    auto launch = [&](auto kernel) -> int {
        // raise the dynamic shared-memory limit once per kernel (and device), outside any
        // stream capture that later launches may run under
        static int configured_device[8] = {-1, -1, -1, -1, -1, -1, -1, -1};   // per epilogue
        int dev = 0;
        NQS_CK(cudaGetDevice(&dev));
        if (configured_device[epi & 7] != dev) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_gemm)", __FILE__, __LINE__);
            configured_device[epi & 7] = dev;
        }
        kernel<<<grid, TC_THREADS, smem, s>>>(ma, mb, bias, C, M, N, K, BN, tcols, stages);
        NQS_LAUNCHED();
        return NQS_OK;
    };
    switch (epi) {
        case TF_EPI_STORE: return launch(tc_gemm_kernel<TF_EPI_STORE>);
        case TF_EPI_RESID: return launch(tc_gemm_kernel<TF_EPI_RESID>);
        case TF_EPI_GELU: return launch(tc_gemm_kernel<TF_EPI_GELU>);
        case TF_EPI_GELU2: return launch(tc_gemm_kernel<TF_EPI_GELU2>);
        default: set_error("bad GEMM epilogue"); return NQS_ERR_INVALID_ARG;
    }
}

// Read and clear the device status of the tensor-core kernels (synchronous).
int tc_status_take() {
    int v = 0, z = 0;
    NQS_CK(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)));
    if (v) {
        NQS_CK(cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)));
        set_error("a tensor-core GEMM wait timed out (status " + std::to_string(v) + ")");
        return NQS_ERR_TIMEOUT;
    }
    return NQS_OK;
}

}  // namespace nqs

// Diagnostic entry point: C = A . W^T + bias with the tensor-core kernel (see include/nqs.h).
extern "C" int nqs_gemm_bf16(const void* A, const void* W, const float* bias, void* C, int64_t M, int N, int K,
                             int epilogue, void* stream) {
    using namespace nqs;
    if (!A || !W || !C || M < 0) { set_error("null operand or negative M"); return NQS_ERR_INVALID_ARG; }
    NQS_TRY(tc_gemm_bf16(A, (const uint16_t*)W, bias, C, M, N, K, epilogue, (cudaStream_t)stream));
    NQS_CK(cudaStreamSynchronize((cudaStream_t)stream));
    return tc_status_take();
}
