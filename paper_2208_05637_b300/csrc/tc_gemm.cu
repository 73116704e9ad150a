// BF16 GEMM on the fifth-generation tensor cores for the transformer's block contractions:
//   C[M, N] (epilogue) = A[M, K] . W[N, K]^T + bias,   A, W bf16 K-contiguous, fp32 accumulate.
//
// Persistent CTAs walk 128 x BN output tiles (BN <= 128 columns).  A producer warp copies
// 128 x 64 and BN x 64 bf16 boxes (128-byte rows, 128-byte swizzle) with TMA into a ring of
// shared-memory stages completing on mbarriers; an MMA warp issues tcgen05.mma (M = 128,
// N = BN, K = 16 per instruction, four per 64-wide k-block) into one of two TMEM accumulators
// and commits each stage back to its mbarrier; four epilogue warps read the other accumulator
// (their 32 TMEM lanes = rows) with tcgen05.ld and apply the epilogue -- fp32 store (QKV), fp32
// residual add (h += ...), or GELU to bf16 / hi+lo bf16 (MLP hidden) -- while the next tile's
// copies and MMAs proceed.  Each epilogue warp stages 32 rows x 128 bytes of results in
// swizzled shared memory and writes them with one TMA store (a TMA reduce-add for the
// residual), so global writes go out as whole lines without waiting on the warp.  Shared-memory descriptors use the K-major 128B-swizzle canonical layout
// (8-row x 128-byte atoms, stride 1024 bytes); moving 16 elements along K adds 32 bytes to the
// start address.
//
// Every wait on an mbarrier is bounded by a clock budget; a timeout records a nonzero status
// in g_tc_status and raises a CTA-wide abort flag that ends the other roles' loops; the
// producer waits (bounded) for its copies in flight, the TMEM is freed and the CTA returns.  The
// host reads the status with tc_status_take().
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>
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

// TMA store / reduce-add of a 2D box from shared memory, tracked by the thread's bulk groups.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(src)) : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(src)) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another role of the CTA has raised `abort`.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t phase, volatile int* abort) {
    const long long t0 = clock64();
    while (!mbar_try(bar, phase)) {
        if (*abort) return false;
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            *abort = 1;
            atomicExch(&g_tc_status, 1);
            return false;
        }
    }
    return true;
}

// Epilogue of 16 accumulator columns of one row: bias, then store / residual add / GELU.
template <int EPI>
__device__ __forceinline__ void epilogue16(const float (&v16)[16], const float* __restrict__ bias, void* Cv,
                                           int64_t row, int N, int col0) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int col = col0 + 8 * half;
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

// Staged epilogue of 16 accumulator columns (piece `p16` of a 128-byte chunk) of the thread's
// row: the results go to the warp's staging rows in shared memory (row = lane, 128 bytes,
// 16-byte units swizzled as unit ^ (lane & 7), the layout a 128B-swizzle tensor map expects),
// from where one lane writes the whole 32-row chunk with a TMA store.  fp32 epilogues fill
// four 16-byte units per piece, bf16 ones two (GELU2 also two of its lo part, 4 KB further).
template <int EPI>
__device__ __forceinline__ void stage16(const float (&v16)[16], const float* __restrict__ bias, int col0, int p16,
                                        uint32_t stg, int lane) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = v16[j] + (bias ? bias[col0 + j] : 0.f);
    const uint32_t row = stg + (uint32_t)lane * 128;
    const int sw = lane & 7;
    if (EPI == TF_EPI_STORE || EPI == TF_EPI_RESID) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            st_shared_v4(row + (uint32_t)(((p16 * 4 + u) ^ sw) << 4), __float_as_uint(v[4 * u]), __float_as_uint(v[4 * u + 1]),
                         __float_as_uint(v[4 * u + 2]), __float_as_uint(v[4 * u + 3]));
    } else {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float g = gelu_tanh(v[8 * u + j]);
                hi[j] = __float2bfloat16_rn(g);
                if (EPI == TF_EPI_GELU2) lo[j] = __float2bfloat16_rn(g - __bfloat162float(hi[j]));
            }
            const uint32_t off = (uint32_t)(((p16 * 2 + u) ^ sw) << 4);
            st_shared_v4(row + off, pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]),
                         pack_bf16(hi[6], hi[7]));
            if (EPI == TF_EPI_GELU2)
                st_shared_v4(row + 4096 + off, pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]),
                             pack_bf16(lo[6], lo[7]));
        }
    }
}

// Persistent, warp-specialised GEMM: warp 0 issues the TMA copies into a ring of `stages`
// shared-memory stages, warp 1 issues the MMAs into one of two TMEM accumulators, warps 2..5
// (one per TMEM lane quadrant) drain the other accumulator through the epilogue, so a tile's
// epilogue overlaps the next tile's copies and MMAs.  Tiles are taken round robin, N fastest.
constexpr int TC_THREADS = 192;

constexpr int TC_STAGE_BYTES_PER_WARP = 8192;   // two 4 KB chunk buffers, or hi + lo of one

template <int EPI, bool TMA_EPI>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmC, const float* __restrict__ bias, void* __restrict__ Cv,
               int64_t M, int N, int K, int BN, int tmem_cols, int stages, int n_tiles_n, int64_t total_tiles) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nkb = (K + TC_BK - 1) / TC_BK;
    const uint32_t a_bytes = TC_BM * 128;
    const uint32_t b_bytes = (uint32_t)BN * 128;
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)stages * a_bytes;
    uint8_t* sC = sB + (size_t)stages * b_bytes;     // 1024-aligned: a_bytes, b_bytes are multiples of 1024
    uint64_t* full = reinterpret_cast<uint64_t*>(sC + (TMA_EPI ? 4 * TC_STAGE_BYTES_PER_WARP : 0));
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;       // [2] accumulator ready for the epilogue
    uint64_t* tempty = tfull + 2;           // [2] accumulator drained by the epilogue
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
        *abort = 0;
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

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer
            int64_t it = 0;
            for (int64_t t = blockIdx.x; t < total_tiles && !*abort; t += gridDim.x) {
                const int m0 = (int)(t / n_tiles_n) * TC_BM, n0 = (int)(t % n_tiles_n) * BN;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % stages);
                    if (!mbar_wait_or_abort(&empty[s], (uint32_t)(((it / stages) & 1) ^ 1), abort)) break;
                    mbar_expect_tx(&full[s], a_bytes + b_bytes);
                    tma_load_2d(sA + (size_t)s * a_bytes, &tmA, &full[s], kb * TC_BK, m0);
                    tma_load_2d(sB + (size_t)s * b_bytes, &tmB, &full[s], kb * TC_BK, n0);
                }
            }
            // wait (bounded) for this CTA's last copies before it may exit
            for (int64_t j = it - stages < 0 ? 0 : it - stages; j < it; ++j) mbar_wait(&full[j % stages], (uint32_t)((j / stages) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = idesc_bf16(TC_BM, BN);
            int64_t it = 0, acc = 0;
            for (int64_t t = blockIdx.x; t < total_tiles && !*abort; t += gridDim.x, ++acc) {
                const int buf = (int)(acc & 1);
                if (!mbar_wait_or_abort(&tempty[buf], (uint32_t)(((acc >> 1) & 1) ^ 1), abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(buf * (tmem_cols >> 1));
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % stages);
                    if (!mbar_wait_or_abort(&full[s], (uint32_t)((it / stages) & 1), abort)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = su32(sA + (size_t)s * a_bytes), b0 = su32(sB + (size_t)s * b_bytes);
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk)
                        umma_bf16(d_tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (kb | kk) != 0);
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&tfull[buf]);
            }
        }
    } else {
        // ---- epilogue: warp w drains TMEM lanes 32*(w%4) .. +31
        const int quad = warp & 3;
        uint8_t* stg = sC + (size_t)(warp - 2) * TC_STAGE_BYTES_PER_WARP;
        int64_t acc = 0;
        int chunk = 0;
        for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x, ++acc) {
            const int buf = (int)(acc & 1);
            if (!mbar_wait_or_abort(&tfull[buf], (uint32_t)((acc >> 1) & 1), abort)) break;
            tc_fence_after();
            const int64_t row0 = (t / n_tiles_n) * TC_BM + quad * 32;
            const int n0 = (int)(t % n_tiles_n) * BN;
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * (tmem_cols >> 1));
            if constexpr (TMA_EPI) {
                // 128-byte chunks: 32 fp32 or 64 bf16 columns
                constexpr int CW = (EPI == TF_EPI_STORE || EPI == TF_EPI_RESID) ? 32 : 64;
                for (int c = 0; c < BN; c += CW, ++chunk) {
                    uint8_t* sbuf = EPI == TF_EPI_GELU2 ? stg : stg + (chunk & 1) * 4096;
                    // the buffer's previous TMA store must have finished reading it
                    if (lane == 0) {
                        if (EPI == TF_EPI_GELU2) bulk_wait_read<0>();
                        else bulk_wait_read<1>();
                    }
                    __syncwarp();
#pragma unroll
                    for (int p = 0; p < CW / 16; ++p) {
                        float v16[16];
                        tmem_ld16(tbase + (uint32_t)(c + 16 * p), v16);
                        stage16<EPI>(v16, bias, n0 + c + 16 * p, p, su32(sbuf), lane);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0 && row0 < M) {
                        if (EPI == TF_EPI_RESID) tma_reduce_add_2d(&tmC, sbuf, n0 + c, (int)row0);
                        else tma_store_2d(&tmC, sbuf, n0 + c, (int)row0);
                        if (EPI == TF_EPI_GELU2) tma_store_2d(&tmC, sbuf + 4096, N + n0 + c, (int)row0);
                    }
                    if (lane == 0) bulk_commit();
                }
            } else {
                const int64_t row = row0 + lane;
                for (int c = 0; c < BN; c += 16) {
                    float v16[16];
                    tmem_ld16(tbase + (uint32_t)c, v16);
                    if (row < M) epilogue16<EPI>(v16, bias, Cv, row, N, n0 + c);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        // the staging buffers (and the results) must be complete before the CTA exits
        if (TMA_EPI && lane == 0) bulk_wait_all();
        __syncwarp();
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

// rows x cols row-major matrix of bf16 (or fp32), box of box_rows x (128 bytes of columns)
int make_map(CUtensorMap* map, const void* base, int64_t rows, int cols, int box_rows, bool fp32 = false) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled is unavailable"); return NQS_ERR_CUDA; }
    const int esz = fp32 ? 4 : 2;
    if (((uintptr_t)base & 15) || ((cols * esz) & 15)) { set_error("TMA operand must be 16-byte aligned"); return NQS_ERR_INVALID_ARG; }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr,
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
    // that two CTAs, each with two accumulators of up to 128 columns, share an SM's TMEM
    int BN = N;
    if (N > 128) {
        BN = 0;
        for (int b = 128; b >= 16; b -= 16)
            if (N % b == 0) { BN = b; break; }
    }
    if (BN == 0 || BN % 16 || N % BN) { set_error("tensor-core GEMM: unsupported N"); return NQS_ERR_UNSUPPORTED; }
    // two TMEM accumulators, each a power of two >= BN columns wide; the stage ring fills
    // ~96 KB, so two CTAs share an SM
    int tcols = 64;
    while (tcols < 2 * BN) tcols <<= 1;
    // staged TMA epilogue when the tile splits into 128-byte column chunks (32 fp32, 64 bf16)
    const bool f32_out = epi == TF_EPI_STORE || epi == TF_EPI_RESID;
    const bool tma_epi = BN % (f32_out ? 32 : 64) == 0 && ((uintptr_t)C & 15) == 0;
    const size_t stage_bytes = TC_BM * 128 + (size_t)BN * 128;
    const size_t staging = tma_epi ? 4 * TC_STAGE_BYTES_PER_WARP : 0;
    // fill ~104 KB per CTA with ring stages (at least two) so that two CTAs share an SM
    const int stages = (int)std::max<size_t>(2, std::min<size_t>(6, (104 * 1024 - staging) / stage_bytes));
    const size_t smem = 1024 + (size_t)stages * stage_bytes + staging + (2 * stages + 4) * 8 + 16;
    if (smem > 220 * 1024) { set_error("tensor-core GEMM: shared-memory plan too large"); return NQS_ERR_UNSUPPORTED; }
    CUtensorMap ma, mb, mc;
    NQS_TRY(make_map(&ma, A, M, K, TC_BM));
    NQS_TRY(make_map(&mb, W, N, K, BN));
    if (tma_epi) NQS_TRY(make_map(&mc, C, M, epi == TF_EPI_GELU2 ? 2 * N : N, 32, f32_out));
    else memset(&mc, 0, sizeof(mc));
    const int n_tiles_n = N / BN;
    const int64_t total_tiles = ((M + TC_BM - 1) / TC_BM) * n_tiles_n;
    const int ctas_per_sm = (int)std::max<int64_t>(1, std::min<int64_t>(512 / tcols, (228 * 1024) / (smem + 1024)));
    const int grid = (int)std::min<int64_t>(total_tiles, (int64_t)num_sms() * ctas_per_sm);
    auto launch = [&](auto kernel) -> int {
        // raise the dynamic shared-memory limit once per kernel (and device), outside any
        // stream capture that later launches may run under
        static int configured_device[16] = {-1, -1, -1, -1, -1, -1, -1, -1,
                                            -1, -1, -1, -1, -1, -1, -1, -1};   // per (epilogue, staging)
        const int slot = (epi & 7) * 2 + (tma_epi ? 1 : 0);
        int dev = 0;
        NQS_CK(cudaGetDevice(&dev));
        if (configured_device[slot] != dev) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_gemm)", __FILE__, __LINE__);
            configured_device[slot] = dev;
        }
        kernel<<<grid, TC_THREADS, smem, s>>>(ma, mb, mc, bias, C, M, N, K, BN, tcols, stages, n_tiles_n, total_tiles);
        NQS_LAUNCHED();
        return NQS_OK;
    };
    switch (epi * 2 + (tma_epi ? 1 : 0)) {
        case TF_EPI_STORE * 2: return launch(tc_gemm_kernel<TF_EPI_STORE, false>);
        case TF_EPI_STORE * 2 + 1: return launch(tc_gemm_kernel<TF_EPI_STORE, true>);
        case TF_EPI_RESID * 2: return launch(tc_gemm_kernel<TF_EPI_RESID, false>);
        case TF_EPI_RESID * 2 + 1: return launch(tc_gemm_kernel<TF_EPI_RESID, true>);
        case TF_EPI_GELU * 2: return launch(tc_gemm_kernel<TF_EPI_GELU, false>);
        case TF_EPI_GELU * 2 + 1: return launch(tc_gemm_kernel<TF_EPI_GELU, true>);
        case TF_EPI_GELU2 * 2: return launch(tc_gemm_kernel<TF_EPI_GELU2, false>);
        case TF_EPI_GELU2 * 2 + 1: return launch(tc_gemm_kernel<TF_EPI_GELU2, true>);
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
