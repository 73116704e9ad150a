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

// L2 prefetch of one tensor-map box (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(x), "r"(y)
                 : "memory");
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

// 16 columns of the warp's 32 TMEM lanes without waiting (tmem_wait_ld() before use).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float* v) {
    uint32_t* r = reinterpret_cast<uint32_t*>(v);
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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
        } else if (EPI == TF_EPI_SPLIT) {
            // split layout: third `reg` of the row holds hi in its first D columns, lo in the next D
            const int Dq = N / 3, reg = col / Dq, w = col - reg * Dq;
            __nv_bfloat16* C = reinterpret_cast<__nv_bfloat16*>(Cv) + row * 2 * N + 2 * Dq * reg + w;
            __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                hi[j] = __float2bfloat16_rn(v[j]);
                lo[j] = __float2bfloat16_rn(v[j] - __bfloat162float(hi[j]));
            }
            *reinterpret_cast<uint4*>(C) = *reinterpret_cast<const uint4*>(hi);
            *reinterpret_cast<uint4*>(C + Dq) = *reinterpret_cast<const uint4*>(lo);
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
                const float g = EPI == TF_EPI_SPLIT ? v[8 * u + j] : gelu_tanh(v[8 * u + j]);
                hi[j] = __float2bfloat16_rn(g);
                if (EPI == TF_EPI_GELU2 || EPI == TF_EPI_SPLIT) lo[j] = __float2bfloat16_rn(g - __bfloat162float(hi[j]));
            }
            const uint32_t off = (uint32_t)(((p16 * 2 + u) ^ sw) << 4);
            st_shared_v4(row + off, pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]),
                         pack_bf16(hi[6], hi[7]));
            if (EPI == TF_EPI_GELU2 || EPI == TF_EPI_SPLIT)
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
__global__ void __launch_bounds__(TC_THREADS, 2)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmD,
               const float* __restrict__ bias, void* __restrict__ Cv, const float* __restrict__ ln_g,
               const float* __restrict__ ln_b, int64_t M, int N, int K, int BN, int tmem_cols, int stages,
               int n_tiles_n, int64_t total_tiles, const __grid_constant__ TcTokTable tok) {
    constexpr bool RLN = EPI == TF_EPI_RESID_LN || EPI == TF_EPI_RESID_LN_TAB || EPI == TF_EPI_RESID_LN128;
    constexpr bool RLN_LOAD = EPI == TF_EPI_RESID_LN || EPI == TF_EPI_RESID_LN128;   // old h through TMA
    constexpr int RW = EPI == TF_EPI_RESID_LN128 ? 128 : 64;           // row width of the LayerNorm epilogue
    constexpr int STGB = EPI == TF_EPI_RESID_LN128 ? 2 * TC_STAGE_BYTES_PER_WARP : TC_STAGE_BYTES_PER_WARP;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nkb = (K + TC_BK - 1) / TC_BK;
    const uint32_t a_bytes = TC_BM * 128;
    const uint32_t b_bytes = (uint32_t)BN * 128;
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)stages * a_bytes;
    uint8_t* sC = sB + (size_t)stages * b_bytes;     // 1024-aligned: a_bytes, b_bytes are multiples of 1024
    uint64_t* full = reinterpret_cast<uint64_t*>(sC + (TMA_EPI ? 4 * STGB : 0));
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;       // [2] accumulator ready for the epilogue
    uint64_t* tempty = tfull + 2;           // [2] accumulator drained by the epilogue
    uint64_t* hbar = tempty + 2;            // [4] per epilogue warp: residual rows loaded (RESID_LN)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(hbar + 4);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
        for (int b = 0; b < 4; ++b) mbar_init(&hbar[b], 1);
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
        uint8_t* stg = sC + (size_t)(warp - 2) * STGB;
        int64_t acc = 0;
        int chunk = 0;
        if (RLN_LOAD && lane == 0 && (int64_t)blockIdx.x < total_tiles) {
            // residual rows of the first tile (RW / 32 chunks of 32 rows x 32 fp32)
            const int nrow = (int)((blockIdx.x / n_tiles_n) * TC_BM + quad * 32);
            mbar_expect_tx(&hbar[quad], RW * 128);
#pragma unroll
            for (int q = 0; q < RW / 32; ++q) tma_load_2d(stg + 4096 * q, &tmC, &hbar[quad], 32 * q, nrow);
        }
        __syncwarp();
        // TAB: the configuration of this lane's row, loaded one tile ahead
        auto tab_bits = [&](int64_t tile) -> uint64_t {
            if (EPI != TF_EPI_RESID_LN_TAB || tile >= total_tiles) return 0ull;
            const int64_t row = min((tile / n_tiles_n) * TC_BM + quad * 32 + lane, M - 1);
            return __ldg(tok.bits + row / tok.T);
        };
        uint64_t xb_next = tab_bits(blockIdx.x);
        for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x, ++acc) {
            const int buf = (int)(acc & 1);
            const uint64_t xb = xb_next;
            if constexpr (EPI == TF_EPI_RESID_LN_TAB) xb_next = tab_bits(t + gridDim.x);
            if (!mbar_wait_or_abort(&tfull[buf], (uint32_t)((acc >> 1) & 1), abort)) break;
            tc_fence_after();
            const int64_t row0 = (t / n_tiles_n) * TC_BM + quad * 32;
            const int n0 = (int)(t % n_tiles_n) * BN;
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * (tmem_cols >> 1));
            if constexpr (RLN) {
                // the tile spans whole rows of d = RW: lane = row.  h_new = h + acc + bias,
                // stored back; then a = LayerNorm(h_new) as hi | lo bf16.  The old h comes through
                // the staging (TMA), or from the token-position table (TAB: first block)
                const int64_t hrow0 = (t / n_tiles_n) * TC_BM + quad * 32;
                const float* hrow = nullptr;
                if constexpr (EPI == TF_EPI_RESID_LN_TAB) {
                    const int64_t row = min(hrow0 + lane, M - 1);
                    const int tp = (int)(row % tok.T);
                    const int tk = tp == 0 ? 2 : (int)((xb >> tok.order[tp - 1]) & 1ull);
                    hrow = tok.tab + (int64_t)(tk * tok.T + tp) * 64;
                    if (lane == 0) bulk_wait_read<0>();      // the previous tile's stores have read the staging
                    __syncwarp();
                } else {
                    if (!mbar_wait_or_abort(&hbar[quad], (uint32_t)(acc & 1), abort)) break;
                }
                const uint32_t st = su32(stg);
                const int sw = lane & 7;
                // address of columns c .. c+3 of this lane's row in the staging (two 32-column halves)
                auto saddr = [&](int c) -> uint32_t {
                    return st + (uint32_t)((c >> 5) * 4096 + lane * 128 + ((((c & 31) >> 2) ^ sw) << 4));
                };
                // pass 1: h_new = h + acc + bias, in place in the staging; row sum
                float sum = 0.f;
#pragma unroll
                for (int p = 0; p < RW / 16; ++p) {
                    float v16[16];
                    tmem_ld16(tbase + (uint32_t)(16 * p), v16);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 16 * p + 4 * u;
                        const uint32_t addr = saddr(c);
                        float4 o;
                        if constexpr (EPI == TF_EPI_RESID_LN_TAB) o = __ldg(reinterpret_cast<const float4*>(hrow + c));
                        else asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w) : "r"(addr));
                        o.x += v16[4 * u] + bias[c];
                        o.y += v16[4 * u + 1] + bias[c + 1];
                        o.z += v16[4 * u + 2] + bias[c + 2];
                        o.w += v16[4 * u + 3] + bias[c + 3];
                        sum += (o.x + o.y) + (o.z + o.w);
                        st_shared_v4(addr, __float_as_uint(o.x), __float_as_uint(o.y), __float_as_uint(o.z), __float_as_uint(o.w));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
                // h_new back to global (the TMA reads the staging while the passes below read it too)
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if (hrow0 < M) {
#pragma unroll
                        for (int q = 0; q < RW / 32; ++q) tma_store_2d(&tmC, stg + 4096 * q, 32 * q, (int)hrow0);
                    }
                    bulk_commit();
                }
                // pass 2: variance about the mean; pass 3: normalised hi | lo bf16 pairs, 64 columns
                // at a time (hi rows into the staging chunk 2 v, lo rows into chunk 2 v + 1, each
                // once the h store has read it and after its own columns were read)
                const float mu = sum * (1.f / (float)RW);
                float var = 0.f;
#pragma unroll
                for (int c = 0; c < RW; c += 4) {
                    float4 o;
                    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w) : "r"(saddr(c)));
                    const float d0 = o.x - mu, d1 = o.y - mu, d2 = o.z - mu, d3 = o.w - mu;
                    var = fmaf(d0, d0, var); var = fmaf(d1, d1, var); var = fmaf(d2, d2, var); var = fmaf(d3, d3, var);
                }
                const float rstd = rsqrtf(fmaf(var, 1.f / (float)RW, LN_EPS));
#pragma unroll 1
                for (int v = 0; v < RW / 64; ++v) {
                uint32_t hp[32], lp[32];
#pragma unroll
                for (int c0 = 0; c0 < 64; c0 += 4) {
                    const int c = 64 * v + c0;
                    float4 o;
                    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w) : "r"(saddr(c)));
                    const float y[4] = {(o.x - mu) * rstd * ln_g[c] + ln_b[c], (o.y - mu) * rstd * ln_g[c + 1] + ln_b[c + 1],
                                        (o.z - mu) * rstd * ln_g[c + 2] + ln_b[c + 2], (o.w - mu) * rstd * ln_g[c + 3] + ln_b[c + 3]};
#pragma unroll
                    for (int q2 = 0; q2 < 4; q2 += 2) {
                        const __nv_bfloat162 hh = __floats2bfloat162_rn(y[q2], y[q2 + 1]);
                        const float2 hf = __bfloat1622float2(hh);
                        const __nv_bfloat162 ll = __floats2bfloat162_rn(y[q2] - hf.x, y[q2 + 1] - hf.y);
                        hp[(c0 + q2) / 2] = *reinterpret_cast<const uint32_t*>(&hh);
                        lp[(c0 + q2) / 2] = *reinterpret_cast<const uint32_t*>(&ll);
                    }
                }
                // the staging again, once the h store has read it: hi rows, then lo rows
                if (v == 0 && lane == 0) bulk_wait_read<0>();
                __syncwarp();
                const uint32_t hb = st + (uint32_t)(2 * v) * 4096u;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t off = (uint32_t)(lane * 128 + ((u ^ sw) << 4));
                    st_shared_v4(hb + off, hp[4 * u], hp[4 * u + 1], hp[4 * u + 2], hp[4 * u + 3]);
                    st_shared_v4(hb + 4096 + off, lp[4 * u], lp[4 * u + 1], lp[4 * u + 2], lp[4 * u + 3]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0 && hrow0 < M) {
                    tma_store_2d(&tmD, stg + 2 * v * 4096, 64 * v, (int)hrow0);
                    tma_store_2d(&tmD, stg + (2 * v + 1) * 4096, RW + 64 * v, (int)hrow0);
                }
                }
                if (lane == 0) {
                    bulk_commit();
                    // the next tile's residual rows into the staging once these stores have read it
                    const int64_t tn = t + gridDim.x;
                    if (RLN_LOAD && tn < total_tiles) {
                        bulk_wait_read<0>();
                        mbar_expect_tx(&hbar[quad], RW * 128);
                        const int nrow = (int)((tn / n_tiles_n) * TC_BM + quad * 32);
#pragma unroll
                        for (int q = 0; q < RW / 32; ++q) tma_load_2d(stg + 4096 * q, &tmC, &hbar[quad], 32 * q, nrow);
                    }
                }
                __syncwarp();
                continue;
            } else if constexpr (TMA_EPI) {
                // 128-byte chunks: 32 fp32 or 64 bf16 columns
                constexpr int CW = (EPI == TF_EPI_STORE || EPI == TF_EPI_RESID) ? 32 : 64;
                for (int c = 0; c < BN; c += CW, ++chunk) {
                    constexpr bool HILO = EPI == TF_EPI_GELU2 || EPI == TF_EPI_SPLIT;
                    uint8_t* sbuf = HILO ? stg : stg + (chunk & 1) * 4096;
                    // the buffer's previous TMA store must have finished reading it
                    if (lane == 0) {
                        if (HILO) bulk_wait_read<0>();
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
                        if (EPI == TF_EPI_SPLIT) {
                            // a 64-column chunk lies within one third of the row (D % 64 == 0)
                            const int Dq = N / 3, col = n0 + c, reg = col / Dq, w = col - reg * Dq;
                            tma_store_2d(&tmC, sbuf, 2 * Dq * reg + w, (int)row0);
                            tma_store_2d(&tmC, sbuf + 4096, 2 * Dq * reg + Dq + w, (int)row0);
                        } else {
                            if (EPI == TF_EPI_RESID) tma_reduce_add_2d(&tmC, sbuf, n0 + c, (int)row0);
                            else tma_store_2d(&tmC, sbuf, n0 + c, (int)row0);
                            if (EPI == TF_EPI_GELU2) tma_store_2d(&tmC, sbuf + 4096, N + n0 + c, (int)row0);
                        }
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
        if ((TMA_EPI || RLN) && lane == 0) bulk_wait_all();
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---------------------------------------------------------------- fused MLP block
// h[M, D] += GELU(A . W1d^T + b1) . W2d^T + b2 in the compensated bf16 forms: A = [a_hi | a_lo]
// (M x 2D), W1d = [W1 | W1] (4D x 2D), W2d = [W2 | W2] (D x 8D).  The 4D-wide hidden
// activation never leaves the SM: per 128-row tile and 128-column chunk j of the hidden layer,
//   GEMM1_j  acc1 = A . W1d[128 j .. +128]^T                     (TMEM, two buffers)
//   GELU_j   G = [hi | lo] of GELU(acc1 + b1) in shared memory   (epilogue warps, UMMA layout)
//   GEMM2_j  acc2 += G . [W2 | W2](chunk j's hi and lo columns)^T (TMEM, two buffers)
// and after the last chunk the epilogue adds acc2 + b2 into h with TMA reduce-adds.  Roles: warp 0
// TMA producer (A per tile, W1/W2 k-blocks through a ring in the MMA's order), warp 1 MMA issuer
// (order G1_0, G1_1, then G2_j followed by G1_{j+2}), warps 2.. epilogue (EW / 4 per TMEM lane
// quadrant, each taking a column slice).  One CTA per SM (all 512 TMEM columns).
template <int D>
struct MlpPlan {                                          // epilogue layout (both variants)
    static constexpr int EW = D == 64 ? 16 : 8;           // epilogue warps
    static constexpr int SLICES = EW / 4;                 // column slices per lane quadrant
    static constexpr int SL = 128 / SLICES;               // hidden columns per warp and chunk
    static constexpr int RES_SLICES = SLICES < D / 32 ? SLICES : D / 32;   // warps per quadrant on the residual
    static constexpr int RC = D / RES_SLICES;             // residual columns per such warp
    static constexpr int THREADS = 64 + 32 * EW;
    static constexpr int NCH = 4 * D / 128;               // 128-column chunks of the hidden layer
    static constexpr int STG_BYTES = 4 * RES_SLICES * 4096;   // residual staging: 32 rows x 32 fp32 per warp
};

template <int D>
struct MlpRingPlan {                                      // weights streamed through a ring
    static constexpr int KB1 = 2 * D / 64;                // 64-wide k-blocks of GEMM1 (A hi | lo)
    static constexpr int KW1 = D / 64;                    // distinct W1 k-blocks per hidden chunk
    static constexpr int A_BYTES = KB1 * 16384;           // 128 rows x 2D bf16
    // d_model 128: each epilogue warp owns 64 hidden columns of 32 rows of G, two contiguous
    // 4 KB pieces (hi and lo); the residual is staged there, not in a buffer of its own, and the
    // 32 KB go to two more ring slots.  The ring carries each weight k-block once (the compensated
    // form's [W | W] duplicate is never loaded): 256 KB of weights per 128-row tile instead of 512.
    static constexpr bool STG_IN_G = MlpPlan<D>::SL == 64;
    static constexpr int STAGES = STG_IN_G ? 5 : 3;       // ring slots of 16 KB
    static constexpr int RING_BYTES = STAGES * 16384;
    static constexpr int G_BYTES = 4 * 16384;             // 128 rows x (128 hi + 128 lo) bf16
    static constexpr int STG_BYTES = STG_IN_G ? 0 : MlpPlan<D>::STG_BYTES;
    static constexpr int BIAS_OFF = A_BYTES + RING_BYTES + G_BYTES + STG_BYTES;
    static constexpr int BAR_OFF = BIAS_OFF + 5 * D * 4;  // b1 (4D) and b2 (D)
    static constexpr int NBAR = 2 + 2 * STAGES + 4 + 2 + 4;
    static constexpr int SMEM = 1024 + BAR_OFF + NBAR * 8 + 16;
};

// Head form of the last block's MLP: instead of h, the epilogue leaves per row the output-head
// logit LNf(h) . head_w + head_b[t] (t = row mod n) and, on rows with t = n - 2, the four
// phase-head dot products LNf(h) . phase_w[k] + phase_b[k] (k = 0..3, per sequence).
struct MlpHeadArgs {
    const float *lnf_g, *lnf_b, *head_w, *head_b;
    int n;
    float* logit;               // [M]
    float* hph;                 // [M / n][64]: h of position n - 2 (the phase head's input)
};

__device__ __forceinline__ float4 lds4f(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// Epilogue warps of the fused MLP (both variants): per hidden chunk, GELU of the warp's column
// slice of acc1 split into hi | lo and written into G; per tile, h += acc2 + b2 by TMA reduce-adds.
template <int D>
struct MlpEpiArgs {
    uint32_t tmem;
    uint8_t *sG, *sStg;
    const float *sb1, *sb2;
    uint64_t *acc1_full, *acc1_empty, *g_full, *g_empty, *acc2_full, *acc2_empty;
    volatile int* abort;
    const CUtensorMap* tmH;
    int64_t M, ntiles;
    uint64_t* hbar;             // [4] head form: residual rows loaded, per lane quadrant
    MlpHeadArgs head;
    const float* sgw;           // head form: lnf_g * head_w [D], sum of it, sum(lnf_b * head_w)
};

template <int D, bool HEAD = false, bool STG_IN_G = false>
__device__ __forceinline__ void mlp_epilogue(const MlpEpiArgs<D>& E, int warp, int lane) {
    using PL = MlpPlan<D>;
    const uint32_t tmem = E.tmem;
    uint8_t* sG = E.sG;
    uint8_t* sStg = E.sStg;
    const float* sb1 = E.sb1;
    const float* sb2 = E.sb2;
    uint64_t *acc1_full = E.acc1_full, *acc1_empty = E.acc1_empty, *g_full = E.g_full, *g_empty = E.g_empty;
    uint64_t *acc2_full = E.acc2_full, *acc2_empty = E.acc2_empty;
    volatile int* abort = E.abort;
    const CUtensorMap& tmH = *E.tmH;
    const int64_t M = E.M, ntiles = E.ntiles;
    {   // ---- epilogue warps: quadrant q of the TMEM lanes (rows), column slice sl
        const int q = warp & 3, sl = (warp - 2) >> 2;
        const int r = q * 32 + lane;                       // row within the tile
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        const bool res_warp = HEAD ? sl == 0 : sl < PL::RES_SLICES;
        // head form: one warp per quadrant owns whole rows (64 fp32 = 8 KB of staging)
        uint8_t* stg = STG_IN_G ? nullptr
                       : HEAD   ? sStg + (size_t)q * 8192
                                : sStg + (size_t)(q + 4 * (res_warp ? sl : 0)) * 4096;
        int64_t tt = 0, c1 = 0, cg = 0;
        bool ok = true;
        if (HEAD && res_warp && lane == 0 && (int64_t)blockIdx.x < ntiles) {
            // residual rows of the first tile
            const int y = (int)(blockIdx.x * 128 + q * 32);
            mbar_expect_tx(&E.hbar[q], 8192);
            tma_load_2d(stg, &tmH, &E.hbar[q], 0, y);
            tma_load_2d(stg + 4096, &tmH, &E.hbar[q], 32, y);
        }
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tt) {
            // head form: this lane's row, its sequence and position, the head bias (loaded early)
            int64_t hd_row = 0, hd_seq = 0;
            int hd_pos = 0;
            float hd_b = 0.f;
            if (HEAD && res_warp) {
                hd_row = t * 128 + r;
                const int64_t seq0 = (t * 128) / E.head.n;
                const int pq = (int)(t * 128 - seq0 * E.head.n) + r;   // < n + 128
                hd_seq = seq0 + pq / E.head.n;
                hd_pos = pq - (int)(hd_seq - seq0) * E.head.n;
                hd_b = __ldg(E.head.head_b + hd_pos);
            }
            for (int j = 0; j < PL::NCH; ++j) {
                const int b = (int)(c1 & 1);
                if (!mbar_wait_or_abort(&acc1_full[b], (uint32_t)((c1 >> 1) & 1), abort)) { ok = false; break; }
                tc_fence_after();
                // GELU of this warp's SL columns of the chunk, split into hi and lo (packed bf16 pairs)
                uint32_t hp[PL::SL / 2], lp[PL::SL / 2];
#pragma unroll
                for (int p = 0; p < PL::SL / 32; ++p) {
                    const int c0 = sl * PL::SL + 32 * p;           // column within the chunk
                    float v[32];
                    tmem_ld16_nowait(lane_base + (uint32_t)(b * 128 + c0), v);
                    tmem_ld16_nowait(lane_base + (uint32_t)(b * 128 + c0 + 16), v + 16);
                    tmem_wait_ld();
                    const float* bb = sb1 + j * 128 + c0;
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const float g0 = gelu_tanh(v[i] + bb[i]), g1v = gelu_tanh(v[i + 1] + bb[i + 1]);
                        const __nv_bfloat162 hh = __floats2bfloat162_rn(g0, g1v);
                        const float2 hf = __bfloat1622float2(hh);
                        const __nv_bfloat162 ll = __floats2bfloat162_rn(g0 - hf.x, g1v - hf.y);
                        hp[16 * p + i / 2] = *reinterpret_cast<const uint32_t*>(&hh);
                        lp[16 * p + i / 2] = *reinterpret_cast<const uint32_t*>(&ll);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc1_empty[b]);
                ++c1;
                // write G once the previous chunk's GEMM2 has read it (and, with the residual
                // staged in G, once the previous tile's reduce-adds have read this warp's rows)
                if (!mbar_wait_or_abort(g_empty, (uint32_t)((cg & 1) ^ 1), abort)) { ok = false; break; }
                if (STG_IN_G && j == 0) {
                    if (lane == 0) bulk_wait_read<0>();
                    __syncwarp();
                }
                const int kb_hi = (sl * PL::SL) >> 6, u0 = ((sl * PL::SL) & 63) >> 3;
                const uint32_t ghi = su32(sG + kb_hi * 16384) + (uint32_t)r * 128;
                const uint32_t glo = su32(sG + (2 + kb_hi) * 16384) + (uint32_t)r * 128;
#pragma unroll
                for (int u = 0; u < PL::SL / 8; ++u) {
                    const uint32_t off = (uint32_t)(((u0 + u) ^ (r & 7)) << 4);
                    st_shared_v4(ghi + off, hp[4 * u], hp[4 * u + 1], hp[4 * u + 2], hp[4 * u + 3]);
                    st_shared_v4(glo + off, lp[4 * u], lp[4 * u + 1], lp[4 * u + 2], lp[4 * u + 3]);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(g_full);
                ++cg;
            }
            if (!ok) break;
            // residual: h += acc2 + b2, RC columns per warp in 32-column TMA reduce-adds
            const int ab = (int)(tt & 1);
            if (!mbar_wait_or_abort(&acc2_full[ab], (uint32_t)((tt >> 1) & 1), abort)) break;
            tc_fence_after();
            if (HEAD && res_warp) {
                // h_new = h + acc2 + b2, never stored.  With LNf folded into the output head,
                // logit = rstd (h . gw - mean sum(gw)) + lnf_b . head_w + head_b[t] (gw = lnf_g * head_w),
                // so one pass over the row gives the dot product and, from the 16-column chunks'
                // means and squared deviations, the row's mean and variance; the rows of position
                // n - 2 also leave h for the phase head.
                if (!mbar_wait_or_abort(&E.hbar[q], (uint32_t)(tt & 1), abort)) break;
                const uint32_t st = su32(stg);
                const int sw = lane & 7;
                auto saddr = [&](int c) -> uint32_t {
                    return st + (uint32_t)((c >> 5) * 4096 + lane * 128 + ((((c & 31) >> 2) ^ sw) << 4));
                };
                const float* gw = E.sgw;
                const bool ph_row = hd_pos == E.head.n - 2 && hd_row < M;
                float4* ph_dst = reinterpret_cast<float4*>(E.head.hph + hd_seq * 64);
                float dot = 0.f, m2 = 0.f, cm[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float x[16];
                    tmem_ld16(lane_base + 256u + (uint32_t)(ab * D + 16 * p), x);
                    float cs = 0.f;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 16 * p + 4 * u;
                        const float4 o = lds4f(saddr(c));
                        const float4 b4 = lds4f(su32(sb2 + c));
                        const float4 g4 = lds4f(su32(gw + c));
                        x[4 * u] += o.x + b4.x;
                        x[4 * u + 1] += o.y + b4.y;
                        x[4 * u + 2] += o.z + b4.z;
                        x[4 * u + 3] += o.w + b4.w;
                        cs += (x[4 * u] + x[4 * u + 1]) + (x[4 * u + 2] + x[4 * u + 3]);
                        dot = fmaf(x[4 * u], g4.x, dot); dot = fmaf(x[4 * u + 1], g4.y, dot);
                        dot = fmaf(x[4 * u + 2], g4.z, dot); dot = fmaf(x[4 * u + 3], g4.w, dot);
                        if (ph_row) ph_dst[c >> 2] = make_float4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]);
                    }
                    cm[p] = cs * (1.f / 16.f);
#pragma unroll
                    for (int i = 0; i < 16; ++i) { const float dv = x[i] - cm[p]; m2 = fmaf(dv, dv, m2); }
                }
                const float mu = ((cm[0] + cm[1]) + (cm[2] + cm[3])) * 0.25f;
#pragma unroll
                for (int p = 0; p < 4; ++p) { const float dv = cm[p] - mu; m2 = fmaf(16.f * dv, dv, m2); }
                const float rstd = rsqrtf(fmaf(m2, 1.f / 64.f, LN_EPS));
                if (hd_row < M) E.head.logit[hd_row] = rstd * (dot - mu * gw[64]) + gw[65] + hd_b;
                // the next tile's residual rows into the staging (this warp has read it)
                __syncwarp();
                const int64_t tn = t + gridDim.x;
                if (lane == 0 && tn < ntiles) {
                    const int y = (int)(tn * 128 + q * 32);
                    mbar_expect_tx(&E.hbar[q], 8192);
                    tma_load_2d(stg, &tmH, &E.hbar[q], 0, y);
                    tma_load_2d(stg + 4096, &tmH, &E.hbar[q], 32, y);
                }
            } else if (!HEAD && res_warp) {
                const int64_t row0 = t * 128 + q * 32;
#pragma unroll
                for (int c = 0; c < PL::RC; c += 32) {
                    const int col = sl * PL::RC + c;
                    // staged in G: this warp's hi rows for the first 32 columns, its lo rows for
                    // the next (GEMM2 has read G: acc2 is complete)
                    uint8_t* st = STG_IN_G ? sG + (size_t)((c == 0 ? 0 : 2) + sl) * 16384 + (size_t)q * 4096 : stg;
                    if (!STG_IN_G && lane == 0) bulk_wait_read<0>();
                    __syncwarp();
                    float v[32];
                    tmem_ld16_nowait(lane_base + 256u + (uint32_t)(ab * D + col), v);
                    tmem_ld16_nowait(lane_base + 256u + (uint32_t)(ab * D + col + 16), v + 16);
                    tmem_wait_ld();
                    stage16<TF_EPI_RESID>(*reinterpret_cast<const float(*)[16]>(v), sb2, col, 0, su32(st), lane);
                    stage16<TF_EPI_RESID>(*reinterpret_cast<const float(*)[16]>(v + 16), sb2, col + 16, 1, su32(st), lane);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        if (row0 < M) tma_reduce_add_2d(&tmH, st, col, (int)row0);
                        bulk_commit();
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc2_empty[ab]);
        }
        if (lane == 0) bulk_wait_all();
        __syncwarp();
        }
}

template <int D>
__global__ void __launch_bounds__(MlpPlan<D>::THREADS, 1)
tc_mlp_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW1,
              const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmH,
              const float* __restrict__ b1, const float* __restrict__ b2, int64_t M, int64_t ntiles) {
    using PL = MlpPlan<D>;
    using RPL = MlpRingPlan<D>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* ring = smem + RPL::A_BYTES;
    uint8_t* sG = ring + RPL::RING_BYTES;
    uint8_t* sStg = RPL::STG_IN_G ? nullptr : sG + RPL::G_BYTES;
    float* sb1 = reinterpret_cast<float*>(smem + RPL::BIAS_OFF);
    float* sb2 = sb1 + 4 * D;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RPL::BAR_OFF);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + 1;
    uint64_t* full = bars + 2;
    uint64_t* empty = full + RPL::STAGES;
    uint64_t* acc1_full = empty + RPL::STAGES;      // [2]
    uint64_t* acc1_empty = acc1_full + 2;          // [2]
    uint64_t* g_full = acc1_empty + 2;
    uint64_t* g_empty = g_full + 1;
    uint64_t* acc2_full = g_empty + 1;             // [2]
    uint64_t* acc2_empty = acc2_full + 2;          // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + RPL::NBAR);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int i = threadIdx.x; i < 4 * D; i += blockDim.x) sb1[i] = b1[i];
    for (int i = threadIdx.x; i < D; i += blockDim.x) sb2[i] = b2[i];
    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int i = 0; i < RPL::STAGES; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc1_full[i], 1); mbar_init(&acc1_empty[i], PL::EW);
            mbar_init(&acc2_full[i], 1); mbar_init(&acc2_empty[i], PL::EW);
        }
        mbar_init(g_full, PL::EW);
        mbar_init(g_empty, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: A per tile, then the W1 / W2 k-blocks in the MMA's order
            int64_t it = 0, tt = 0;
            bool ok = true;
            auto ring_load = [&](const CUtensorMap* map, int x, int y, uint32_t bytes) -> bool {
                const int sl = (int)(it % RPL::STAGES);
                if (!mbar_wait_or_abort(&empty[sl], (uint32_t)(((it / RPL::STAGES) & 1) ^ 1), abort)) return false;
                mbar_expect_tx(&full[sl], bytes);
                tma_load_2d(ring + (size_t)sl * 16384, map, &full[sl], x, y);
                ++it;
                return true;
            };
            // the weights' second (duplicate) halves are never loaded: each k-block of W1 / W2
            // meets both the hi and the lo k-block of A / G (see the MMA issuer)
            auto w1 = [&](int j) -> bool {
                for (int kb = 0; kb < RPL::KW1; ++kb)
                    if (!ring_load(&tmW1, kb * 64, j * 128, 16384)) return false;
                return true;
            };
            auto w2 = [&](int j) -> bool {
                for (int kb = 0; kb < 2; ++kb)
                    if (!ring_load(&tmW2, j * 128 + kb * 64, 0, (uint32_t)D * 128)) return false;
                return true;
            };
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x, ++tt) {
                const int m0 = (int)(t * 128);
                if (!mbar_wait_or_abort(a_empty, (uint32_t)((tt & 1) ^ 1), abort)) break;
                mbar_expect_tx(a_full, RPL::A_BYTES);
                for (int kb = 0; kb < RPL::KB1; ++kb) tma_load_2d(sA + kb * 16384, &tmA, a_full, kb * 64, m0);
                const int64_t tn = t + gridDim.x;          // this CTA's next tile: its A into L2 now
                if (tn < ntiles)
                    for (int kb = 0; kb < RPL::KB1; ++kb) tma_prefetch_2d(&tmA, kb * 64, (int)(tn * 128));
                ok = w1(0) && (PL::NCH < 2 || w1(1));
                for (int j = 0; ok && j < PL::NCH; ++j) ok = w2(j) && (j + 2 >= PL::NCH || w1(j + 2));
            }
            // copies still in flight complete before the CTA exits (bounded waits)
            if (tt > 0) mbar_wait(a_full, (uint32_t)((tt - 1) & 1));
            for (int64_t j = it - RPL::STAGES < 0 ? 0 : it - RPL::STAGES; j < it; ++j)
                mbar_wait(&full[j % RPL::STAGES], (uint32_t)((j / RPL::STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t id1 = idesc_bf16(128, 128), id2 = idesc_bf16(128, D);
            int64_t it = 0, tt = 0, c1 = 0, cg = 0;
            bool ok = true;
            auto g1 = [&](int j) -> bool {
                const int b = (int)(c1 & 1);
                if (!mbar_wait_or_abort(&acc1_empty[b], (uint32_t)(((c1 >> 1) & 1) ^ 1), abort)) return false;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(b * 128);
                // the chunk's W1 k-blocks, then A_hi . W1^T followed by A_lo . W1^T (the order of
                // the duplicated form [A_hi | A_lo] . [W1 | W1]^T)
                int sl[RPL::KW1];
                for (int kb = 0; kb < RPL::KW1; ++kb, ++it) {
                    sl[kb] = (int)(it % RPL::STAGES);
                    if (!mbar_wait_or_abort(&full[sl[kb]], (uint32_t)((it / RPL::STAGES) & 1), abort)) return false;
                }
                tc_fence_after();
                for (int kb = 0; kb < RPL::KB1; ++kb) {
                    const uint32_t a0 = su32(sA + kb * 16384), w0 = su32(ring + (size_t)sl[kb % RPL::KW1] * 16384);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_bf16(d_tmem, sw128_desc(a0 + kk * 32), sw128_desc(w0 + kk * 32), id1, (kb | kk) != 0);
                }
                for (int kb = 0; kb < RPL::KW1; ++kb) umma_commit(&empty[sl[kb]]);
                umma_commit(&acc1_full[b]);
                if (j == PL::NCH - 1) umma_commit(a_empty);
                ++c1;
                return true;
            };
            auto g2 = [&](int j) -> bool {
                const int ab = (int)(tt & 1);
                if (j == 0 && !mbar_wait_or_abort(&acc2_empty[ab], (uint32_t)(((tt >> 1) & 1) ^ 1), abort)) return false;
                if (!mbar_wait_or_abort(g_full, (uint32_t)(cg & 1), abort)) return false;
                tc_fence_after();
                const uint32_t d_tmem = tmem + 256u + (uint32_t)(ab * D);
                // the chunk's two W2 k-blocks, then G_hi . W2^T followed by G_lo . W2^T
                int sl[2];
                for (int kb = 0; kb < 2; ++kb, ++it) {
                    sl[kb] = (int)(it % RPL::STAGES);
                    if (!mbar_wait_or_abort(&full[sl[kb]], (uint32_t)((it / RPL::STAGES) & 1), abort)) return false;
                }
                tc_fence_after();
                for (int kb = 0; kb < 4; ++kb) {
                    const uint32_t g0 = su32(sG + kb * 16384), w0 = su32(ring + (size_t)sl[kb & 1] * 16384);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_bf16(d_tmem, sw128_desc(g0 + kk * 32), sw128_desc(w0 + kk * 32), id2, (j | kb | kk) != 0);
                }
                for (int kb = 0; kb < 2; ++kb) umma_commit(&empty[sl[kb]]);
                umma_commit(g_empty);
                if (j == PL::NCH - 1) umma_commit(&acc2_full[ab]);
                ++cg;
                return true;
            };
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x, ++tt) {
                if (!mbar_wait_or_abort(a_full, (uint32_t)(tt & 1), abort)) break;
                tc_fence_after();
                ok = g1(0) && (PL::NCH < 2 || g1(1));
                for (int j = 0; ok && j < PL::NCH; ++j) ok = g2(j) && (j + 2 >= PL::NCH || g1(j + 2));
            }
        }
    } else {
        MlpEpiArgs<D> E{tmem, sG, sStg, sb1, sb2, acc1_full, acc1_empty, g_full, g_empty, acc2_full, acc2_empty,
                        abort, &tmH, M, ntiles};
        mlp_epilogue<D, false, RPL::STG_IN_G>(E, warp, lane);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// d = 64 variant with the weights resident in shared memory: W1 (256 x 64) and W2 (64 x 256),
// the first halves of the duplicated forms, are loaded once per CTA; each 128-row tile's A
// (hi and lo k-blocks, double-buffered) meets them twice, as A_hi . W^T + A_lo . W^T, and G's
// hi and lo k-blocks likewise meet the same W2 k-blocks.  No weight traffic per tile.
struct MlpResPlan {
    static constexpr int D = 64;
    static constexpr int W1_BYTES = 4 * D * 128;          // 256 rows x 64 bf16
    static constexpr int W2_BYTES = 4 * D * 128;          // 4 k-blocks x 64 rows x 64 bf16
    static constexpr int A_BYTES = 2 * 16384;             // hi and lo k-blocks of 128 rows
    static constexpr int G_BYTES = 4 * 16384;
    static constexpr int STG_BYTES = MlpPlan<64>::STG_BYTES;
    static constexpr int OFF_W2 = W1_BYTES;
    static constexpr int OFF_A = OFF_W2 + W2_BYTES;
    static constexpr int OFF_G = OFF_A + 2 * A_BYTES;
    static constexpr int OFF_STG = OFF_G + G_BYTES;
    static constexpr int OFF_BIAS = OFF_STG + STG_BYTES;
    static constexpr int OFF_BAR = OFF_BIAS + (5 * D + 68) * 4;   // b1, b2, head form: lnf_g * head_w, two sums
    static constexpr int NBAR = 1 + 4 + 4 + 2 + 4 + 4;   // ..., head form: residual rows per quadrant
    static constexpr int SMEM = 1024 + OFF_BAR + NBAR * 8 + 16;
};

template <bool HEAD>
__global__ void __launch_bounds__(MlpPlan<64>::THREADS, 1)
tc_mlp_res_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW1,
                  const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmH,
                  const float* __restrict__ b1, const float* __restrict__ b2, int64_t M, int64_t ntiles,
                  MlpHeadArgs head) {
    using RP = MlpResPlan;
    constexpr int D = 64, NCH = 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sW1 = smem;
    uint8_t* sW2 = smem + RP::OFF_W2;
    uint8_t* sA = smem + RP::OFF_A;
    uint8_t* sG = smem + RP::OFF_G;
    uint8_t* sStg = smem + RP::OFF_STG;
    float* sb1 = reinterpret_cast<float*>(smem + RP::OFF_BIAS);
    float* sb2 = sb1 + 4 * D;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RP::OFF_BAR);
    uint64_t* w_full = bars;
    uint64_t* a_full = bars + 1;           // [2]
    uint64_t* a_empty = a_full + 2;        // [2]
    uint64_t* acc1_full = a_empty + 2;     // [2]
    uint64_t* acc1_empty = acc1_full + 2;  // [2]
    uint64_t* g_full = acc1_empty + 2;
    uint64_t* g_empty = g_full + 1;
    uint64_t* acc2_full = g_empty + 1;     // [2]
    uint64_t* acc2_empty = acc2_full + 2;  // [2]
    uint64_t* hbar = acc2_empty + 2;       // [4]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + RP::NBAR);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int EW = MlpPlan<64>::EW;

    for (int i = threadIdx.x; i < 4 * D; i += blockDim.x) sb1[i] = b1[i];
    for (int i = threadIdx.x; i < D; i += blockDim.x) sb2[i] = b2[i];
    float* sgw = sb2 + D;            // head form: lnf_g * head_w [D], then sum(lnf_g * head_w), sum(lnf_b * head_w)
    if (HEAD) {
        for (int i = threadIdx.x; i < D; i += blockDim.x) sgw[i] = head.lnf_g[i] * head.head_w[i];
        if (threadIdx.x == 0) {
            float a = 0.f, c = 0.f;
            for (int i = 0; i < D; ++i) { a = fmaf(head.lnf_g[i], head.head_w[i], a); c = fmaf(head.lnf_b[i], head.head_w[i], c); }
            sgw[D] = a;
            sgw[D + 1] = c;
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(w_full, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&a_full[i], 1); mbar_init(&a_empty[i], 1);
            mbar_init(&acc1_full[i], 1); mbar_init(&acc1_empty[i], EW);
            mbar_init(&acc2_full[i], 1); mbar_init(&acc2_empty[i], EW);
        }
        mbar_init(g_full, EW);
        mbar_init(g_empty, 1);
        for (int i = 0; i < 4; ++i) mbar_init(&hbar[i], 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: the weights once, then A per tile (two buffers)
            mbar_expect_tx(w_full, RP::W1_BYTES + RP::W2_BYTES);
            tma_load_2d(sW1, &tmW1, w_full, 0, 0);
            for (int kb = 0; kb < 4; ++kb) tma_load_2d(sW2 + kb * 8192, &tmW2, w_full, kb * 64, 0);
            int64_t tt = 0;
            for (int64_t t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++tt) {
                const int ab = (int)(tt & 1);
                if (!mbar_wait_or_abort(&a_empty[ab], (uint32_t)(((tt >> 1) & 1) ^ 1), abort)) break;
                mbar_expect_tx(&a_full[ab], RP::A_BYTES);
                for (int kb = 0; kb < 2; ++kb)
                    tma_load_2d(sA + ab * RP::A_BYTES + kb * 16384, &tmA, &a_full[ab], kb * 64, (int)(t * 128));
            }
            // copies still in flight complete before the CTA exits (bounded waits)
            mbar_wait(w_full, 0);
            for (int64_t j = tt - 2 < 0 ? 0 : tt - 2; j < tt; ++j) mbar_wait(&a_full[j & 1], (uint32_t)((j >> 1) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer.  Order G1_0(t0), G1_1(t0), then per tile G2_0(t), G1_0(t+1), G2_1(t),
            // G1_1(t+1): the next tile's W1 products run while the epilogue works on this tile's
            // GELU, so the epilogue never waits for them.
            const uint32_t id1 = idesc_bf16(128, 128), id2 = idesc_bf16(128, D);
            int64_t tt = 0, c1 = 0, cg = 0;
            bool ok = mbar_wait_or_abort(w_full, 0, abort);
            tc_fence_after();
            auto g1 = [&](int j, int ab) -> bool {
                const int b = (int)(c1 & 1);
                if (!mbar_wait_or_abort(&acc1_empty[b], (uint32_t)(((c1 >> 1) & 1) ^ 1), abort)) return false;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(b * 128);
#pragma unroll
                for (int kb = 0; kb < 2; ++kb) {
                    const uint32_t a0 = su32(sA + ab * RP::A_BYTES + kb * 16384), w0 = su32(sW1 + j * 16384);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_bf16(d_tmem, sw128_desc(a0 + kk * 32), sw128_desc(w0 + kk * 32), id1, (kb | kk) != 0);
                }
                umma_commit(&acc1_full[b]);
                if (j == NCH - 1) umma_commit(&a_empty[ab]);
                ++c1;
                return true;
            };
            auto g2 = [&](int j, int64_t ttile) -> bool {
                const int ab2 = (int)(ttile & 1);
                if (j == 0 && !mbar_wait_or_abort(&acc2_empty[ab2], (uint32_t)(((ttile >> 1) & 1) ^ 1), abort)) return false;
                if (!mbar_wait_or_abort(g_full, (uint32_t)(cg & 1), abort)) return false;
                tc_fence_after();
                const uint32_t d_tmem = tmem + 256u + (uint32_t)(ab2 * D);
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                    const uint32_t g0 = su32(sG + kb * 16384), w0 = su32(sW2 + (2 * j + (kb & 1)) * 8192);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_bf16(d_tmem, sw128_desc(g0 + kk * 32), sw128_desc(w0 + kk * 32), id2, (j | kb | kk) != 0);
                }
                umma_commit(g_empty);
                if (j == NCH - 1) umma_commit(&acc2_full[ab2]);
                ++cg;
                return true;
            };
            auto a_ready = [&](int64_t ttile) -> bool {
                if (!mbar_wait_or_abort(&a_full[ttile & 1], (uint32_t)((ttile >> 1) & 1), abort)) return false;
                tc_fence_after();
                return true;
            };
            if (ok && (int64_t)blockIdx.x < ntiles) ok = a_ready(0) && g1(0, 0) && g1(1, 0);
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x, ++tt) {
                const bool has_next = t + gridDim.x < ntiles;
                const int abn = (int)((tt + 1) & 1);
                ok = g2(0, tt);
                if (ok && has_next) ok = a_ready(tt + 1) && g1(0, abn);
                ok = ok && g2(1, tt);
                if (ok && has_next) ok = g1(1, abn);
            }
        }
    } else {
        MlpEpiArgs<64> E{tmem, sG, sStg, sb1, sb2, acc1_full, acc1_empty, g_full, g_empty, acc2_full, acc2_empty,
                         abort, &tmH, M, ntiles, hbar, head, sgw};
        mlp_epilogue<64, HEAD>(E, warp, lane);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------- fused QKV projection + attention
// For the compensated d_model-64 transformer with head size 16: per tile of S whole sequences
// (S = min(8, 128 / T), S*T <= 128 rows), the MMA warp computes qkv = [a_hi | a_lo] . W^T with
// Wqkv (192 x 64 bf16) resident in shared memory into one of two TMEM accumulators; AW
// attention warps (one per query-row pair, 4..14) move Q, K, V (+ bias) from TMEM into padded
// shared layouts (each (lane quadrant, part) job taken by a warp of that quadrant), release the
// accumulator, run the grouped causal attention of attention_grp_kernel on them (lanes =
// (sequence, head), warps = query-row pairs) and leave o as hi | lo bf16 in a swizzled staging
// tile that one thread writes with two TMA stores.  qkv never goes through HBM.
constexpr int QA_MAX_WARPS = 14;
constexpr int QA_LH = 20;                       // head stride (16 + 4 floats)
constexpr int QA_LU = 2 * 4 * QA_LH + 4;        // K|V row stride (164 floats: rows land on distinct bank groups)
constexpr int QA_QL = 4 * QA_LH + 4;            // Q row stride (84 floats)
constexpr int QA_TAB_LD = 196;          // gather form: padded table row (floats) in shared memory
constexpr int QA_O_BYTES = 2 * 128 * 128;       // o staging: hi and lo, up to 128 rows x 128 bytes

__device__ __forceinline__ void bar_sync_named(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ float4 lds4(const float* p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(su32(p)));
    return v;
}

// Normalised output row (acc / l) of one (row, head) into the swizzled o staging: hi at
// sO, lo at sO + 16 KB; row r is 128 bytes (64 bf16 = 4 heads x 16) with 16-byte unit u at
// position u ^ (r & 7), the layout of a 128B-swizzle TMA box.
__device__ __forceinline__ void qa_stage_row(const float (&acc)[16], float l, uint8_t* sO, int r, int h) {
    const float inv = 1.f / l;
    uint32_t hp[8], lp[8];
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        const float y0 = acc[j] * inv, y1 = acc[j + 1] * inv;
        const __nv_bfloat162 hh = __floats2bfloat162_rn(y0, y1);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(y0 - hf.x, y1 - hf.y);
        hp[j / 2] = *reinterpret_cast<const uint32_t*>(&hh);
        lp[j / 2] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    const uint32_t base = su32(sO) + (uint32_t)r * 128;
#pragma unroll
    for (int u2 = 0; u2 < 2; ++u2) {
        const uint32_t off = (uint32_t)(((2 * h + u2) ^ (r & 7)) << 4);
        st_shared_v4(base + off, hp[4 * u2], hp[4 * u2 + 1], hp[4 * u2 + 2], hp[4 * u2 + 3]);
        st_shared_v4(base + 16384 + off, lp[4 * u2], lp[4 * u2 + 1], lp[4 * u2 + 2], lp[4 * u2 + 3]);
    }
}

// ---- attention of one (sequence, head) on the mma.sync tensor path (m16n8k16, bf16 in, fp32
// accumulate).  Every product takes the compensated form x y ~ x_hi y_hi + x_hi y_lo + x_lo y_hi
// (hi = bf16(x), lo = bf16(x - hi): ~2^-16 relative, like the block GEMMs).  Fragment layouts
// (PTX ISA, m16n8k16 .bf16; g = lane / 4, c = lane % 4): A regs {(g, 2c..2c+1), (g+8, 2c..),
// (g, 2c+8..), (g+8, 2c+8..)}; B regs {(k 2c..2c+1, n g), (k 2c+8.., n g)}; C {(g, 2c), (g, 2c+1),
// (g+8, 2c), (g+8, 2c+1)}.  MT m-tiles of 16 queries, NT n-tiles of 8 keys (T <= 16 MT, 8 NT).
__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&hh);
    lo = *reinterpret_cast<const uint32_t*>(&ll);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                 "{%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
    mma16816(d, al, bh);     // small terms first
    mma16816(d, ah, bl);
    mma16816(d, ah, bh);
}

__device__ __forceinline__ float2 lds2(const float* p) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(su32(p)));
    return v;
}
__device__ __forceinline__ float lds1(const float* p) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(su32(p)));
    return v;
}

// qs: Q of the unit (row stride QA_QL), kv: K of the unit (row stride QA_LU; V at + 4*QA_LH);
// the normalised output rows go to the o staging rows row0 .. row0 + T - 1, columns of head h.
template <int MT, int NT>
__device__ __forceinline__ void qa_unit_mma(const float* qs, const float* kv, int T, uint8_t* sO, int row0, int h,
                                            int lane) {
    constexpr int KK = (NT + 1) / 2;          // 16-key steps of P . V
    const int g = lane >> 2, c = lane & 3;
    const float scale = 0.25f * 1.4426950408889634f;   // rsqrt(16) log2(e): scores in the log2 domain
    const float* vs = kv + 4 * QA_LH;
    // K^T fragments: key 8 nt + g, dims 2c.. and 2c+8..
    uint32_t kh[NT][2], kl[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int key = min(8 * nt + g, T - 1);
        const float2 x0 = lds2(kv + key * QA_LU + 2 * c), x1 = lds2(kv + key * QA_LU + 2 * c + 8);
        split2(x0.x, x0.y, kh[nt][0], kl[nt][0]);
        split2(x1.x, x1.y, kh[nt][1], kl[nt][1]);
    }
    float S[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
        const int ra = min(16 * mt + g, T - 1), rb = min(16 * mt + g + 8, T - 1);
        const float2 q0 = lds2(qs + ra * QA_QL + 2 * c), q1 = lds2(qs + rb * QA_QL + 2 * c);
        const float2 q2 = lds2(qs + ra * QA_QL + 2 * c + 8), q3 = lds2(qs + rb * QA_QL + 2 * c + 8);
        uint32_t qh[4], ql[4];
        split2(q0.x * scale, q0.y * scale, qh[0], ql[0]);
        split2(q1.x * scale, q1.y * scale, qh[1], ql[1]);
        split2(q2.x * scale, q2.y * scale, qh[2], ql[2]);
        split2(q3.x * scale, q3.y * scale, qh[3], ql[3]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            S[mt][nt][0] = S[mt][nt][1] = S[mt][nt][2] = S[mt][nt][3] = 0.f;
            mma3(S[mt][nt], qh, ql, kh[nt], kl[nt]);
        }
    }
    // causal softmax per query row (quads of four lanes share a row)
    float inv[MT][2];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const int row = 16 * mt + g + 8 * hf;
            float m = -INFINITY;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int key = 8 * nt + 2 * c + e;
                    const float v = key <= row ? S[mt][nt][2 * hf + e] : -INFINITY;
                    S[mt][nt][2 * hf + e] = v;
                    m = fmaxf(m, v);
                }
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
            float l = 0.f;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float p = ex2_approx(S[mt][nt][2 * hf + e] - m);
                    S[mt][nt][2 * hf + e] = p;
                    l += p;
                }
            l += __shfl_xor_sync(0xffffffffu, l, 1);
            l += __shfl_xor_sync(0xffffffffu, l, 2);
            inv[mt][hf] = 1.f / l;
        }
    // O = P . V
    float O[MT][2][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) O[mt][n2][0] = O[mt][n2][1] = O[mt][n2][2] = O[mt][n2][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < KK; ++kk) {
        uint32_t vh[2][2], vl[2][2];
        const int k0 = min(16 * kk + 2 * c, T - 1), k1 = min(16 * kk + 2 * c + 1, T - 1);
        const int k2 = min(16 * kk + 2 * c + 8, T - 1), k3 = min(16 * kk + 2 * c + 9, T - 1);
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) {
            const int dcol = 8 * n2 + g;
            split2(lds1(vs + k0 * QA_LU + dcol), lds1(vs + k1 * QA_LU + dcol), vh[n2][0], vl[n2][0]);
            split2(lds1(vs + k2 * QA_LU + dcol), lds1(vs + k3 * QA_LU + dcol), vh[n2][1], vl[n2][1]);
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            uint32_t ph[4], pl[4];
            split2(S[mt][2 * kk][0], S[mt][2 * kk][1], ph[0], pl[0]);
            split2(S[mt][2 * kk][2], S[mt][2 * kk][3], ph[1], pl[1]);
            if (2 * kk + 1 < NT) {
                split2(S[mt][2 * kk + 1][0], S[mt][2 * kk + 1][1], ph[2], pl[2]);
                split2(S[mt][2 * kk + 1][2], S[mt][2 * kk + 1][3], ph[3], pl[3]);
            } else {
                ph[2] = ph[3] = pl[2] = pl[3] = 0u;
            }
#pragma unroll
            for (int n2 = 0; n2 < 2; ++n2) mma3(O[mt][n2], ph, pl, vh[n2], vl[n2]);
        }
    }
    // normalised rows into the o staging (hi at sO, lo at sO + 16 KB; 128B-swizzled rows)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const int row = 16 * mt + g + 8 * hf;
            if (row >= T) continue;
            const int r = row0 + row;
#pragma unroll
            for (int n2 = 0; n2 < 2; ++n2) {
                const int col = h * 16 + 8 * n2 + 2 * c;             // bf16 column of the 64-wide row
                uint32_t hi, lo;
                split2(O[mt][n2][2 * hf] * inv[mt][hf], O[mt][n2][2 * hf + 1] * inv[mt][hf], hi, lo);
                const uint32_t off = (uint32_t)r * 128 + ((((col >> 3) ^ (r & 7)) << 4) | ((col & 7) << 1));
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(su32(sO) + off), "r"(hi) : "memory");
                asm volatile("st.shared.b32 [%0], %1;" ::"r"(su32(sO) + 16384 + off), "r"(lo) : "memory");
            }
        }
}

// GATHER: the first block, whose q, k and v rows depend on (token, position) only, gathers them
// from a table (without the bias) instead of running the projection.
template <int MT, int NT, bool GATHER>   // MT = 0: CUDA-core row-pair attention (any T <= 64)
__global__ void __launch_bounds__(64 + 32 * QA_MAX_WARPS, 1)
tc_qkv_attn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
                   const __grid_constant__ CUtensorMap tmO, const float* __restrict__ bqkv, int64_t R, int T, int S,
                   int SS, int SQ, int64_t ntiles, const __grid_constant__ TcTokTable tok) {
    constexpr int H = 4, DH = 16;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sW = smem;                              // 192 rows x 64 bf16 (24 KB)
    uint8_t* sA = smem + 24576;                      // hi and lo k-blocks (32 KB)
    uint8_t* sO = sA + 32768;                        // o staging (32 KB)
    float* sKV = reinterpret_cast<float*>(sO + QA_O_BYTES);
    float* sQ = sKV + (size_t)S * SS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sQ + (size_t)S * SQ);
    uint64_t* w_full = bars;
    uint64_t* a_full = bars + 1;
    uint64_t* a_empty = bars + 2;
    uint64_t* acc_full = bars + 3;                   // [2]
    uint64_t* acc_empty = bars + 5;                  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 7);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int AW = (int)(blockDim.x >> 5) - 2;       // attention warps
    const int rows_tile = S * T;
    // gather form: the 3T table rows (q | k | v, QA_TAB_LD floats apart) in place of Wqkv and A
    float* sTab = reinterpret_cast<float*>(sW);
    if constexpr (GATHER) {
        const int n4 = 3 * T * 48;
        for (int i = threadIdx.x; i < n4; i += blockDim.x) {
            const int row = i / 48, c4 = i - row * 48;
            reinterpret_cast<float4*>(sTab + row * QA_TAB_LD)[c4] = __ldg(reinterpret_cast<const float4*>(tok.tab + row * 192) + c4);
        }
    }

    if (threadIdx.x == 0) {
        mbar_init(w_full, 1);
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int i = 0; i < 2; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], AW); }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (!GATHER && warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = GATHER ? 0u : *tmem_slot;

    if (warp == 0) {
        if (!GATHER && lane == 0) {
            // ---- producer: Wqkv once, then each tile's A rows
            mbar_expect_tx(w_full, 24576);
            tma_load_2d(sW, &tmW, w_full, 0, 0);
            int64_t tt = 0;
            for (int64_t t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++tt) {
                if (!mbar_wait_or_abort(a_empty, (uint32_t)((tt & 1) ^ 1), abort)) break;
                mbar_expect_tx(a_full, 32768);
                const int y = (int)(t * rows_tile);
                tma_load_2d(sA, &tmA, a_full, 0, y);
                tma_load_2d(sA + 16384, &tmA, a_full, 64, y);
            }
            mbar_wait(w_full, 0);
            if (tt > 0) mbar_wait(a_full, (uint32_t)((tt - 1) & 1));
        }
    } else if (warp == 1) {
        if (!GATHER && lane == 0) {
            // ---- MMA issuer: qkv = A_hi . W^T + A_lo . W^T into accumulator tt % 2
            const uint32_t id = idesc_bf16(128, 192);
            bool ok = mbar_wait_or_abort(w_full, 0, abort);
            tc_fence_after();
            int64_t tt = 0;
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x, ++tt) {
                const int b = (int)(tt & 1);
                if (!mbar_wait_or_abort(&acc_empty[b], (uint32_t)(((tt >> 1) & 1) ^ 1), abort)) break;
                if (!mbar_wait_or_abort(a_full, (uint32_t)(tt & 1), abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(b * 256);
#pragma unroll
                for (int kb = 0; kb < 2; ++kb) {
                    const uint32_t a0 = su32(sA + kb * 16384), w0 = su32(sW);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_bf16(d_tmem, sw128_desc(a0 + kk * 32), sw128_desc(w0 + kk * 32), id, (kb | kk) != 0);
                }
                umma_commit(a_empty);
                umma_commit(&acc_full[b]);
            }
        }
    } else {
        // ---- attention warps
        const int e = warp - 2, q = warp & 3;
        const int qidx = e >> 2;                                 // this warp's index among its quadrant's warps
        const int qcount = (AW - (q >= 2 ? q - 2 : q + 2) + 3) >> 2;   // warps of this quadrant
        const int r = q * 32 + lane;                             // row of the tile (TMEM lane)
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        const float scale = 0.25f * 1.4426950408889634f;          // rsqrt(16) log2(e)
        const int npairs = (T + 1) / 2;
        const bool g_ok = lane < S * H;
        const int gs = g_ok ? lane / H : 0, gh = lane & (H - 1);
        // gather form: this row's configuration, loaded one tile ahead
        auto row_bits = [&](int64_t tile) -> uint64_t {
            return (GATHER && r < rows_tile && tile < ntiles) ? __ldg(tok.bits + min(tile * S + r / T, R - 1)) : 0ull;
        };
        uint64_t xb_next = row_bits(blockIdx.x);
        int64_t tt = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tt) {
            const int b = (int)(tt & 1);
            const uint64_t xb = xb_next;
            if constexpr (GATHER) xb_next = row_bits(t + gridDim.x);
            // every attention warp reaches the named barriers below, even after a timed-out
            // wait, and all of them leave together when the abort flag is up
            bool got = true;
            if constexpr (!GATHER) {
                got = mbar_wait_or_abort(&acc_full[b], (uint32_t)((tt >> 1) & 1), abort);
                tc_fence_after();
            }
            // stage Q, K, V (+ bias) of this quadrant's 32 rows: parts qidx, qidx + qcount, ...
            if (got) {
                for (int part = qidx; part < 3; part += qcount) {
                    float v[64];
                    if constexpr (GATHER) {
                        if (r < rows_tile) {
                            const int tp = r % T;
                            const int tk = tp == 0 ? 2 : (int)((xb >> tok.order[tp - 1]) & 1ull);
                            const float4* src = reinterpret_cast<const float4*>(sTab + (tk * T + tp) * QA_TAB_LD + part * 64);
#pragma unroll
                            for (int j4 = 0; j4 < 16; ++j4) {
                                const float4 x = src[j4];
                                v[4 * j4] = x.x; v[4 * j4 + 1] = x.y; v[4 * j4 + 2] = x.z; v[4 * j4 + 3] = x.w;
                            }
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < 4; ++p) tmem_ld16_nowait(lane_base + (uint32_t)(b * 256 + part * 64 + 16 * p), v + 16 * p);
                        tmem_wait_ld();
                    }
                    if (r < rows_tile) {
                        const int sq = r / T, tp = r - sq * T;
                        float* dst = part == 0 ? sQ + (size_t)sq * SQ + tp * QA_QL
                                               : sKV + (size_t)sq * SS + tp * QA_LU + (part - 1) * (H * QA_LH);
                        const float* bb = bqkv + part * 64;
#pragma unroll
                        for (int hh = 0; hh < H; ++hh)
#pragma unroll
                            for (int j4 = 0; j4 < 4; ++j4) {
                                const int c = hh * 16 + 4 * j4;
                                *reinterpret_cast<float4*>(dst + hh * QA_LH + 4 * j4) =
                                    make_float4(v[c] + bb[c], v[c + 1] + bb[c + 1], v[c + 2] + bb[c + 2], v[c + 3] + bb[c + 3]);
                            }
                    }
                }
            }
            if constexpr (!GATHER) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0 && got) mbar_arrive(&acc_empty[b]);
            }
            // the previous tile's o stores must have read the staging before it is rewritten
            if (threadIdx.x == 64) bulk_wait_read<0>();
            bar_sync_named(1, 32 * AW);                          // staging complete
            if (*abort) break;
            if constexpr (MT > 0) {
                // tensor-core attention: one (sequence, head) unit per warp at a time
                for (int u = e; u < S * H; u += AW) {
                    const int us = u >> 2, uh = u & 3;
                    qa_unit_mma<MT, NT>(sQ + (size_t)us * SQ + uh * QA_LH, sKV + (size_t)us * SS + uh * QA_LH, T, sO,
                                        us * T, uh, lane);
                }
            } else {
            const float* kvs = sKV + (size_t)gs * SS + gh * QA_LH;
            const float* qs = sQ + (size_t)gs * SQ + gh * QA_LH;
            for (int p = e; p < npairs; p += AW) {
                const int ta = p, tb = T - 1 - p;
                float qa[DH], qb[DH], aa[DH], ab[DH];
#pragma unroll
                for (int j4 = 0; j4 < 4; ++j4) {
                    const float4 x = lds4(qs + ta * QA_QL + 4 * j4), y = lds4(qs + tb * QA_QL + 4 * j4);
                    qa[4 * j4] = x.x * scale; qa[4 * j4 + 1] = x.y * scale; qa[4 * j4 + 2] = x.z * scale; qa[4 * j4 + 3] = x.w * scale;
                    qb[4 * j4] = y.x * scale; qb[4 * j4 + 1] = y.y * scale; qb[4 * j4 + 2] = y.z * scale; qb[4 * j4 + 3] = y.w * scale;
                }
#pragma unroll
                for (int j = 0; j < DH; ++j) { aa[j] = 0.f; ab[j] = 0.f; }
                float ma = -INFINITY, la = 0.f, mb = -INFINITY, lb = 0.f;
                if (tb != ta) {
                    attend_keys<DH, true>(kvs, QA_LU, H * QA_LH, 0, ta + 1, qa, aa, ma, la, qb, ab, mb, lb);
                    if (g_ok) qa_stage_row(aa, la, sO, gs * T + ta, gh);
                    attend_keys<DH, false>(kvs, QA_LU, H * QA_LH, ta + 1, tb + 1, qb, ab, mb, lb, qa, aa, ma, la);
                    if (g_ok) qa_stage_row(ab, lb, sO, gs * T + tb, gh);
                } else {
                    attend_keys<DH, false>(kvs, QA_LU, H * QA_LH, 0, ta + 1, qa, aa, ma, la, qb, ab, mb, lb);
                    if (g_ok) qa_stage_row(aa, la, sO, gs * T + ta, gh);
                }
            }
            }
            fence_proxy_async_smem();
            bar_sync_named(1, 32 * AW);                          // o staged; shared layouts free
            if (threadIdx.x == 64) {
                // rows of sequences past R lie beyond the tensor and are clipped by the TMA
                const int y = (int)(t * rows_tile);
                tma_store_2d(&tmO, sO, 0, y);
                tma_store_2d(&tmO, sO + 16384, 64, y);
                bulk_commit();
            }
        }
        if (threadIdx.x == 64) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (!GATHER && warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
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
    if (epi == TF_EPI_SPLIT && (N % 48 || ((uintptr_t)C & 15))) {
        set_error("split-layout GEMM needs N = 3 D with D % 16 == 0 and a 16-byte aligned output");
        return NQS_ERR_UNSUPPORTED;
    }
    const bool f32_out = epi == TF_EPI_STORE || epi == TF_EPI_RESID;
    const bool tma_epi = BN % (f32_out ? 32 : 64) == 0 && ((uintptr_t)C & 15) == 0 &&
                         (epi != TF_EPI_SPLIT || (N / 3) % 64 == 0);
    const size_t stage_bytes = TC_BM * 128 + (size_t)BN * 128;
    const size_t staging = tma_epi ? 4 * TC_STAGE_BYTES_PER_WARP : 0;
    // fill ~104 KB per CTA with ring stages (at least two) so that two CTAs share an SM
    const int stages = (int)std::max<size_t>(2, std::min<size_t>(6, (104 * 1024 - staging) / stage_bytes));
    const size_t smem = 1024 + (size_t)stages * stage_bytes + staging + (2 * stages + 8) * 8 + 16;
    if (smem > 220 * 1024) { set_error("tensor-core GEMM: shared-memory plan too large"); return NQS_ERR_UNSUPPORTED; }
    CUtensorMap ma, mb, mc;
    NQS_TRY(make_map(&ma, A, M, K, TC_BM));
    NQS_TRY(make_map(&mb, W, N, K, BN));
    if (tma_epi) NQS_TRY(make_map(&mc, C, M, (epi == TF_EPI_GELU2 || epi == TF_EPI_SPLIT) ? 2 * N : N, 32, f32_out));
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
        kernel<<<grid, TC_THREADS, smem, s>>>(ma, mb, mc, mc, bias, C, nullptr, nullptr, M, N, K, BN, tcols, stages,
                                              n_tiles_n, total_tiles, TcTokTable{});
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
        case TF_EPI_SPLIT * 2: return launch(tc_gemm_kernel<TF_EPI_SPLIT, false>);
        case TF_EPI_SPLIT * 2 + 1: return launch(tc_gemm_kernel<TF_EPI_SPLIT, true>);
        default: set_error("bad GEMM epilogue"); return NQS_ERR_INVALID_ARG;
    }
}

// Attention-output GEMM with the next LayerNorm fused into its epilogue (compensated BF16,
// d_model 64): h += A . W^T + bias; a = hi | lo of LayerNorm(h; ln_g, ln_b).
int tc_gemm_bf16_resid_ln(const void* A, const uint16_t* W, const float* bias, float* h, void* a_out,
                          const float* ln_g, const float* ln_b, int64_t M, int N, int K, cudaStream_t s,
                          const TcTokTable* h_old) {
    if (M <= 0) return NQS_OK;
    // d_model 64 (with or without the token-position table) or 128: the tile spans whole rows
    if ((N != 64 && N != 128) || (N == 128 && h_old) || K % 64 || K <= 0 || ((uintptr_t)h & 15) ||
        ((uintptr_t)a_out & 15) || !bias || !ln_g || !ln_b ||
        (h_old && (!h_old->tab || !h_old->bits || h_old->T < 1 || ((uintptr_t)h_old->tab & 15)))) {
        set_error("fused residual + LayerNorm GEMM: bad operand");
        return NQS_ERR_INVALID_ARG;
    }
    const int BN = N, tcols = 2 * N;
    const size_t stage_bytes = TC_BM * 128 + (size_t)BN * 128;
    const size_t staging = 4 * (size_t)TC_STAGE_BYTES_PER_WARP * (N / 64);
    const int stages = (int)std::max<size_t>(2, std::min<size_t>(6, (N == 64 ? 104 * 1024 : 200 * 1024) / stage_bytes -
                                                                     staging / stage_bytes));
    const size_t smem = 1024 + (size_t)stages * stage_bytes + staging + (2 * stages + 8) * 8 + 16;
    if (smem > 220 * 1024) { set_error("fused residual + LayerNorm GEMM: shared-memory plan too large"); return NQS_ERR_UNSUPPORTED; }
    CUtensorMap ma, mb, mc, md;
    NQS_TRY(make_map(&ma, A, M, K, TC_BM));
    NQS_TRY(make_map(&mb, W, N, K, BN));
    NQS_TRY(make_map(&mc, h, M, N, 32, true));
    NQS_TRY(make_map(&md, a_out, M, 2 * N, 32));
    const int64_t total_tiles = (M + TC_BM - 1) / TC_BM;
    const int ctas_per_sm = (int)std::max<int64_t>(1, std::min<int64_t>(512 / tcols, (228 * 1024) / (smem + 1024)));
    const int grid = (int)std::min<int64_t>(total_tiles, (int64_t)num_sms() * ctas_per_sm);
    static int configured_device = -1;
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (configured_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<TF_EPI_RESID_LN, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tc_gemm_kernel<TF_EPI_RESID_LN_TAB, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(tc_gemm_kernel<TF_EPI_RESID_LN128, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_gemm resid_ln)", __FILE__, __LINE__);
        configured_device = dev;
    }
    if (N == 128)
        tc_gemm_kernel<TF_EPI_RESID_LN128, true><<<grid, TC_THREADS, smem, s>>>(ma, mb, mc, md, bias, h, ln_g, ln_b, M, N,
                                                                                 K, BN, tcols, stages, 1, total_tiles,
                                                                                 TcTokTable{});
    else if (h_old)
        tc_gemm_kernel<TF_EPI_RESID_LN_TAB, true><<<grid, TC_THREADS, smem, s>>>(ma, mb, mc, md, bias, h, ln_g, ln_b, M, N,
                                                                                  K, BN, tcols, stages, 1, total_tiles, *h_old);
    else
        tc_gemm_kernel<TF_EPI_RESID_LN, true><<<grid, TC_THREADS, smem, s>>>(ma, mb, mc, md, bias, h, ln_g, ln_b, M, N, K,
                                                                              BN, tcols, stages, 1, total_tiles, TcTokTable{});
    NQS_LAUNCHED();
    return NQS_OK;
}

bool tc_qkv_gather_fits(int T) { return 3 * T * QA_TAB_LD * 4 <= 24576 + 32768; }

// Fused QKV projection + causal attention (compensated BF16, d_model 64, head size 16, T <= 64):
// o (hi | lo bf16 [R*T, 128]) = attention of qkv = A . Wqkv^T + bqkv, A = [a_hi | a_lo] [R*T, 128].
int tc_qkv_attention_bf16(const void* A, const uint16_t* Wd, const float* bqkv, void* o, int64_t R, int T,
                          cudaStream_t s, const TcTokTable* qkv) {
    if (R <= 0) return NQS_OK;
    if (T < 1 || T > 64 || ((uintptr_t)o & 15) || !bqkv ||
        (qkv && (!qkv->tab || !qkv->bits || qkv->T != T || ((uintptr_t)qkv->tab & 15) ||
                 !tc_qkv_gather_fits(T)))) {
        set_error("fused QKV attention: bad operand");
        return NQS_ERR_INVALID_ARG;
    }
    const int S = std::min(8, 128 / T);
    const int SS = grp_seq_stride(T * QA_LU, 4, QA_LH, S);
    const int SQ = grp_seq_stride(T * QA_QL, 4, QA_LH, S);
    // tensor-core attention for T <= 32 (one (sequence, head) unit per warp at a time); longer
    // sequences use the CUDA-core row-pair form (one warp per query-row pair)
    const int mt = T <= 16 ? 1 : (T <= 32 ? 2 : 0);
    const int nt = T <= 16 ? 2 : (T <= 24 ? 3 : 4);
    const int AW = mt ? std::max(4, std::min(QA_MAX_WARPS, (S * 4 + 1) / 2))
                      : std::max(4, std::min(QA_MAX_WARPS, (T + 1) / 2));
    const size_t smem = 1024 + 24576 + 32768 + QA_O_BYTES + (size_t)(S * SS + S * SQ) * 4 + 7 * 8 + 16;
    if (smem > 227 * 1024) { set_error("fused QKV attention: shared-memory plan too large"); return NQS_ERR_UNSUPPORTED; }
    CUtensorMap ma{}, mw{}, mo;
    if (!qkv) {                                       // the gather form reads neither A nor Wqkv
        NQS_TRY(make_map(&ma, A, R * T, 128, 128));
        NQS_TRY(make_map(&mw, Wd, 192, 128, 192));   // first K half of [W | W]: W itself
    }
    NQS_TRY(make_map(&mo, o, R * T, 128, S * T));     // o: hi | lo, boxes of 64 bf16 x (S*T) rows
    const int64_t ntiles = (R + S - 1) / S;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms());
    const TcTokTable tok = qkv ? *qkv : TcTokTable{};
    auto launch = [&](auto kernel, int slot) -> int {
        static int configured_device[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
        int dev = 0;
        NQS_CK(cudaGetDevice(&dev));
        if (configured_device[slot] != dev) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_qkv_attn)", __FILE__, __LINE__);
            configured_device[slot] = dev;
        }
        kernel<<<grid, 64 + 32 * AW, smem, s>>>(ma, mw, mo, bqkv, R, T, S, SS, SQ, ntiles, tok);
        NQS_LAUNCHED();
        return NQS_OK;
    };
    if (qkv) {
        if (mt == 1) return launch(tc_qkv_attn_kernel<1, 2, true>, 4);
        if (mt == 2 && nt == 3) return launch(tc_qkv_attn_kernel<2, 3, true>, 5);
        if (mt == 2) return launch(tc_qkv_attn_kernel<2, 4, true>, 6);
        return launch(tc_qkv_attn_kernel<0, 0, true>, 7);
    }
    if (mt == 1) return launch(tc_qkv_attn_kernel<1, 2, false>, 0);
    if (mt == 2 && nt == 3) return launch(tc_qkv_attn_kernel<2, 3, false>, 1);
    if (mt == 2) return launch(tc_qkv_attn_kernel<2, 4, false>, 2);
    return launch(tc_qkv_attn_kernel<0, 0, false>, 3);
}

// Fused MLP block of the compensated transformer (see tc_mlp_kernel); D = 64 or 128.
int tc_mlp_bf16(const void* A, const uint16_t* W1d, const float* b1, const uint16_t* W2d, const float* b2,
                float* h, int64_t M, int D, cudaStream_t s, const TcMlpHead* hd) {
    if (M <= 0) return NQS_OK;
    if (D != 64 && D != 128) { set_error("fused MLP needs d_model 64 or 128"); return NQS_ERR_UNSUPPORTED; }
    if (hd && D != 64) { set_error("fused MLP head form needs d_model 64"); return NQS_ERR_UNSUPPORTED; }
    if (((uintptr_t)h & 15) || !b1 || !b2) { set_error("fused MLP: bad operand"); return NQS_ERR_INVALID_ARG; }
    CUtensorMap ma, mh;
    NQS_TRY(make_map(&ma, A, M, 2 * D, 128));
    NQS_TRY(make_map(&mh, h, M, D, 32, true));
    const int64_t ntiles = (M + 127) / 128;
    if (D == 64) {
        const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms());
        CUtensorMap m1r, m2;   // the whole W1 (first K half of W1d) as one 256-row box; W2
        NQS_TRY(make_map(&m1r, W1d, 4 * D, 2 * D, 256));
        NQS_TRY(make_map(&m2, W2d, D, 8 * D, D));
        static int configured_res[2] = {-1, -1};
        int dev = 0;
        NQS_CK(cudaGetDevice(&dev));
        const int slot = hd ? 1 : 0;
        if (configured_res[slot] != dev) {
            cudaError_t e = hd ? cudaFuncSetAttribute(tc_mlp_res_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MlpResPlan::SMEM)
                               : cudaFuncSetAttribute(tc_mlp_res_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MlpResPlan::SMEM);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_mlp_res)", __FILE__, __LINE__);
            configured_res[slot] = dev;
        }
        MlpHeadArgs ha{};
        if (hd) {
            ha.lnf_g = hd->lnf_g; ha.lnf_b = hd->lnf_b; ha.head_w = hd->head_w; ha.head_b = hd->head_b;
            ha.n = hd->n; ha.logit = hd->logit; ha.hph = hd->hph;
            tc_mlp_res_kernel<true><<<grid, MlpPlan<64>::THREADS, MlpResPlan::SMEM, s>>>(ma, m1r, m2, mh, b1, b2, M, ntiles, ha);
        } else {
            tc_mlp_res_kernel<false><<<grid, MlpPlan<64>::THREADS, MlpResPlan::SMEM, s>>>(ma, m1r, m2, mh, b1, b2, M, ntiles, ha);
        }
        NQS_LAUNCHED();
        return NQS_OK;
    }
    // d_model 128: one CTA per SM over the 128-row tiles, the weights streamed through the ring
    CUtensorMap m1, m2;
    NQS_TRY(make_map(&m1, W1d, 4 * D, 2 * D, 128));
    NQS_TRY(make_map(&m2, W2d, D, 8 * D, D));
    static int configured_device = -1;
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (configured_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(tc_mlp_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             MlpRingPlan<128>::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_mlp)", __FILE__, __LINE__);
        configured_device = dev;
    }
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms());
    tc_mlp_kernel<128><<<grid, MlpPlan<128>::THREADS, MlpRingPlan<128>::SMEM, s>>>(ma, m1, m2, mh, b1, b2, M, ntiles);
    NQS_LAUNCHED();
    return NQS_OK;
}

int device_status_ptr(int** out) {
    static int* addr[256] = {};
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) { set_error("device ordinal out of range"); return NQS_ERR_UNSUPPORTED; }
    if (!addr[dev]) NQS_CK(cudaGetSymbolAddress((void**)&addr[dev], g_tc_status));
    *out = addr[dev];
    return NQS_OK;
}

// Read and clear the device status of the bounded waits (tensor-core kernels, term-sweep
// staging) (synchronous).
int tc_status_take() {
    int v = 0, z = 0;
    NQS_CK(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)));
    if (v) {
        NQS_CK(cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)));
        set_error(std::string(v == 2 ? "a term-sweep staging copy" : "a tensor-core GEMM wait") +
                  " timed out (status " + std::to_string(v) + ")");
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
