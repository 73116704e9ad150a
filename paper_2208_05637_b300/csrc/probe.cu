// Throughput probe of the SM pipes the term sweep and the FP32 network run on: 32-bit
// population count (POPC), three-input logic (LOP3), three-input integer add (IADD3) and fp32
// fused multiply-add (FFMA), in instructions per SM per clock.
//
// One CTA of 1024 threads per SM runs a loop whose body is eight independent chains of the
// instruction under test (so issue is not limited by dependent latency); every CTA reads its
// SM's clock counter before and after the loop, and the figure is the CTA's instruction count
// divided by its own elapsed cycles -- a per-clock rate, independent of the clock frequency the
// GPU happens to run at.  The chains feed a store so the compiler keeps them.
#include "nqs_internal.h"

namespace nqs {
namespace {

constexpr int PROBE_THREADS = 1024;
constexpr int PROBE_ITERS = 4096;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_SMEM = 160 * 1024;   // dynamic shared memory that keeps one CTA per SM

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS, 1)
pipe_probe_kernel(uint32_t seed, uint32_t* __restrict__ sink, long long* __restrict__ cycles) {
    uint32_t v[PROBE_CHAINS];
    float f[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) {
        v[c] = seed * (threadIdx.x + 1) + c * 0x9E3779B9u;
        f[c] = (float)(v[c] & 0xffff) * 1e-5f;
    }
    extern __shared__ uint32_t probe_pad[];
    if (threadIdx.x == 0) probe_pad[0] = seed;
    const uint32_t a = seed ^ 0x5bd1e995u, b = seed + 0x1b873593u;
    const float fa = 0.999f, fb = 1e-7f;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) {
            if (KIND == 0) {
                v[c] = __popc(v[c] ^ a);               // one POPC plus one LOP3
            } else if (KIND == 1) {
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v[c]) : "r"(a), "r"(b));
            } else if (KIND == 2) {
                asm volatile("add.u32 %0, %0, %1;" : "+r"(v[c]) : "r"(a));
            } else {
                f[c] = fmaf(f[c], fa, fb);
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) acc ^= v[c] ^ __float_as_uint(f[c]);
    sink[blockIdx.x * PROBE_THREADS + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

int probe_pipes(double* out) {
    const int sms = num_sms();
    uint32_t* sink = nullptr;
    long long* cyc = nullptr;
    NQS_CK(cudaMalloc(&sink, (size_t)sms * PROBE_THREADS * 4));
    if (cudaMalloc(&cyc, (size_t)sms * 8) != cudaSuccess) {
        cudaFree(sink);
        return cuda_fail(cudaErrorMemoryAllocation, "cudaMalloc(probe cycles)", __FILE__, __LINE__);
    }
    std::vector<long long> h(sms);
    int st = NQS_OK;
    cudaError_t ea = cudaSuccess;
    if (ea == cudaSuccess) ea = cudaFuncSetAttribute(pipe_probe_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (ea == cudaSuccess) ea = cudaFuncSetAttribute(pipe_probe_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (ea == cudaSuccess) ea = cudaFuncSetAttribute(pipe_probe_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (ea == cudaSuccess) ea = cudaFuncSetAttribute(pipe_probe_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_SMEM);
    if (ea != cudaSuccess) st = cuda_fail(ea, "pipe probe attributes", __FILE__, __LINE__);
    for (int kind = 0; kind < 4 && st == NQS_OK; ++kind) {
        for (int rep = 0; rep < 2 && st == NQS_OK; ++rep) {   // the first run warms up
            switch (kind) {
                case 0: pipe_probe_kernel<0><<<sms, PROBE_THREADS, PROBE_SMEM>>>(0x1234567u + rep, sink, cyc); break;
                case 1: pipe_probe_kernel<1><<<sms, PROBE_THREADS, PROBE_SMEM>>>(0x1234567u + rep, sink, cyc); break;
                case 2: pipe_probe_kernel<2><<<sms, PROBE_THREADS, PROBE_SMEM>>>(0x1234567u + rep, sink, cyc); break;
                default: pipe_probe_kernel<3><<<sms, PROBE_THREADS, PROBE_SMEM>>>(0x1234567u + rep, sink, cyc); break;
            }
            count_launch();
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, (size_t)sms * 8, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_fail(e, "pipe probe", __FILE__, __LINE__);
        }
        if (st != NQS_OK) break;
        // median over the CTAs of instructions per cycle
        std::sort(h.begin(), h.end());
        const double ops = (double)PROBE_THREADS * PROBE_ITERS * PROBE_CHAINS;
        out[kind] = ops / (double)h[sms / 2];
    }
    cudaFree(sink);
    cudaFree(cyc);
    return st;
}

}  // namespace nqs

extern "C" int nqs_probe_pipes(double* per_sm_per_clock) {
    if (!per_sm_per_clock) { nqs::set_error("per_sm_per_clock is NULL"); return NQS_ERR_INVALID_ARG; }
    return nqs::probe_pipes(per_sm_per_clock);
}
