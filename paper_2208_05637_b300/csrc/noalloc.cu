// nqs_local_energy_noalloc: the local-energy call without any allocation.
//
// Some callers cannot allocate device memory at the point where they need a local energy:
// code running under an allocator that forbids cudaMalloc/cudaFree while it is active (for
// example inside a memory pool's or a framework's restricted region), plugins that are handed
// only the input and output buffers, and embedded runtimes that reserve all device memory up
// front.  For them this entry point keeps its scratch (per-sample log psi, the sweep's counts
// and row offsets, the x' stream and its coefficient sums) in one file-scope device array of
// NQS_NOALLOC_SCRATCH_BYTES, allocated when the library's module is loaded and held by every
// GPU that loads the library until the process exits.  It calls no cudaMalloc, cudaFree or
// allocating library routine.
//
// Set-up: the first call on each device looks up the array's device address with
// cudaGetSymbolAddress while that device is current and caches it.  When CUDA loads modules
// lazily (the default since CUDA 12.2), that lookup is also what loads this file's module and
// so allocates the array: make the first call on each device outside any no-allocation region
// and before any stream capture.  All calls share the one array and it keeps whatever the previous call
// left in it: every word a call reads is written earlier in the same call, so nothing needs
// clearing, but two calls whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and must be serialised by the caller.
#include <mutex>

#include "nqs_internal.h"

namespace nqs {
namespace {

constexpr size_t kScratchBytes = (size_t)NQS_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal out of range for the static scratch table");
        return NQS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)", __FILE__, __LINE__);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return NQS_OK;
}

struct Plan {
    float *la, *ph;
    int32_t* cnt;
    int64_t* off;
    uint32_t* valid;
    uint64_t* xprime;
    float4* S;
    int64_t chunk, ntiles;
};

// Carve the scratch for B samples processed `chunk` at a time; returns the bytes used.
size_t carve(Carver& c, const HamDev& h, int64_t B, int64_t chunk, int64_t ntiles, int64_t feas, Plan& p) {
    p.chunk = chunk;
    p.ntiles = ntiles;
    p.la = c.take<float>(B);
    p.ph = c.take<float>(B);
    p.cnt = c.take<int32_t>(chunk * ntiles);
    p.off = c.take<int64_t>(chunk * ntiles + 1);
    p.valid = c.take<uint32_t>(sweep_valid_words(h, chunk));
    p.xprime = c.take<uint64_t>(chunk * feas);
    p.S = c.take<float4>(chunk * feas);
    return c.used;
}

}  // namespace
}  // namespace nqs

using namespace nqs;

extern "C" int nqs_local_energy_noalloc(nqs_ham_t h, nqs_model_t m, const uint64_t* bits,
                                        int64_t B, float* eloc, void* stream) {
    if (!h || !m || B < 0) { set_error("ham/model is NULL or B < 0"); return NQS_ERR_INVALID_ARG; }
    if (!m->d_params) { set_error("no parameters bound"); return NQS_ERR_INVALID_ARG; }
    if (h->n != m->mc.n) { set_error("Hamiltonian and model qubit counts differ"); return NQS_ERR_INVALID_ARG; }
    if (m->mc.arch != NQS_ARCH_PRODUCT && m->mc.arch != NQS_ARCH_MADE) {
        set_error("nqs_local_energy_noalloc serves the product and MADE models");
        return NQS_ERR_UNSUPPORTED;
    }
    if (h->words != 1) { set_error("nqs_local_energy_noalloc supports n_qubits <= 64"); return NQS_ERR_NQUBITS; }
    if (B == 0) return NQS_OK;
    if (!bits || !eloc) { set_error("bits/eloc is NULL"); return NQS_ERR_INVALID_ARG; }

    const int64_t ntiles = sweep_tiles(h->dev);
    const int64_t feas = feasible_groups(h, m->mc.n_up, m->mc.n_dn);
    // largest chunk (<= 1024 samples) whose buffers fit next to the per-sample log psi
    Plan plan{};
    int64_t chunk = std::min<int64_t>(B, 1024);
    for (;; chunk = chunk / 2) {
        Carver probe(nullptr);
        if (carve(probe, h->dev, B, chunk, ntiles, feas, plan) <= kScratchBytes) break;
        if (chunk == 1) {
            set_error("nqs_local_energy_noalloc: " + std::to_string(B) + " samples with up to " +
                      std::to_string(feas) + " connected rows each need more than the " +
                      std::to_string(kScratchBytes >> 20) + " MiB static scratch; use "
                      "nqs_local_energy with a caller-allocated workspace or a smaller B");
            return NQS_ERR_CAPACITY;
        }
    }
    void* base = nullptr;
    NQS_TRY(scratch_address(&base));
    Carver c(base);
    carve(c, h->dev, B, chunk, ntiles, feas, plan);

    cudaStream_t s = (cudaStream_t)stream;
    NQS_TRY(launch_logpsi_rows(m->mc, m->d_params, bits, B, plan.la, plan.ph, s));
    for (int64_t lo = 0; lo < B; lo += plan.chunk) {
        const int64_t nb = std::min(plan.chunk, B - lo);
        NQS_TRY(launch_sweep_count(h->dev, m->mc.n_up, m->mc.n_dn, bits + lo, nb, plan.cnt, plan.valid, s));
        NQS_TRY(launch_scan_i32(plan.cnt, nb * ntiles, plan.off, s));
        NQS_TRY(launch_sweep_emit(h->dev, m->mc.n_up, m->mc.n_dn, m->mc.compensated, bits + lo,
                                  nb, plan.off, plan.valid, plan.xprime, plan.S, s));
        NQS_TRY(launch_eloc_rows(m->mc, m->d_params, bits + lo, nb, plan.la + lo, plan.ph + lo,
                                 plan.off, ntiles, plan.xprime, plan.S, eloc + 2 * lo, s));
    }
    return NQS_OK;
}
