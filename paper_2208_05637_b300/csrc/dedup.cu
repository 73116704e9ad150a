// Unique flipped configurations of a local-energy chunk.  The connected x' = x ^ m of the
// chunk's samples repeat across samples (every x' lies in the same particle-number sector), so
// log psi is evaluated once per distinct x' and the per-row contributions of Eq. local_energy_auto,
// <x|P|x'> psi(x')/psi(x), gather it back (the cross-sample counterpart of the per-sample
// unique flippings of the tensorized local energy).  Each row of the network forward depends on its own
// configuration only, so the values are those of the row-by-row evaluation bit for bit.
//
// The distinct keys are found with an open-addressing hash table (linear probing, 64-bit
// atomicCAS, load factor at most 1/2, sized for the chunk's rows) and numbered by a warp-
// aggregated atomic counter over the occupied slots.
#include "nqs_internal.h"

namespace nqs {
namespace {

constexpr uint64_t DD_EMPTY = ~0ull;   // not a configuration of any sector with N_up + N_dn < n

__device__ __forceinline__ uint64_t dd_mix(uint64_t z) {   // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void dd_insert_kernel(const uint64_t* __restrict__ xp, int64_t rows_max, const int64_t* __restrict__ rows_dev,
                                 unsigned long long* table, int64_t mask, int32_t* __restrict__ slot) {
    const int64_t rows = rows_dev ? min(*rows_dev, rows_max) : rows_max;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = xp[i];
        int64_t h = (int64_t)(dd_mix(key) & (uint64_t)mask);
        // at most mask + 1 probes: the table is never full
        for (int64_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(table + h, (unsigned long long)DD_EMPTY, (unsigned long long)key);
            if (prev == DD_EMPTY || prev == key) { slot[i] = (int32_t)h; break; }
            h = (h + 1) & mask;
        }
    }
}

// Number the occupied slots (one atomic per warp) and list their keys.  The numbering order
// depends on the schedule; every row's value does not.
__global__ void dd_compact_kernel(const unsigned long long* __restrict__ table, int64_t n, int32_t* __restrict__ id,
                                  uint64_t* __restrict__ uniq, unsigned long long* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
        const int64_t h = base + threadIdx.x;
        const unsigned long long key = h < n ? table[h] : DD_EMPTY;
        const bool occ = key != DD_EMPTY;
        const unsigned m = __ballot_sync(0xffffffffu, occ);
        unsigned long long first = 0;
        if (lane == 0 && m) first = atomicAdd(count, (unsigned long long)__popc(m));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (occ) {
            const int64_t u = (int64_t)first + __popc(m & ((1u << lane) - 1u));
            uniq[u] = key;
            id[h] = (int32_t)u;
        }
    }
}

// Row i of the chunk (sample lo = the segment holding i): S(x, x') times psi(x')/psi(x), with
// log psi of x' and of the sample x from the unique list; the diagonal row x' = x keeps S alone.
__global__ void dd_contrib_kernel(const uint64_t* __restrict__ xp, int64_t rows_max, const int64_t* __restrict__ rows_dev,
                                  const int32_t* __restrict__ slot,
                                  const int32_t* __restrict__ id, const float* __restrict__ la_u,
                                  const float* __restrict__ ph_u, const uint64_t* __restrict__ xsample,
                                  const int32_t* __restrict__ sslot,
                                  const int64_t* __restrict__ seg, int64_t seg_stride, int64_t nseg,
                                  const float4* __restrict__ S, float2* __restrict__ contrib) {
    const int64_t rows = min(*rows_dev, rows_max);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nseg - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (seg[mid * seg_stride] <= i) lo = mid; else hi = mid - 1;
        }
        const float4 s4 = S[i];
        const float sre = s4.x + s4.y, sim = s4.z + s4.w;
        float cr = sre, ci = sim;
        if (xp[i] != xsample[lo]) {
            const int32_t u = id[slot[i]], ux = id[sslot[lo]];
            const float mag = expf(la_u[u] - la_u[ux]);
            float sn, cs;
            sincosf(ph_u[u] - ph_u[ux], &sn, &cs);
            const float rr = mag * cs, ri = mag * sn;
            cr = sre * rr - sim * ri;
            ci = sre * ri + sim * rr;
        }
        contrib[i] = make_float2(cr, ci);
    }
}

inline int dd_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16)); }

}  // namespace

int64_t dedup_table_slots(int64_t rows_cap) {
    int64_t h = 1024;
    while (h < 2 * rows_cap) h <<= 1;
    return h;
}

void dedup_layout(Carver& c, int64_t rows_cap, int64_t chunk, DedupBufs& d) {
    d.hcap = dedup_table_slots(rows_cap + chunk);
    d.sslot = c.take<int32_t>(chunk);
    d.table = c.take<uint64_t>(d.hcap);
    d.id = c.take<int32_t>(d.hcap);
    d.count = c.take<unsigned long long>(1);
    d.slot = c.take<int32_t>(rows_cap);
    d.uniq = c.take<uint64_t>(rows_cap);
    d.la_u = c.take<float>(rows_cap);
    d.ph_u = c.take<float>(rows_cap);
}

int dedup_rows(const uint64_t* xp, const int64_t* rows_dev, int64_t rows_max, const uint64_t* xs, int64_t nb,
               int64_t max_keys, const DedupBufs& d, int64_t* n_unique, cudaStream_t s) {
    *n_unique = 0;
    if (rows_max + nb <= 0) return NQS_OK;
    // at least twice the distinct keys, within the layout's table
    const int64_t hc = dedup_table_slots(std::max<int64_t>(1, std::min(max_keys, rows_max + nb)));
    if (hc > d.hcap || hc > (1ll << 31)) { set_error("x' dedup: table too small"); return NQS_ERR_CAPACITY; }
    ProfScope ps("dedup", s, 0.0, (double)(rows_max + nb) * (8 + 4) + (double)hc * (8 * 2 + 4));
    NQS_CK(cudaMemsetAsync(d.table, 0xff, (size_t)hc * sizeof(uint64_t), s));
    NQS_CK(cudaMemsetAsync(d.count, 0, sizeof(unsigned long long), s));
    unsigned long long* tab = reinterpret_cast<unsigned long long*>(d.table);
    if (rows_max > 0) {   // the row count stays on the device (no host round trip before the table)
        dd_insert_kernel<<<dd_grid(rows_max), 256, 0, s>>>(xp, rows_max, rows_dev, tab, hc - 1, d.slot);
        NQS_LAUNCHED();
    }
    if (nb > 0) {   // the samples themselves: their log psi comes from the same list
        dd_insert_kernel<<<dd_grid(nb), 256, 0, s>>>(xs, nb, nullptr, tab, hc - 1, d.sslot);
        NQS_LAUNCHED();
    }
    dd_compact_kernel<<<dd_grid(hc), 256, 0, s>>>(reinterpret_cast<const unsigned long long*>(d.table), hc, d.id, d.uniq,
                                                  d.count);
    NQS_LAUNCHED();
    unsigned long long nu = 0;
    NQS_CK(cudaMemcpyAsync(&nu, d.count, sizeof(nu), cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    *n_unique = (int64_t)nu;
    return NQS_OK;
}

int dedup_contrib(const uint64_t* xp, const int64_t* rows_dev, int64_t rows_max, const DedupBufs& d,
                  const uint64_t* xsample, const int64_t* seg, int64_t seg_stride, int64_t nseg, const float4* S,
                  float2* contrib, cudaStream_t s) {
    if (rows_max <= 0) return NQS_OK;
    ProfScope ps("dedup_contrib", s, 0.0, (double)rows_max * (8 + 4 + 8 + 8 + 16 + 8));
    dd_contrib_kernel<<<dd_grid(rows_max), 256, 0, s>>>(xp, rows_max, rows_dev, d.slot, d.id, d.la_u, d.ph_u, xsample,
                                                        d.sslot, seg, seg_stride, nseg, S, contrib);
    NQS_LAUNCHED();
    return NQS_OK;
}

}  // namespace nqs
