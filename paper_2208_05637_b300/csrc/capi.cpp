// C ABI of the library: argument validation, handle management, the host term-grouping pass,
// workspace layout and orchestration of the device kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "nqs_internal.h"

namespace nqs {

// ------------------------------------------------------------------ errors and bookkeeping
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    cudaGetLastError();   // clear a non-sticky error so later runtime calls do not report it again
    set_error(std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
              std::to_string(line) + ")");
    return NQS_ERR_CUDA;
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

// ------------------------------------------------------------------ profiling
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
    double work, bytes;
};
struct ProfAcc {
    double ms = 0.0;
    int64_t launches = 0;
    double work = 0.0, bytes = 0.0;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof_pending;
static std::map<std::string, ProfAcc> g_prof_acc;

ProfScope::ProfScope(const char* n, cudaStream_t s, double w, double by) : name(n), stream(s), work(w), bytes(by) {
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&e0) != cudaSuccess) { e0 = nullptr; return; }
    cudaEventRecord(e0, stream);
}

ProfScope::~ProfScope() {
    if (!e0) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
    cudaEventRecord(e1, stream);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.push_back({name, e0, e1, work, bytes});
}

bool prof_enabled() { return g_prof_on; }

static void prof_drain() {
    for (auto& r : g_prof_pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto& acc = g_prof_acc[r.name];
        acc.ms += ms;
        acc.launches += 1;
        acc.work += r.work;
        acc.bytes += r.bytes;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_pending.clear();
}

// ------------------------------------------------------------------ helpers
static int check_device_ptr(const void* p, const char* what) {
    if (!p) {
        set_error(std::string(what) + " is NULL");
        return NQS_ERR_INVALID_ARG;
    }
    return NQS_OK;
}

// Number of configurations with n_up and n_dn electrons in n / 2 orbitals per spin (saturating
// at 2^62): the most distinct x' a local-energy chunk can have.
static int64_t sector_dim(int n, int n_up, int n_dn) {
    auto binom = [](int a, int b) -> double {
        double r = 1.0;
        for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
        return r;
    };
    const double v = binom(n / 2, n_up) * binom(n / 2, n_dn);
    return v >= 4.6e18 ? (int64_t)1 << 62 : (int64_t)(v + 0.5);
}


constexpr int64_t ELOC_CHUNK = 1024;   // samples per local-energy chunk

// The term sweep of nb samples: count pass, row offsets, emit pass (rows sample-major).
static int sweep_chunk(const nqs_ham_s* h, int n_up, int n_dn, int compensated, const uint64_t* bits, int64_t nb,
                       int32_t* cnt, int64_t* off, uint32_t* valid, uint64_t* xprime, float4* S, cudaStream_t s) {
    {
        ProfScope ps("sweep_count", s);
        NQS_TRY(launch_sweep_count(h->dev, n_up, n_dn, bits, nb, cnt, valid, s));
    }
    NQS_TRY(launch_scan_i32(cnt, nb * sweep_tiles(h->dev), off, s));
    ProfScope ps("term_sweep", s);
    return launch_sweep_emit(h->dev, n_up, n_dn, compensated, bits, nb, off, valid, xprime, S, s);
}

struct ElocBufs {
    float *la, *ph;
    int32_t* cnt;
    int64_t* off;
    uint32_t* valid;     // the count pass's validity words
    uint64_t* xprime;
    float4* S;
    float2* contrib;     // transformer: per-row ratio-weighted contributions
    TfBufs tf;
    DedupBufs dd;        // transformer: the chunk's distinct x'
    ChainBufs ch;        // transformer: prefix sharing
    bool dedup;          // x' dedup applies (the all-ones word is then no configuration)
    int chain_depth;     // prefix sharing at this depth (0..3), or -1
    int64_t chunk, ntiles, rows_cap;
};

// Prefix-sharing depth of the transformer local energy (-1: the hash dedup path).  Automatic:
// the dedup when the sector holds fewer configurations than a chunk has connected rows (they
// then repeat a lot), prefix sharing at depth 3 otherwise.
static int chain_depth_for(const nqs_model_s* m, const nqs_ham_s* h) {
    if (m->mc.arch != NQS_ARCH_TRANSFORMER) return -1;
    const bool full = m->mc.n_up + m->mc.n_dn >= m->mc.n;   // the dedup's empty key is then a configuration
    if (!chain_supported(m->mc)) return full ? -2 : -1;     // -2: neither form applies
    if (m->prefix_depth >= 0) return m->prefix_depth;
    if (full) return 3;
    const int64_t rows = ELOC_CHUNK * feasible_groups(h, m->mc.n_up, m->mc.n_dn);
    return sector_dim(m->mc.n, m->mc.n_up, m->mc.n_dn) > rows ? 3 : -1;
}

static void eloc_layout(Carver& c, const nqs_model_s* m, const nqs_ham_s* h, int64_t B,
                        ElocBufs& e) {
    e.chain_depth = chain_depth_for(m, h);
    const int64_t chunk_max = e.chain_depth >= 0 ? chain_chunk(m->mc, e.chain_depth) : ELOC_CHUNK;
    e.chunk = std::max<int64_t>(1, std::min(B, chunk_max));
    e.ntiles = sweep_tiles(h->dev);
    e.rows_cap = e.chunk * feasible_groups(h, m->mc.n_up, m->mc.n_dn);
    e.la = c.take<float>(std::max<int64_t>(B, 1));
    e.ph = c.take<float>(std::max<int64_t>(B, 1));
    e.cnt = c.take<int32_t>(e.chunk * e.ntiles);
    e.off = c.take<int64_t>(e.chunk * e.ntiles + 1);
    e.valid = c.take<uint32_t>(sweep_valid_words(h->dev, e.chunk));
    e.xprime = c.take<uint64_t>(e.rows_cap * h->words);
    e.S = c.take<float4>(e.rows_cap);
    e.contrib = nullptr;
    e.dedup = false;
    if (m->mc.arch == NQS_ARCH_TRANSFORMER) {
        e.contrib = c.take<float2>(e.rows_cap);
        if (e.chain_depth >= 0) {
            chain_layout(c, m->mc, e.chain_depth, e.chunk, e.rows_cap, m->pass_bytes, e.ch);
            return;
        }
        tf_layout(c, m->mc, std::min(std::max<int64_t>(B, e.rows_cap), tf_seq_capacity(m->mc)), e.tf);
        e.dedup = m->mc.n_up + m->mc.n_dn < m->mc.n;
        if (e.dedup) dedup_layout(c, e.rows_cap, e.chunk, e.dd);
    }
}

// Transformer weights for one call: fp32 masters, and the bf16 copies refreshed from them.
static int tf_weights(const nqs_model_s* m, TfWeights& w, cudaStream_t s) {
    w.bf16 = m->d_bf16;
    return tf_prepare_weights(m->mc, m->d_params, w, s);
}

}  // namespace nqs

using namespace nqs;

// ====================================================================== C ABI
extern "C" {

const char* nqs_strerror(int status) {
    switch (status) {
        case NQS_OK: return "ok";
        case NQS_ERR_INVALID_ARG: return "invalid argument";
        case NQS_ERR_NQUBITS: return "unsupported number of qubits";
        case NQS_ERR_CAPACITY: return "output capacity too small";
        case NQS_ERR_WORKSPACE: return "workspace too small";
        case NQS_ERR_CUDA: return "CUDA error";
        case NQS_ERR_TIMEOUT: return "device wait timed out";
        case NQS_ERR_NAN: return "non-finite input";
        case NQS_ERR_ALLOC: return "allocation failed";
        case NQS_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

const char* nqs_last_error(void) { return g_last_error.c_str(); }

int64_t nqs_launch_count(void) { return g_launches.load(); }

int nqs_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return NQS_OK;
}

int nqs_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    g_prof_acc.clear();
    return NQS_OK;
}

int nqs_profile_read(const char* kernel, double* total_ms, int64_t* launches) {
    if (!kernel || !total_ms || !launches) return NQS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    auto it = g_prof_acc.find(kernel);
    *total_ms = it == g_prof_acc.end() ? 0.0 : it->second.ms;
    *launches = it == g_prof_acc.end() ? 0 : it->second.launches;
    return NQS_OK;
}

int nqs_profile_work(const char* kernel, double* flops, double* bytes) {
    if (!kernel || !flops || !bytes) return NQS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    auto it = g_prof_acc.find(kernel);
    *flops = it == g_prof_acc.end() ? 0.0 : it->second.work;
    *bytes = it == g_prof_acc.end() ? 0.0 : it->second.bytes;
    return NQS_OK;
}

// ------------------------------------------------------------------ Hamiltonian
int nqs_ham_create(int n_qubits, int64_t n_terms, const uint64_t* x_mask, const uint64_t* z_mask,
                   const double* coeff, nqs_ham_t* out) {
    if (!out) { set_error("out is NULL"); return NQS_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 128) { set_error("n_qubits must be in 1..128"); return NQS_ERR_NQUBITS; }
    if (n_terms < 1 || !x_mask || !z_mask || !coeff) {
        set_error("need n_terms >= 1 and non-NULL x_mask, z_mask, coeff");
        return NQS_ERR_INVALID_ARG;
    }
    const int W = words_of(n_qubits);
    // masks as 128-bit values (the high word zero for one-word registers)
    auto valid_word = [&](int w) -> uint64_t {
        const int bits = std::min(64, n_qubits - 64 * w);
        return bits >= 64 ? ~0ull : ((1ull << bits) - 1);
    };
    std::vector<U128> xs((size_t)n_terms), zs((size_t)n_terms);
    for (int64_t k = 0; k < n_terms; ++k) {
        const uint64_t x0 = x_mask[k * W], z0 = z_mask[k * W];
        const uint64_t x1 = W > 1 ? x_mask[k * W + 1] : 0, z1 = W > 1 ? z_mask[k * W + 1] : 0;
        if (((x0 | z0) & ~valid_word(0)) || (W > 1 && ((x1 | z1) & ~valid_word(1)))) {
            set_error("term " + std::to_string(k) + " has a mask bit >= n_qubits");
            return NQS_ERR_INVALID_ARG;
        }
        if (!std::isfinite(coeff[k])) {
            set_error("term " + std::to_string(k) + " has a non-finite coefficient");
            return NQS_ERR_NAN;
        }
        xs[k] = U128{x0, x1};
        zs[k] = U128{z0, z1};
    }

    // 1. merge equal (x, z) by fp64 summation in input order (stable sort keeps input order)
    std::vector<int64_t> idx(n_terms);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
        return xs[a] != xs[b] ? xs[a] < xs[b] : zs[a] < zs[b];
    });
    auto* h = new (std::nothrow) nqs_ham_s();
    if (!h) return NQS_ERR_ALLOC;
    h->n = n_qubits;
    h->words = W;
    h->K_in = n_terms;
    const U128 A{spin_mask_word(n_qubits, 0, 0), spin_mask_word(n_qubits, 0, 1)};
    const U128 Bm{spin_mask_word(n_qubits, 1, 0), spin_mask_word(n_qubits, 1, 1)};
    auto popc = [](const U128& v) { return __builtin_popcountll(v.lo) + __builtin_popcountll(v.hi); };
    auto push = [&](std::vector<uint64_t>& dst, const U128& v) {
        dst.push_back(v.lo);
        if (W > 1) dst.push_back(v.hi);
    };
    std::vector<double> c_signed;
    U128 last_x{~0ull, ~0ull};
    for (int64_t i = 0; i < n_terms;) {
        const U128 x = xs[idx[i]], z = zs[idx[i]];
        double acc = 0.0;
        int64_t j = i;
        for (; j < n_terms && xs[idx[j]] == x && zs[idx[j]] == z; ++j) acc += coeff[idx[j]];
        i = j;
        if (acc == 0.0) continue;   // 2. drop exact zeros
        // 3. group by x (the flip pattern)
        if (h->grp_off.empty() || last_x != x) {
            push(h->grp_mask, x);
            last_x = x;
            h->grp_off.push_back((int64_t)c_signed.size());
            const uint32_t na = (uint32_t)popc(x & A), nb = (uint32_t)popc(x & Bm);
            h->grp_meta.push_back(na | (nb << 8));
        }
        // 4. fold (-i)^r, r = popcount(x & z), into the coefficient
        const int r = popc(x & z) & 3;
        double re = 0.0, im = 0.0, sgn = 1.0;
        switch (r) {
            case 0: re = acc; sgn = 1.0; break;
            case 1: im = -acc; sgn = -1.0; break;
            case 2: re = -acc; sgn = -1.0; break;
            default: im = acc; sgn = 1.0; break;
        }
        if (r & 1) h->grp_meta.back() |= META_HAS_IMAG;
        push(h->term_z, z);
        h->term_c_re.push_back(re);
        h->term_c_im.push_back(im);
        c_signed.push_back(sgn * acc);
    }
    h->K = (int64_t)c_signed.size();
    h->grp_off.push_back(h->K);
    h->G = (int64_t)h->grp_meta.size();
    if (h->K == 0) {
        // keep one zero term so the device tables are never empty
        h->grp_mask.assign(W, 0);
        h->grp_off.assign({0, 1});
        h->grp_meta.assign(1, 0);
        h->term_z.assign(W, 0);
        h->term_c_re.assign(1, 0.0);
        h->term_c_im.assign(1, 0.0);
        c_signed.assign(1, 0.0);
        h->K = 1;
        h->G = 1;
    }
    if (h->K > (int64_t)0xffffffffll) { delete h; set_error("too many terms"); return NQS_ERR_UNSUPPORTED; }

    // Tabulated groups (Eq. mtx_element factored): a real group whose flip mask m has at most
    // SWEEP_TAB_BITS bits and whose terms share z outside m has
    //     S_g(x) = (-1)^{popcount(x & zc)} T_g[bits of x at the positions of m],
    //     T_g[b] = sum_k c'_k (-1)^{popcount(b & z_k)}   (b, z_k restricted to m),
    // with zc = z_k & ~m the common part; T_g is summed in fp64 here and stored as fp32 hi + lo.
    std::vector<int32_t> g_tab((size_t)h->G, -1);
    std::vector<uint32_t> g_pos((size_t)h->G, 0u);
    std::vector<uint64_t> g_zc((size_t)h->G * W, 0ull);
    std::vector<float2> tab;
    for (int64_t g = 0; g < h->G && h->K > 0; ++g) {
        const U128 m{h->grp_mask[g * W], W > 1 ? h->grp_mask[g * W + 1] : 0ull};
        const int nb = popc(m);
        if (nb < 1 || nb > SWEEP_TAB_BITS || (h->grp_meta[g] & META_HAS_IMAG)) continue;
        const int64_t k0 = h->grp_off[g], k1 = h->grp_off[g + 1];
        auto zk = [&](int64_t k) { return U128{h->term_z[k * W], W > 1 ? h->term_z[k * W + 1] : 0ull}; };
        const U128 notm{~m.lo, ~m.hi};
        const U128 zc = zk(k0) & notm;
        bool uniform = true;
        for (int64_t k = k0 + 1; k < k1 && uniform; ++k) uniform = (zk(k) & notm) == zc;
        if (!uniform) continue;
        int pos[SWEEP_TAB_BITS];
        int np = 0;
        for (int q = 0; q < 128; ++q)
            if ((q < 64 ? (m.lo >> q) : (m.hi >> (q - 64))) & 1ull) pos[np++] = q;
        uint32_t packed = 0;
        for (int i = 0; i < np; ++i) packed |= (uint32_t)pos[i] << (8 * i);
        g_tab[g] = (int32_t)(tab.size() / SWEEP_TAB_SIZE);
        g_pos[g] = packed;
        g_zc[g * W] = zc.lo;
        if (W > 1) g_zc[g * W + 1] = zc.hi;
        for (int b = 0; b < SWEEP_TAB_SIZE; ++b) {
            U128 xb{0ull, 0ull};
            for (int i = 0; i < np; ++i)
                if ((b >> i) & 1) xb = with_bit(xb, pos[i]);
            double t = 0.0;
            for (int64_t k = k0; k < k1; ++k) t += (popc(xb & zk(k)) & 1) ? -c_signed[k] : c_signed[k];
            const float hi = (float)t;
            tab.push_back(make_float2(hi, (float)(t - (double)hi)));
        }
    }
    if (tab.empty()) tab.assign(SWEEP_TAB_SIZE, make_float2(0.f, 0.f));
    const int64_t ntab = (int64_t)tab.size();

    // device copy: one allocation, arrays 256-byte aligned; the term records carry one zero
    // padding record
    const int rec = W;   // uint4 per term record
    Carver c(nullptr);
    c.take<uint64_t>(h->G * W); c.take<uint32_t>(h->G + 1); c.take<uint32_t>(h->G);
    c.take<uint4>((h->K + 1) * rec);
    c.take<int32_t>(h->G); c.take<uint32_t>(h->G); c.take<uint64_t>(h->G * W); c.take<float2>(ntab);
    cudaGetDevice(&h->device);
    if (cudaMalloc(&h->d_block, c.used) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_error("cudaMalloc of the Hamiltonian tables failed");
        return NQS_ERR_ALLOC;
    }
    Carver d(h->d_block);
    auto* d_mask = d.take<uint64_t>(h->G * W);
    auto* d_off = d.take<uint32_t>(h->G + 1);
    auto* d_meta = d.take<uint32_t>(h->G);
    auto* d_t = d.take<uint4>((h->K + 1) * rec);
    auto* d_gtab = d.take<int32_t>(h->G);
    auto* d_gpos = d.take<uint32_t>(h->G);
    auto* d_gzc = d.take<uint64_t>(h->G * W);
    auto* d_tab = d.take<float2>(ntab);
    std::vector<uint32_t> off32(h->grp_off.begin(), h->grp_off.end());
    std::vector<uint4> tt((size_t)(h->K + 1) * rec, make_uint4(0u, 0u, 0u, 0u));
    for (int64_t k = 0; k < h->K; ++k) {
        const float hi = (float)c_signed[k];
        const float lo = (float)(c_signed[k] - (double)hi);
        uint32_t hb, lb;
        std::memcpy(&hb, &hi, 4);
        std::memcpy(&lb, &lo, 4);
        const uint64_t z0 = h->term_z[k * W];
        if (W == 1) {
            tt[k] = make_uint4((uint32_t)z0, (uint32_t)(z0 >> 32), hb, lb);
        } else {
            const uint64_t z1 = h->term_z[k * W + 1];
            tt[2 * k] = make_uint4((uint32_t)z0, (uint32_t)(z0 >> 32), (uint32_t)z1, (uint32_t)(z1 >> 32));
            tt[2 * k + 1] = make_uint4(hb, lb, 0u, 0u);
        }
    }
    int any_imag = 0;
    for (uint32_t mt : h->grp_meta) any_imag |= (mt & META_HAS_IMAG) ? 1 : 0;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(d_mask, h->grp_mask.data(), h->G * W * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_off, off32.data(), (h->G + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_meta, h->grp_meta.data(), h->G * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_t, tt.data(), tt.size() * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_gtab, g_tab.data(), h->G * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_gpos, g_pos.data(), h->G * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_gzc, g_zc.data(), h->G * W * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_tab, tab.data(), ntab * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(h->d_block);
        delete h;
        return cuda_fail(e, "copy of the Hamiltonian tables", __FILE__, __LINE__);
    }
    h->dev = HamDev{h->n, W, h->K, h->G, d_mask, d_off, d_meta, d_t, any_imag, d_gtab, d_gpos, d_gzc, d_tab};
    *out = h;
    return NQS_OK;
}

int nqs_ham_info(nqs_ham_t ham, int64_t* n_terms_merged, int64_t* n_groups) {
    if (!ham) return NQS_ERR_INVALID_ARG;
    if (n_terms_merged) *n_terms_merged = ham->K;
    if (n_groups) *n_groups = ham->G;
    return NQS_OK;
}

int nqs_ham_export(nqs_ham_t h, uint64_t* grp_mask, int64_t* grp_offset, uint64_t* term_z,
                   double* term_c_re, double* term_c_im) {
    if (!h) return NQS_ERR_INVALID_ARG;
    if (grp_mask) std::memcpy(grp_mask, h->grp_mask.data(), h->G * h->words * 8);
    if (grp_offset) std::memcpy(grp_offset, h->grp_off.data(), (h->G + 1) * 8);
    if (term_z) std::memcpy(term_z, h->term_z.data(), h->K * h->words * 8);
    if (term_c_re) std::memcpy(term_c_re, h->term_c_re.data(), h->K * 8);
    if (term_c_im) std::memcpy(term_c_im, h->term_c_im.data(), h->K * 8);
    return NQS_OK;
}

void nqs_ham_destroy(nqs_ham_t h) {
    if (!h) return;
    if (h->d_block) cudaFree(h->d_block);
    delete h;
}

// ------------------------------------------------------------------ model
static void add_param(nqs_model_s* m, const std::string& name, int64_t numel, int64_t* slot) {
    if (slot) *slot = m->n_params;
    m->params.push_back({name, m->n_params, numel});
    m->n_params += numel;
}

int nqs_model_create(const nqs_model_desc* d, nqs_model_t* out) {
    if (!d || !out) { set_error("desc/out is NULL"); return NQS_ERR_INVALID_ARG; }
    *out = nullptr;
    const int n = d->n_qubits;
    if (n < 4 || n > MAX_Q || (n & 1)) { set_error("n_qubits must be even and in 4..128"); return NQS_ERR_NQUBITS; }
    if (n > 64 && d->arch == NQS_ARCH_TRANSFORMER) {
        set_error("the transformer supports n_qubits <= 64 (two-word registers: product and MADE models)");
        return NQS_ERR_NQUBITS;
    }
    const int n_orb = n / 2;
    if (d->n_up < 0 || d->n_dn < 0 || d->n_up > n_orb || d->n_dn > n_orb) {
        set_error("n_up/n_dn outside 0..n_qubits/2");
        return NQS_ERR_INVALID_ARG;
    }
    if (d->precision != NQS_PREC_FP32 && d->precision != NQS_PREC_BF16) {
        set_error("precision must be NQS_PREC_FP32 or NQS_PREC_BF16");
        return NQS_ERR_INVALID_ARG;
    }
    std::vector<char> seen((size_t)n, 0);
    for (int t = 0; t < n; ++t) {
        int q = d->order[t];
        if (q < 0 || q >= n || seen[q]) { set_error("order is not a permutation"); return NQS_ERR_INVALID_ARG; }
        seen[q] = 1;
    }
    auto* m = new (std::nothrow) nqs_model_s();
    if (!m) return NQS_ERR_ALLOC;
    m->desc = *d;
    ModelConst& mc = m->mc;
    mc.arch = d->arch; mc.n = n; mc.n_up = d->n_up; mc.n_dn = d->n_dn;
    mc.hidden = d->hidden; mc.layers = d->layers; mc.heads = d->heads;
    mc.precision = d->precision; mc.compensated = d->compensated;
    for (int t = 0; t < n; ++t) {
        mc.order[t] = (uint8_t)d->order[t];
        mc.pos[d->order[t]] = (uint8_t)t;
        int cnt = 0;
        for (int u = t + 1; u < n; ++u) cnt += ((d->order[u] & 1) == (d->order[t] & 1));
        mc.after[t] = (uint8_t)cnt;
    }
    const int h = d->hidden;
    if (d->arch == NQS_ARCH_PRODUCT) {
        if (d->precision != NQS_PREC_FP32) { delete m; set_error("product model is fp32 only"); return NQS_ERR_UNSUPPORTED; }
        add_param(m, "p", n, &mc.p_prob);
    } else if (d->arch == NQS_ARCH_MADE) {
        if (h < 1 || h > 64 || d->layers < 1 || d->layers > MADE_MAX_LAYERS) {
            delete m;
            set_error("MADE needs 1 <= hidden <= 64 and 1 <= layers <= 4");
            return NQS_ERR_UNSUPPORTED;
        }
        if (d->precision != NQS_PREC_FP32) { delete m; set_error("MADE runs in fp32"); return NQS_ERR_UNSUPPORTED; }
        add_param(m, "made.W0", (int64_t)h * n, &mc.made_W[0]);
        add_param(m, "made.b0", h, &mc.made_b[0]);
        for (int l = 1; l < d->layers; ++l) {
            add_param(m, "made.W" + std::to_string(l), (int64_t)h * h, &mc.made_W[l]);
            add_param(m, "made.b" + std::to_string(l), h, &mc.made_b[l]);
        }
        add_param(m, "made.Wout", (int64_t)n * h, &mc.made_Wout);
        add_param(m, "made.bout", n, &mc.made_bout);
        add_param(m, "phase.W0", (int64_t)h * (n - 2), &mc.ph_W0);
        add_param(m, "phase.b0", h, &mc.ph_b0);
        add_param(m, "phase.W1", 4 * (int64_t)h, &mc.ph_W1);
        add_param(m, "phase.b1", 4, &mc.ph_b1);
    } else if (d->arch == NQS_ARCH_TRANSFORMER) {
        if (d->heads < 1 || h % d->heads || d->layers < 1 || d->layers > TF_MAX_LAYERS || h > 256) {
            delete m;
            set_error("transformer needs heads | hidden, 1 <= layers <= 8, hidden <= 256");
            return NQS_ERR_UNSUPPORTED;
        }
        const int dh = h / d->heads;
        if (dh != 16 && dh != 32) { delete m; set_error("transformer head size must be 16 or 32"); return NQS_ERR_UNSUPPORTED; }
        if (d->heads > 8) { delete m; set_error("transformer supports at most 8 heads"); return NQS_ERR_UNSUPPORTED; }
        if ((size_t)n * (4 * h + 5) * 4 > 200 * 1024) {
            delete m;
            set_error("transformer attention block (n x 4*d_model floats) exceeds shared memory");
            return NQS_ERR_UNSUPPORTED;
        }
        add_param(m, "tok_emb", 3 * (int64_t)h, &mc.tok_emb);
        add_param(m, "pos_emb", (int64_t)n * h, &mc.pos_emb);
        for (int l = 0; l < d->layers; ++l) {
            std::string p = "blk" + std::to_string(l) + ".";
            add_param(m, p + "ln1_g", h, &mc.ln1_g[l]);
            add_param(m, p + "ln1_b", h, &mc.ln1_b[l]);
            add_param(m, p + "wqkv", 3 * (int64_t)h * h, &mc.wqkv[l]);
            add_param(m, p + "bqkv", 3 * (int64_t)h, &mc.bqkv[l]);
            add_param(m, p + "wo", (int64_t)h * h, &mc.wo[l]);
            add_param(m, p + "bo", h, &mc.bo[l]);
            add_param(m, p + "ln2_g", h, &mc.ln2_g[l]);
            add_param(m, p + "ln2_b", h, &mc.ln2_b[l]);
            add_param(m, p + "w1", 4 * (int64_t)h * h, &mc.w1[l]);
            add_param(m, p + "b1", 4 * (int64_t)h, &mc.b1[l]);
            add_param(m, p + "w2", 4 * (int64_t)h * h, &mc.w2[l]);
            add_param(m, p + "b2", h, &mc.b2[l]);
        }
        add_param(m, "lnf_g", h, &mc.lnf_g);
        add_param(m, "lnf_b", h, &mc.lnf_b);
        add_param(m, "head_w", h, &mc.head_w);
        add_param(m, "head_b", n, &mc.head_b);
        add_param(m, "phase_w", 4 * (int64_t)h, &mc.phase_w);
        add_param(m, "phase_b", 4, &mc.phase_b);
    } else {
        delete m;
        set_error("unknown arch");
        return NQS_ERR_INVALID_ARG;
    }
    *out = m;
    return NQS_OK;
}

int nqs_model_param_count(nqs_model_t m, int64_t* n) {
    if (!m || !n) return NQS_ERR_INVALID_ARG;
    *n = m->n_params;
    return NQS_OK;
}

int nqs_model_param_tensors(nqs_model_t m, int* n) {
    if (!m || !n) return NQS_ERR_INVALID_ARG;
    *n = (int)m->params.size();
    return NQS_OK;
}

int nqs_model_param_info(nqs_model_t m, int index, const char** name, int64_t* offset,
                         int64_t* numel) {
    if (!m || index < 0 || index >= (int)m->params.size()) return NQS_ERR_INVALID_ARG;
    if (name) *name = m->params[index].name.c_str();
    if (offset) *offset = m->params[index].offset;
    if (numel) *numel = m->params[index].numel;
    return NQS_OK;
}

int nqs_model_bind_params(nqs_model_t m, const float* p) {
    if (!m || !p) { set_error("model/params is NULL"); return NQS_ERR_INVALID_ARG; }
    if (((uintptr_t)p) & 15) { set_error("parameter vector must be 16-byte aligned"); return NQS_ERR_INVALID_ARG; }
    m->d_params = p;
    if (m->mc.arch == NQS_ARCH_TRANSFORMER && m->mc.precision == NQS_PREC_BF16 && !m->d_bf16) {
        const size_t bytes = (size_t)tf_bf16_weight_elems(m->mc) * 2;
        if (cudaMalloc((void**)&m->d_bf16, bytes) != cudaSuccess) {
            cudaGetLastError();
            m->d_bf16 = nullptr;
            set_error("cudaMalloc of the bf16 weight copies failed");
            return NQS_ERR_ALLOC;
        }
    }
    return NQS_OK;
}

static void graph_release(SamplerGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
}

int nqs_model_set_prefix_reuse(nqs_model_t m, int depth) {
    if (!m || depth < -1 || depth > 3) { set_error("need a model and depth in -1..3"); return NQS_ERR_INVALID_ARG; }
    if (m->mc.arch != NQS_ARCH_TRANSFORMER) { set_error("prefix reuse applies to the transformer"); return NQS_ERR_UNSUPPORTED; }
    if (depth >= 0 && !chain_supported(m->mc)) {
        set_error("prefix reuse needs head size 16 or 32, 1/2/4/8 heads and d_model <= 128 (d_model 256: head size 32 "
                  "with at most 4 heads)");
        return NQS_ERR_UNSUPPORTED;
    }
    m->prefix_depth = depth;
    return NQS_OK;
}

int nqs_model_set_pass_bytes(nqs_model_t m, int64_t bytes) {
    if (!m || bytes < 0) { set_error("need a model and bytes >= 0"); return NQS_ERR_INVALID_ARG; }
    if (m->mc.arch != NQS_ARCH_TRANSFORMER) { set_error("sub-pass size applies to the transformer"); return NQS_ERR_UNSUPPORTED; }
    m->pass_bytes = bytes;
    return NQS_OK;
}

void nqs_model_destroy(nqs_model_t m) {
    if (!m) return;
    graph_release(m->graph);
    if (m->graph.ev) cudaEventDestroy(m->graph.ev);
    if (m->graph.side) cudaStreamDestroy(m->graph.side);
    if (m->d_bf16) cudaFree(m->d_bf16);
    if (m->d_scache) cudaFree(m->d_scache);
    delete m;
}

int nqs_workspace_size(nqs_model_t m, nqs_ham_t h, int op, int64_t batch, size_t* bytes) {
    if (!m || !bytes || batch < 0) return NQS_ERR_INVALID_ARG;
    Carver c(nullptr);
    switch (op) {
        case NQS_OP_SAMPLE: {
            SamplerBufs b;
            NQS_TRY(sampler_layout(c, std::max<int64_t>(batch, 1), std::max<int64_t>(batch, 1), b, words_of(m->mc.n)));
            if (m->mc.arch == NQS_ARCH_TRANSFORMER) {
                TfBufs tb;
                tf_layout(c, m->mc, std::min(b.cap, tf_seq_capacity(m->mc)), tb);
            }
            break;
        }
        case NQS_OP_LOGPSI:
            c.take<char>(256);
            if (m->mc.arch == NQS_ARCH_TRANSFORMER) {
                TfBufs tb;
                tf_layout(c, m->mc, std::max<int64_t>(1, std::min(batch, tf_seq_capacity(m->mc))), tb);
            }
            break;
        case NQS_OP_LOCAL_ENERGY: {
            if (!h) return NQS_ERR_INVALID_ARG;
            ElocBufs e;
            eloc_layout(c, m, h, batch, e);
            break;
        }
        case NQS_OP_TERM_SWEEP: {
            if (!h) return NQS_ERR_INVALID_ARG;
            int64_t T = sweep_tiles(h->dev);
            c.take<int32_t>(std::max<int64_t>(batch, 1) * T);
            c.take<int64_t>(std::max<int64_t>(batch, 1) * T + 1);
            c.take<uint32_t>(sweep_valid_words(h->dev, std::max<int64_t>(batch, 1)));
            c.take<float4>(std::max<int64_t>(batch, 1) * feasible_groups(h, m->mc.n_up, m->mc.n_dn));
            break;
        }
        case NQS_OP_BACKWARD:
            if (m->mc.arch == NQS_ARCH_MADE) c.take<float>(std::max<int64_t>(batch, 1) * made_act_stride(m->mc));
            else if (m->mc.arch == NQS_ARCH_TRANSFORMER) c.take<char>(tf_bwd_workspace(m->mc, std::max<int64_t>(batch, 1)));
            else c.take<char>(256);
            break;
        default:
            return NQS_ERR_INVALID_ARG;
    }
    *bytes = c.used + 256;
    return NQS_OK;
}

static int need_ws(nqs_model_t m, nqs_ham_t h, int op, int64_t batch, void* ws, size_t ws_bytes) {
    size_t need = 0;
    NQS_TRY(nqs_workspace_size(m, h, op, batch, &need));
    if (!ws || ws_bytes < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return NQS_ERR_WORKSPACE;
    }
    if (((uintptr_t)ws) & 255) { set_error("workspace must be 256-byte aligned"); return NQS_ERR_INVALID_ARG; }
    return NQS_OK;
}

static int need_params(nqs_model_t m) {
    if (!m) return NQS_ERR_INVALID_ARG;
    if (!m->d_params) { set_error("no parameters bound"); return NQS_ERR_INVALID_ARG; }
    return NQS_OK;
}

// ------------------------------------------------------------------ hot path
int nqs_sample(nqs_model_t m, int64_t n_samples, int64_t max_unique, uint64_t seed,
               uint64_t* bits_out, int64_t* counts_out, int64_t capacity, int64_t* n_unique,
               float* p_trace, int64_t trace_stride, void* ws, size_t ws_bytes, void* stream) {
    NQS_TRY(need_params(m));
    if (n_samples < 1 || n_samples >= (1ll << 31) || max_unique < 1 || !n_unique || capacity < 0) {
        set_error("need 1 <= n_samples < 2^31, max_unique >= 1, n_unique non-NULL");
        return NQS_ERR_INVALID_ARG;
    }
    NQS_TRY(need_ws(m, nullptr, NQS_OP_SAMPLE, n_samples, ws, ws_bytes));
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    SamplerBufs b;
    NQS_TRY(sampler_layout(c, n_samples, max_unique, b, words_of(m->mc.n)));
    if (p_trace && trace_stride < b.cap) {
        set_error("trace_stride must be >= min(n_samples, 2*max_unique)");
        return NQS_ERR_INVALID_ARG;
    }
    TfWeights w;
    TfBufs tb{};
    TfCtx ctx{&w, &tb};
    if (m->mc.arch == NQS_ARCH_TRANSFORMER) {
        tf_layout(c, m->mc, std::min(b.cap, tf_seq_capacity(m->mc)), tb);
        NQS_TRY(tf_weights(m, w, s));
        // incremental forward when its cache (the keys and values of every step for every
        // buffer slot, model-owned) stays within SAMPLER_CACHE_MAX_BYTES and the pass buffers
        // hold one position of every slot
        const int64_t need = tf_step_cache_bytes(m->mc, b.cap);
        if (need <= SAMPLER_CACHE_MAX_BYTES && b.cap <= tb.R * m->mc.n) {
            if (m->scache_bytes < (size_t)need) {
                if (m->d_scache) NQS_CK(cudaFree(m->d_scache));
                m->d_scache = nullptr;
                m->scache_bytes = 0;
                void* p = nullptr;
                const cudaError_t e = cudaMalloc(&p, (size_t)need);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    set_error("sampler cache allocation failed");
                    return NQS_ERR_ALLOC;
                }
                m->d_scache = p;
                m->scache_bytes = (size_t)need;
            }
            sampler_bind_cache(b, m->mc, m->d_scache);
            // the one-kernel step takes block 0 from the (token, position) tables of this call
            if (tf_step_fused_supported(m->mc)) {
                NQS_TRY(tf_tok_tables(m->mc, m->d_params, w, m->mc.n, tb.tab_h, tb.tab_qkv, s));
                ctx.tok_tables = true;
            }
        }
    }
    int64_t U = 0;
    // captured and replayed as a graph: one-word buffers within the one-CTA bookkeeping's size
    const bool graphable = b.cap <= SAMPLER_GRAPH_MAX_CAP && b.words == 1;
    SamplerGraph& G = m->graph;
    const bool same = G.n_samples == n_samples && G.max_unique == max_unique && G.ws == ws &&
                      G.trace == p_trace && G.trace_stride == trace_stride && G.params == m->d_params &&
                      G.bf16 == (const void*)m->d_bf16 && G.cache == (const void*)b.kv;
    if (graphable && same && !G.failed && (G.exec || G.seen)) {
        // replay (capturing first if this shape has run once eagerly): the steps run on the
        // library's stream, ordered after the caller's stream by an event
        if (!G.side) NQS_CK(cudaStreamCreateWithFlags(&G.side, cudaStreamNonBlocking));
        if (!G.ev) NQS_CK(cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming));
        NQS_CK(cudaEventRecord(G.ev, s));
        NQS_CK(cudaStreamWaitEvent(G.side, G.ev, 0));
        if (!G.exec) {
            cudaGraph_t graph = nullptr;
            const int64_t before = g_launches.load();
            NQS_CK(cudaStreamBeginCapture(G.side, cudaStreamCaptureModeRelaxed));
            const int st = sampler_steps(m->mc, m->d_params, n_samples, max_unique, b, p_trace, trace_stride,
                                         &ctx, true, G.side);
            G.kernels = g_launches.load() - before;   // kernel nodes of the graph (counted at capture)
            g_launches.fetch_sub(G.kernels);          // counted again at every replay instead
            const cudaError_t ce = cudaStreamEndCapture(G.side, &graph);
            cudaError_t ie = cudaErrorUnknown;
            if (st == NQS_OK && ce == cudaSuccess && graph) ie = cudaGraphInstantiate(&G.exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                cudaGetLastError();
                G.exec = nullptr;
                G.failed = true;
            }
        }
        if (G.exec) {
            ProfScope ps("sample", G.side);
            NQS_TRY(sampler_init(b, n_samples, seed, G.side));
            NQS_CK(cudaGraphLaunch(G.exec, G.side));
            g_launches.fetch_add(G.kernels, std::memory_order_relaxed);
        } else {
            NQS_TRY(run_sampler(m->mc, m->d_params, n_samples, max_unique, seed, b, p_trace, trace_stride,
                                &ctx, true, G.side));
        }
        NQS_CK(cudaMemcpyAsync(&U, b.U, sizeof(int64_t), cudaMemcpyDeviceToHost, G.side));
        NQS_CK(cudaStreamSynchronize(G.side));
    } else {
        if (graphable && !same) {
            graph_release(G);
            G.n_samples = n_samples; G.max_unique = max_unique; G.ws = ws; G.trace = p_trace;
            G.trace_stride = trace_stride; G.params = m->d_params; G.bf16 = m->d_bf16; G.cache = b.kv;
            G.failed = false;
        }
        G.seen = graphable;
        NQS_TRY(run_sampler(m->mc, m->d_params, n_samples, max_unique, seed, b, p_trace, trace_stride,
                            &ctx, graphable, s));
        NQS_CK(cudaMemcpyAsync(&U, b.U, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        NQS_CK(cudaStreamSynchronize(s));
    }
    if (m->mc.precision == NQS_PREC_BF16) NQS_TRY(tc_status_take());
    *n_unique = U;
    if (U > capacity) {
        set_error("sample capacity " + std::to_string(capacity) + " < unique count " + std::to_string(U));
        return NQS_ERR_CAPACITY;
    }
    if (U > 0) {
        NQS_TRY(check_device_ptr(bits_out, "bits_out"));
        NQS_TRY(check_device_ptr(counts_out, "counts_out"));
        NQS_TRY(launch_copy_samples(b, bits_out, counts_out, U, s));
    }
    return NQS_OK;
}

int nqs_logpsi(nqs_model_t m, const uint64_t* bits, int64_t B, float* la, float* ph, void* ws,
               size_t ws_bytes, void* stream) {
    NQS_TRY(need_params(m));
    if (B < 0) return NQS_ERR_INVALID_ARG;
    if (B == 0) return NQS_OK;
    if (!bits || !la || !ph) { set_error("bits/log_abs/phase is NULL"); return NQS_ERR_INVALID_ARG; }
    if (m->mc.arch == NQS_ARCH_TRANSFORMER) {
        NQS_TRY(need_ws(m, nullptr, NQS_OP_LOGPSI, B, ws, ws_bytes));
        cudaStream_t s = (cudaStream_t)stream;
        Carver c(ws);
        c.take<char>(256);
        TfBufs tb;
        tf_layout(c, m->mc, std::max<int64_t>(1, std::min(B, tf_seq_capacity(m->mc))), tb);
        TfWeights w;
        NQS_TRY(tf_weights(m, w, s));
        NQS_TRY(tf_logpsi(m->mc, m->d_params, w, bits, B, la, ph, tb, s));
        if (m->mc.precision == NQS_PREC_BF16) {   // bounded-wait status of the tensor-core GEMMs
            NQS_CK(cudaStreamSynchronize(s));
            return tc_status_take();
        }
        return NQS_OK;
    }
    (void)ws; (void)ws_bytes;
    return launch_logpsi_rows(m->mc, m->d_params, bits, B, la, ph, (cudaStream_t)stream);
}

int nqs_term_sweep(nqs_ham_t h, int n_up, int n_dn, int compensated, const uint64_t* bits,
                   int64_t B, int64_t* row_offset, uint64_t* xprime, float* s_re, float* s_im,
                   int64_t capacity, int64_t* n_rows, void* ws, size_t ws_bytes, void* stream) {
    if (!h || !n_rows || B < 0 || capacity < 0) return NQS_ERR_INVALID_ARG;
    int n_orb = h->n / 2;
    if ((h->n & 1) || n_up < 0 || n_dn < 0 || n_up > n_orb || n_dn > n_orb) {
        set_error("sector outside the Hamiltonian's qubits");
        return NQS_ERR_INVALID_ARG;
    }
    if (B == 0) { *n_rows = 0; return NQS_OK; }
    if (!bits || !row_offset) { set_error("bits/row_offset is NULL"); return NQS_ERR_INVALID_ARG; }
    // workspace check against a throwaway model-free layout
    int64_t T = sweep_tiles(h->dev);
    Carver need(nullptr);
    need.take<int32_t>(B * T); need.take<int64_t>(B * T + 1);
    need.take<uint32_t>(sweep_valid_words(h->dev, B));
    need.take<float4>(B * feasible_groups(h, n_up, n_dn));
    if (!ws || ws_bytes < need.used) { set_error("workspace too small"); return NQS_ERR_WORKSPACE; }
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    int32_t* cnt = c.take<int32_t>(B * T);
    int64_t* off = c.take<int64_t>(B * T + 1);
    uint32_t* valid = c.take<uint32_t>(sweep_valid_words(h->dev, B));
    float4* S = c.take<float4>(B * feasible_groups(h, n_up, n_dn));
    {
        ProfScope ps("sweep_count", s);
        NQS_TRY(launch_sweep_count(h->dev, n_up, n_dn, bits, B, cnt, valid, s));
    }
    NQS_TRY(launch_scan_i32(cnt, B * T, off, s));
    int64_t total = 0;
    NQS_CK(cudaMemcpyAsync(&total, off + B * T, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    *n_rows = total;
    if (total > capacity) { set_error("row capacity too small"); return NQS_ERR_CAPACITY; }
    if (total > 0 && (!xprime || !s_re || !s_im)) { set_error("xprime/s_re/s_im is NULL"); return NQS_ERR_INVALID_ARG; }
    {
        ProfScope ps("term_sweep", s);
        NQS_TRY(launch_sweep_emit(h->dev, n_up, n_dn, compensated, bits, B, off, valid, xprime, S, s));
    }
    NQS_TRY(launch_unpack_rows(off, T, B, S, row_offset, s_re, s_im, capacity, off + B * T, s));
    NQS_CK(cudaStreamSynchronize(s));
    return tc_status_take();
}

int nqs_local_energy(nqs_ham_t h, nqs_model_t m, const uint64_t* bits, int64_t B, float* eloc,
                     void* ws, size_t ws_bytes, void* stream) {
    NQS_TRY(need_params(m));
    if (!h || B < 0) return NQS_ERR_INVALID_ARG;
    if (h->n != m->mc.n) { set_error("Hamiltonian and model qubit counts differ"); return NQS_ERR_INVALID_ARG; }
    if (B == 0) return NQS_OK;
    if (!bits || !eloc) { set_error("bits/eloc is NULL"); return NQS_ERR_INVALID_ARG; }
    NQS_TRY(need_ws(m, h, NQS_OP_LOCAL_ENERGY, B, ws, ws_bytes));
    cudaStream_t s = (cudaStream_t)stream;
    Carver c(ws);
    ElocBufs e;
    eloc_layout(c, m, h, B, e);
    if (e.chain_depth == -2) {
        set_error("transformer local energy: a completely filled sector needs the prefix-sharing form, which this "
                  "head shape does not support");
        return NQS_ERR_UNSUPPORTED;
    }
    if (m->mc.arch == NQS_ARCH_TRANSFORMER && e.chain_depth >= 0) {
        // prefix sharing: the samples' log psi come from level 0 of each chunk's jobs
        ProfScope ps_all("local_energy", s);
        TfWeights w;
        NQS_TRY(tf_weights(m, w, s));
        for (int64_t lo = 0; lo < B; lo += e.chunk) {
            const int64_t nb = std::min(e.chunk, B - lo);
            NQS_TRY(sweep_chunk(h, m->mc.n_up, m->mc.n_dn, m->mc.compensated, bits + lo, nb, e.cnt, e.off, e.valid,
                                    e.xprime, e.S, s));
            const int64_t rows_max = nb * (e.rows_cap / e.chunk);
            NQS_TRY(chain_local_energy(m->mc, m->d_params, w, e.ch, e.chain_depth, bits + lo, nb, e.off, e.ntiles,
                                       e.xprime, e.S, e.off + nb * e.ntiles, rows_max, e.la + lo, e.ph + lo,
                                       e.contrib, s));
            NQS_TRY(tc_status_take());
            NQS_TRY(tf_segment_sum(e.off, e.ntiles, nb, e.contrib, m->mc.compensated, eloc + 2 * lo, s));
        }
        return NQS_OK;
    }
    if (m->mc.arch == NQS_ARCH_TRANSFORMER) {
        ProfScope ps_all("local_energy", s);
        TfWeights w;
        NQS_TRY(tf_weights(m, w, s));
        // the samples' log psi come from the chunk's unique list
        for (int64_t lo = 0; lo < B; lo += e.chunk) {
            const int64_t nb = std::min(e.chunk, B - lo);
            NQS_TRY(sweep_chunk(h, m->mc.n_up, m->mc.n_dn, m->mc.compensated, bits + lo, nb, e.cnt, e.off, e.valid,
                                    e.xprime, e.S, s));
            {
                // log psi once per distinct x' of the chunk, then the rows' contributions; the row
                // count stays on the device (bounded by the chunk's feasible groups)
                const int64_t* rows_dev = e.off + nb * e.ntiles;
                const int64_t rows_max = nb * (e.rows_cap / e.chunk);
                // the table holds the distinct keys: at most the rows plus samples, and at most
                // the sector's configurations
                const int64_t keys = std::min(rows_max + nb, sector_dim(m->mc.n, m->mc.n_up, m->mc.n_dn));
                int64_t nu = 0;
                NQS_TRY(dedup_rows(e.xprime, rows_dev, rows_max, bits + lo, nb, keys, e.dd, &nu, s));
                NQS_TRY(tc_status_take());     // bounded waits of the sweep (and the GEMMs so far)
                for (int64_t r0 = 0; r0 < nu; r0 += e.tf.R) {
                    const int64_t R = std::min(e.tf.R, nu - r0);
                    NQS_TRY(tf_forward(m->mc, m->d_params, w, e.dd.uniq + r0, R, m->mc.n, e.tf, s, true));
                    HeadArgsHost ha{};
                    ha.mode = 0; ha.la = e.dd.la_u + r0; ha.ph = e.dd.ph_u + r0;
                    NQS_TRY(tf_heads(m->mc, m->d_params, e.dd.uniq + r0, R, m->mc.n, e.tf, ha, s));
                }
                NQS_TRY(dedup_contrib(e.xprime, rows_dev, rows_max, e.dd, bits + lo, e.off, e.ntiles, nb, e.S, e.contrib,
                                      s));
                NQS_TRY(tf_segment_sum(e.off, e.ntiles, nb, e.contrib, m->mc.compensated, eloc + 2 * lo, s));
            }
        }
        return NQS_OK;
    }
    const int64_t W = h->words;   // uint64 words per configuration
    NQS_TRY(launch_logpsi_rows(m->mc, m->d_params, bits, B, e.la, e.ph, s));
    for (int64_t lo = 0; lo < B; lo += e.chunk) {
        const int64_t nb = std::min(e.chunk, B - lo);
        NQS_TRY(sweep_chunk(h, m->mc.n_up, m->mc.n_dn, m->mc.compensated, bits + lo * W, nb, e.cnt, e.off, e.valid,
                                e.xprime, e.S, s));
        {
            // algorithmic work for the profile (read back only while profiling): per connected row
            // other than the sample itself, the dense MACs of the row's forward (MADE: input and
            // hidden layers, output logits, phase MLP) -- 2 FLOP each; compulsory bytes: the
            // row's x' and S
            double flops = 0.0, bytes = 0.0;
            if (prof_enabled()) {
                int64_t rows = 0;
                NQS_CK(cudaMemcpyAsync(&rows, e.off + nb * e.ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                NQS_CK(cudaStreamSynchronize(s));
                const double n = m->mc.n, hid = m->mc.hidden, L = m->mc.layers;
                const double macs = m->mc.arch == NQS_ARCH_MADE
                                        ? n * hid + (L - 1) * hid * hid + n * hid + (n - 2) * hid + 4 * hid
                                        : n;
                flops = 2.0 * macs * (double)std::max<int64_t>(0, rows - nb);
                bytes = (double)rows * (8.0 * W + 16.0);
            }
            ProfScope ps("eloc_rows", s, flops, bytes);
            NQS_TRY(launch_eloc_rows(m->mc, m->d_params, bits + lo * W, nb, e.la + lo, e.ph + lo, e.off,
                                     e.ntiles, e.xprime, e.S, eloc + 2 * lo, s));
        }
    }
    return NQS_OK;
}

int nqs_logpsi_backward(nqs_model_t m, const uint64_t* bits, int64_t B, const float* g_abs,
                        const float* g_phase, float* grad, void* ws, size_t ws_bytes,
                        void* stream) {
    NQS_TRY(need_params(m));
    if (B < 0) return NQS_ERR_INVALID_ARG;
    if (B == 0) return NQS_OK;
    if (!bits || !g_abs || !g_phase || !grad) { set_error("null pointer argument"); return NQS_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (m->mc.arch == NQS_ARCH_PRODUCT)
        return launch_product_backward(m->mc, m->d_params, bits, B, g_abs, grad, s);
    NQS_TRY(need_ws(m, nullptr, NQS_OP_BACKWARD, B, ws, ws_bytes));
    if (m->mc.arch == NQS_ARCH_TRANSFORMER) {
        ProfScope ps("tf_backward", s);
        Carver c(ws);
        void* base = c.take<char>(tf_bwd_workspace(m->mc, B));
        return tf_backward(m->mc, m->d_params, bits, B, g_abs, g_phase, grad, base, s);
    }
    Carver c(ws);
    const int64_t ld = made_act_stride(m->mc);
    float* acts = c.take<float>(B * ld);
    {
        ProfScope ps("made_backward", s);
        NQS_TRY(launch_made_backward(m->mc, m->d_params, bits, B, g_abs, g_phase, acts, ld, s));
    }
    {
        ProfScope ps("grad_reduce", s);
        NQS_TRY(made_grad_reduce(m->mc, acts, ld, B, grad, s));
    }
    return NQS_OK;
}

int nqs_logpsi_backward_phase(nqs_model_t m, int phase, const uint64_t* bits, int64_t B, const float* g_abs,
                              const float* g_phase, float* grad, void* ws, size_t ws_bytes, void* stream) {
    NQS_TRY(need_params(m));
    if (B < 0 || (phase != 1 && phase != 2)) { set_error("need B >= 0 and phase 1 or 2"); return NQS_ERR_INVALID_ARG; }
    if (B == 0) return NQS_OK;
    if (!bits || (phase == 2 && (!g_abs || !g_phase || !grad))) { set_error("null pointer argument"); return NQS_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (m->mc.arch != NQS_ARCH_TRANSFORMER) {
        // nothing to recompute ahead: phase 2 is the whole backward
        return phase == 1 ? NQS_OK : nqs_logpsi_backward(m, bits, B, g_abs, g_phase, grad, ws, ws_bytes, stream);
    }
    NQS_TRY(need_ws(m, nullptr, NQS_OP_BACKWARD, B, ws, ws_bytes));
    ProfScope ps(phase == 1 ? "tf_backward_recompute" : "tf_backward", s);
    Carver c(ws);
    void* base = c.take<char>(tf_bwd_workspace(m->mc, B));
    return tf_backward(m->mc, m->d_params, bits, B, g_abs, g_phase, grad, base, s, phase);
}

int nqs_energy_stats(const float* eloc, const int64_t* counts, int64_t B, double* stats,
                     float* g_abs, float* g_phase, void* stream) {
    if (B < 1 || !eloc || !counts || !stats) { set_error("need B >= 1 and eloc/counts/stats"); return NQS_ERR_INVALID_ARG; }
    if ((g_abs == nullptr) != (g_phase == nullptr)) { set_error("g_abs and g_phase go together"); return NQS_ERR_INVALID_ARG; }
    return launch_energy_stats(eloc, counts, B, stats, g_abs, g_phase, (cudaStream_t)stream);
}

int nqs_energy_sums(const float* eloc, const int64_t* counts, int64_t B, double* sums, float* g_abs_e,
                    float* g_phase_e, float* g_abs_w, void* stream) {
    if (B < 1 || !eloc || !counts || !sums) { set_error("need B >= 1 and eloc/counts/sums"); return NQS_ERR_INVALID_ARG; }
    if (!((g_abs_e && g_phase_e && g_abs_w) || (!g_abs_e && !g_phase_e && !g_abs_w))) {
        set_error("g_abs_e, g_phase_e and g_abs_w go together");
        return NQS_ERR_INVALID_ARG;
    }
    return launch_energy_sums(eloc, counts, B, sums, g_abs_e, g_phase_e, g_abs_w, (cudaStream_t)stream);
}

int nqs_adam_step(float* p, const float* g, float* mm, float* v, int64_t n, int step, float lr,
                  float b1, float b2, float eps, void* stream) {
    if (!p || !g || !mm || !v || n < 0 || step < 1) { set_error("bad Adam arguments"); return NQS_ERR_INVALID_ARG; }
    if (n == 0) return NQS_OK;
    return launch_adam(p, g, mm, v, n, step, lr, b1, b2, eps, (cudaStream_t)stream);
}

}  // extern "C"
