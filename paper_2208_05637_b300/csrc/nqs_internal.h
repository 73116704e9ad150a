// Internal declarations shared by the C-ABI layer and the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include <string>
#include <vector>

#include "../../include/nqs.h"

namespace nqs {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define NQS_CK(call)                                                              \
    do {                                                                          \
        cudaError_t e__ = (call);                                                 \
        if (e__ != cudaSuccess) return ::nqs::cuda_fail(e__, #call, __FILE__, __LINE__); \
    } while (0)

// Check for launch errors right after a <<<>>> launch and count the launch.
#define NQS_LAUNCHED()                                                            \
    do {                                                                          \
        ::nqs::count_launch();                                                    \
        cudaError_t e__ = cudaGetLastError();                                     \
        if (e__ != cudaSuccess) return ::nqs::cuda_fail(e__, "kernel launch", __FILE__, __LINE__); \
    } while (0)

#define NQS_TRY(x)                                                                \
    do {                                                                          \
        int s__ = (x);                                                            \
        if (s__ != NQS_OK) return s__;                                            \
    } while (0)

void count_launch();

// Per-kernel CUDA-event timing (enabled by nqs_profile_enable).
struct ProfScope {
    ProfScope(const char* name, cudaStream_t s, double flops = 0.0, double bytes = 0.0);
    ~ProfScope();
    const char* name;
    cudaStream_t stream;
    double work, bytes;        // algorithmic FLOPs and bytes of the bracketed launch
    cudaEvent_t e0 = nullptr;
};

int num_sms();
bool prof_enabled();   // per-kernel profiling is on (nqs_profile_enable)

// ------------------------------------------------------------------ bit strings
// Configurations and Pauli masks of n <= 64 qubits are one uint64 (bit j = qubit j); of
// 64 < n <= 128 qubits two consecutive uint64 words, qubits 0..63 in the first (U128 below).
// Kernels that serve both widths are templates over the bit-string type.
struct U128 {
    uint64_t lo, hi;
};
__host__ __device__ __forceinline__ U128 operator^(const U128& a, const U128& b) { return U128{a.lo ^ b.lo, a.hi ^ b.hi}; }
__host__ __device__ __forceinline__ U128 operator&(const U128& a, const U128& b) { return U128{a.lo & b.lo, a.hi & b.hi}; }
__host__ __device__ __forceinline__ U128 operator|(const U128& a, const U128& b) { return U128{a.lo | b.lo, a.hi | b.hi}; }
__host__ __device__ __forceinline__ bool operator==(const U128& a, const U128& b) { return a.lo == b.lo && a.hi == b.hi; }
__host__ __device__ __forceinline__ bool operator!=(const U128& a, const U128& b) { return !(a == b); }
__host__ __device__ __forceinline__ bool operator<(const U128& a, const U128& b) {
    return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo;
}
__host__ __device__ __forceinline__ bool operator<=(const U128& a, const U128& b) { return !(b < a); }
// bit q of a configuration
__host__ __device__ __forceinline__ int qbit(uint64_t x, int q) { return (int)((x >> q) & 1ull); }
__host__ __device__ __forceinline__ int qbit(const U128& x, int q) {
    return q < 64 ? (int)((x.lo >> q) & 1ull) : (int)((x.hi >> (q - 64)) & 1ull);
}
// x with bit q set
__host__ __device__ __forceinline__ uint64_t with_bit(uint64_t x, int q) { return x | (1ull << q); }
__host__ __device__ __forceinline__ U128 with_bit(U128 x, int q) {
    if (q < 64) x.lo |= 1ull << q; else x.hi |= 1ull << (q - 64);
    return x;
}
template <class BT> __host__ __device__ __forceinline__ BT bits_zero();
template <> __host__ __device__ __forceinline__ uint64_t bits_zero<uint64_t>() { return 0ull; }
template <> __host__ __device__ __forceinline__ U128 bits_zero<U128>() { return U128{0ull, 0ull}; }
inline int words_of(int n) { return (n + 63) / 64; }

// ------------------------------------------------------------------ Hamiltonian
// group meta word: bits 0-7 n_alpha, 8-15 n_beta, bit 16 "has sigma_2-odd terms"
constexpr uint32_t META_HAS_IMAG = 1u << 16;

struct HamDev {
    int n;
    int words;      // uint64 words per mask (1: n <= 64, 2: n <= 128)
    int64_t K;      // merged terms
    int64_t G;      // groups
    const uint64_t* grp_mask;  // G masks of `words` words each
    const uint32_t* grp_off;   // G+1
    const uint32_t* grp_meta;  // G
    // K + 1 records (the last a zero term).  One word: 16 bytes {z low half, z high half, bits of
    // the fp32 hi and lo of the signed real magnitude of c'} -- one 16-byte load per term.  Two
    // words: 32 bytes {z word 0 (two halves), z word 1 (two halves)}, {c' hi, c' lo, 0, 0}.
    const uint4* term;
    int any_imag;              // some group holds a term with an odd sigma_2 count
    // tabulated groups (real, at most SWEEP_TAB_BITS flipped qubits, one z outside the flips):
    const int32_t* grp_tab;    // G: table index, or -1
    const uint32_t* grp_pos;   // G: the flipped qubits, one byte each
    const uint64_t* grp_zc;    // G masks of `words` words: the z bits outside the flips
    const float2* tab;         // SWEEP_TAB_SIZE (hi, lo) entries per table
};
constexpr int SWEEP_TAB_BITS = 4;                    // flipped qubits of a tabulated group
constexpr int SWEEP_TAB_SIZE = 1 << SWEEP_TAB_BITS;  // entries of its table

}  // namespace nqs

struct nqs_ham_s {
    int n = 0;
    int words = 1;                              // uint64 words per mask
    // masks below hold `words` words each (grp_mask: G masks, term_z: K masks)
    int device = 0;
    int64_t K_in = 0, K = 0, G = 0;
    std::vector<uint64_t> grp_mask;
    std::vector<int64_t> grp_off;
    std::vector<uint32_t> grp_meta;
    std::vector<uint64_t> term_z;
    std::vector<double> term_c_re, term_c_im;   // phase-folded c' (exactly one is nonzero)
    void* d_block = nullptr;                    // one device allocation for all arrays
    nqs::HamDev dev{};
};

namespace nqs {

// Spin masks (0: even qubits, spin up; 1: odd qubits, spin down): word w of the mask of an
// n-qubit register
inline uint64_t spin_mask_word(int n, int spin, int w) {
    uint64_t m = 0;
    for (int j = spin; j < n; j += 2)
        if (j / 64 == w) m |= (1ull << (j % 64));
    return m;
}

// Groups whose flip can keep some sector state inside the (n_up, n_dn) sector: an upper bound
// (at least 1) on the rows the term sweep writes for one sample.
inline int64_t feasible_groups(const nqs_ham_s* h, int n_up, int n_dn) {
    const int n_orb = h->n / 2;
    int64_t cnt = 0;
    for (int64_t g = 0; g < h->G; ++g) {
        const int na = h->grp_meta[g] & 0xff, nb = (h->grp_meta[g] >> 8) & 0xff;
        if ((na & 1) || (nb & 1)) continue;
        if (na / 2 > std::min(n_up, n_orb - n_up)) continue;
        if (nb / 2 > std::min(n_dn, n_orb - n_dn)) continue;
        ++cnt;
    }
    return std::max<int64_t>(cnt, 1);
}

// ------------------------------------------------------------------ model
constexpr int MAX_Q = 128;   // qubits of the row-wise models (the transformer: 64)
constexpr int MADE_MAX_LAYERS = 4;
constexpr int TF_MAX_LAYERS = 8;

// Plain-old-data model description handed to kernels by value.
struct ModelConst {
    int arch, n, n_up, n_dn, hidden, layers, heads, precision, compensated;
    uint8_t order[MAX_Q];   // order[t] = qubit of position t
    uint8_t pos[MAX_Q];     // pos[q] = position of qubit q (the inverse of order)
    uint8_t after[MAX_Q];   // same-spin positions after t
    // parameter tensor offsets (floats) into the flat vector
    // PRODUCT: p
    int64_t p_prob;
    // MADE
    int64_t made_W[MADE_MAX_LAYERS], made_b[MADE_MAX_LAYERS];
    int64_t made_Wout, made_bout, ph_W0, ph_b0, ph_W1, ph_b1;
    // TRANSFORMER
    int64_t tok_emb, pos_emb;
    int64_t ln1_g[TF_MAX_LAYERS], ln1_b[TF_MAX_LAYERS], wqkv[TF_MAX_LAYERS], bqkv[TF_MAX_LAYERS];
    int64_t wo[TF_MAX_LAYERS], bo[TF_MAX_LAYERS], ln2_g[TF_MAX_LAYERS], ln2_b[TF_MAX_LAYERS];
    int64_t w1[TF_MAX_LAYERS], b1[TF_MAX_LAYERS], w2[TF_MAX_LAYERS], b2[TF_MAX_LAYERS];
    int64_t lnf_g, lnf_b, head_w, head_b, phase_w, phase_b;
};

struct ParamInfo {
    std::string name;
    int64_t offset, numel;
};

// A captured sampler (all n steps) for one call shape, replayed on a library-owned stream.
struct SamplerGraph {
    int64_t n_samples = -1, max_unique = -1, trace_stride = 0;
    const void* ws = nullptr;
    const float* trace = nullptr;
    const float* params = nullptr;
    const void* bf16 = nullptr;
    const void* cache = nullptr;
    bool seen = false;              // this shape ran once eagerly; capture on the next call
    bool failed = false;            // capture not possible: stay eager for this shape
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;            // kernel launches inside the graph
    cudaStream_t side = nullptr;
    cudaEvent_t ev = nullptr;
};

}  // namespace nqs

struct nqs_model_s {
    nqs_model_desc desc{};
    nqs::ModelConst mc{};
    std::vector<nqs::ParamInfo> params;
    int64_t n_params = 0;
    const float* d_params = nullptr;
    uint16_t* d_bf16 = nullptr;      // bf16 copies of the transformer GEMM weights (BF16 models)
    nqs::SamplerGraph graph;         // captured sampler of the last call shape
    void* d_scache = nullptr;        // sampler cache of the incremental transformer forward
    size_t scache_bytes = 0;
    int prefix_depth = -1;           // transformer local energy: -1 automatic, 0..3 prefix sharing
    int64_t pass_bytes = 0;          // activations of one prefix-sharing sub-pass (0: CHAIN_PASS_BYTES)
};

namespace nqs {

// ------------------------------------------------------------------ workspace carving
// A bump allocator over the caller's workspace; in measure mode it only counts bytes.
struct Carver {
    char* base;
    size_t used = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T*>(base + off) : nullptr;
    }
};

// ------------------------------------------------------------------ launchers (.cu files)
// term sweep (sweep.cu)
constexpr int SWEEP_GT = 256;   // groups per tile (threads per CTA)
constexpr int SWEEP_SB = 32;    // samples per CTA batch (count and emit passes)
constexpr int SWEEP_STAGE = 2048;   // terms of a tile staged in shared memory by the emit pass
constexpr int SWEEP_SMALL = 16;     // groups with more terms are summed by a whole warp
int64_t sweep_tiles(const HamDev& h);
// Validity words (one uint32 per group and 32-sample batch) the count pass hands to the emit pass.
int64_t sweep_valid_words(const HamDev& h, int64_t B);
int launch_sweep_count(const HamDev& h, int n_up, int n_dn, const uint64_t* bits, int64_t B, int32_t* cnt,
                       uint32_t* valid, cudaStream_t s);
int launch_sweep_emit(const HamDev& h, int n_up, int n_dn, int compensated, const uint64_t* bits, int64_t B,
                      const int64_t* off, const uint32_t* valid, uint64_t* xprime, float4* S, cudaStream_t s);
int launch_unpack_rows(const int64_t* off, int64_t ntiles, int64_t B, const float4* S,
                       int64_t* row_offset, float* s_re, float* s_im, int64_t rows_cap,
                       const int64_t* total, cudaStream_t s);

// scans and reductions (reduce.cu)
// Exclusive scan of n int32 -> int64 out[n+1] (out[n] = total); one CTA.
int launch_scan_i32(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s);
// Exclusive scan of n int64 (n read from device *n_dev if non-null) -> out[n+1]; one CTA.
int launch_scan_i64(const int64_t* in, int64_t n_host_max, const int64_t* n_dev, int64_t* out,
                    cudaStream_t s);
int launch_energy_stats(const float* eloc, const int64_t* counts, int64_t B, double* stats,
                        float* g_abs, float* g_phase, cudaStream_t s);
int launch_energy_sums(const float* eloc, const int64_t* counts, int64_t B, double* sums, float* ga_e,
                       float* gp_e, float* ga_w, cudaStream_t s);
int launch_adam(float* p, const float* g, float* m, float* v, int64_t n, int step, float lr,
                float b1, float b2, float eps, cudaStream_t s);
// dW[o][i] += mask(o,i) * sum_b delta[b*ld_d + o] * act[b*ld_a + i]; db[o] += sum_b delta
// mask_kind: 0 none, 1 MADE input (i < deg(o)), 2 MADE hidden (deg(i) <= deg(o)),
//            3 MADE output (deg(i) < o+1); deg(k) = k % (n-1) + 1
int launch_outer_grad(const float* delta, int64_t ld_d, const float* act, int64_t ld_a,
                      int64_t B, int out_dim, int in_dim, int mask_kind, int n_mask,
                      float* dW, float* db, cudaStream_t s);

// models (made.cu): rowwise models (PRODUCT, MADE)
int launch_logpsi_rows(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                       float* la, float* ph, cudaStream_t s);
int launch_eloc_rows(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                     const float* la_x, const float* ph_x, const int64_t* off, int64_t ntiles,
                     const uint64_t* xprime, const float4* S, float* eloc, cudaStream_t s);
int launch_cond_rows(const ModelConst& mc, const float* P, int k, const uint64_t* bits,
                     const int64_t* U, int64_t cap, float* p_out, uint64_t* thr, float* trace,
                     cudaStream_t s);
int launch_made_backward(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                         const float* g_abs, const float* g_phase, float* acts, int64_t ld,
                         cudaStream_t s);
int64_t made_act_stride(const ModelConst& mc);
int made_grad_reduce(const ModelConst& mc, const float* acts, int64_t ld, int64_t B,
                     float* grad, cudaStream_t s);
int launch_product_backward(const ModelConst& mc, const float* P, const uint64_t* bits,
                            int64_t B, const float* g_abs, float* grad, cudaStream_t s);

// transformer (transformer.cu, tc_gemm.cu)
enum { TF_EPI_STORE = 0, TF_EPI_GELU = 1, TF_EPI_RESID = 2, TF_EPI_ACCUM = 3, TF_EPI_GELU2 = 4,
       TF_EPI_RESID_LN = 5,     // h += acc + bias, then a = LayerNorm(h) as hi|lo bf16 (d = 64)
       TF_EPI_RESID_LN_TAB = 6, // the same with the old h taken from a token-position table
       TF_EPI_SPLIT = 7,        // QKV projection into the split layout (bf16 hi and lo planes; see tc_gemm_bf16)
       TF_EPI_RESID_LN128 = 8   // TF_EPI_RESID_LN for d = 128
};
// First-block rows that depend on the (token, position) pair only: the token of position t is 2
// at t = 0 and bit order[t - 1] of the sequence's configuration after it; row (token, t) of a
// table sits at tab + (token * T + t) * width.
struct TcTokTable {
    const float* tab = nullptr;
    const uint64_t* bits = nullptr;   // one configuration per sequence
    int T = 0;
    uint8_t order[MAX_Q] = {};
};
enum { TF_WQKV = 0, TF_WO = 1, TF_W1 = 2, TF_W2 = 3 };
struct TfBufs {
    int64_t R;            // sequences per pass
    float *h, *a, *qkv, *o, *mid;
    float *logit, *hph;      // per-row head logits and per-sequence h of position n - 2 (fused heads)
    float *tab_h, *tab_qkv;  // first-block tables over (token, position): h [3T][d], q|k|v [3T][3d]
    bool fused_heads;        // the last forward left logit / hph instead of the final h
};
struct TfWeights {
    const float* fp32 = nullptr;
    int64_t fp32_off[TF_MAX_LAYERS][4] = {};
    uint16_t* bf16 = nullptr;                // bf16 working copies (model-owned)
    int64_t bf16_off[TF_MAX_LAYERS][4] = {};
};
struct HeadArgsHost {
    int mode = 0;
    float *la = nullptr, *ph = nullptr;
    const uint64_t* xsample = nullptr;
    const float *la_x = nullptr, *ph_x = nullptr;
    const int64_t* seg = nullptr;
    int64_t seg_stride = 1, nseg = 0, row0 = 0;
    const float4* S = nullptr;
    float2* contrib = nullptr;
    float* p_out = nullptr;
    uint64_t* thr = nullptr;
    float* trace = nullptr;
    int step_pos = -1;        // mode 2: h holds only this position (one row per prefix)
};
// Sampler cache of the incremental transformer forward: per layer l and step j a QKV slab of
// cap rows x 3d floats at kv + ((l * n + j) * cap) * 3d (keys and values of the step-j
// prefixes), and the ancestor table anc[r * n + j] = slot of prefix r's ancestor at step j.
struct TfStepCache {
    float* kv = nullptr;
    int64_t cap = 0;
    const int32_t* anc = nullptr;
    const int64_t* Udev = nullptr;   // device count of live prefixes
    // one-kernel step only: with par set, anc is the previous step's table and the kernel composes
    // this step's slots (anc[par[r]][j] for j < k - 1, par[r] at j = k - 1) and writes them to anc_new
    const int32_t* par = nullptr;
    int32_t* anc_new = nullptr;
    // optional first-block tables over (token, position) (tf_tok_tables with T = n)
    const float* tab_h = nullptr;
    const float* tab_qkv = nullptr;
};
// First-block tables of the d_model-64 bf16 models for positions 0..T-1: h0 [3T][64] and the
// QKV projection of LN1_0(h0) without its bias [3T][192] (rows token * T + t).
int tf_tok_tables(const ModelConst& mc, const float* P, const TfWeights& w, int T, float* tab_h, float* tab_qkv,
                  cudaStream_t s);
int64_t tf_seq_capacity(const ModelConst& mc);
void tf_layout(Carver& c, const ModelConst& mc, int64_t R, TfBufs& b);
int64_t tf_bf16_weight_elems(const ModelConst& mc);
int tf_prepare_weights(const ModelConst& mc, const float* P, TfWeights& w, cudaStream_t s);
// head_logits: whole sequences whose heads follow (modes 0 and 1) may have the last block leave
// per-row head logits instead of the final h (compensated d_model 64)
int tf_forward(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
               int64_t R, int T, TfBufs& b, cudaStream_t s, bool head_logits = false);
int tf_heads(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t R, int T,
             const TfBufs& b, const HeadArgsHost& ha, cudaStream_t s);
int tf_step(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits, int64_t R, int k,
            const TfStepCache& kc, TfBufs& b, cudaStream_t s);
// The whole step in one kernel (d_model 64, four heads, bf16 forms): p, the draw thresholds and
// the trace of position k for the R prefixes, as tf_step followed by the mode-2 heads.
bool tf_step_fused_supported(const ModelConst& mc);
int tf_step_fused(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits, int64_t R,
                  int k, const TfStepCache& kc, float* p_out, uint64_t* thr, float* trace, cudaStream_t s);
int64_t tf_step_cache_bytes(const ModelConst& mc, int64_t cap);
int tf_segment_sum(const int64_t* seg, int64_t seg_stride, int64_t nseg, const float2* contrib,
                   int compensated, float* eloc, cudaStream_t s);
int tf_logpsi(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
              int64_t B, float* la, float* ph, TfBufs& b, cudaStream_t s);
// C[M,N] (epi) = A[M,K] (bf16) . W[N,K]^T (bf16) + bias on the tensor cores (tc_gemm.cu).
// C is fp32 for TF_EPI_STORE / TF_EPI_RESID and bf16 for TF_EPI_GELU.  TF_EPI_SPLIT (N = 3 D, the
// QKV projection) writes each value v as hi = bf16(v) and lo = bf16(v - hi) into a bf16 row of
// 2 N: [Q hi | Q lo | K hi | K lo | V hi | V lo], D columns each -- the same 12 D bytes per row
// as the fp32 [Q | K | V] row, with each of Q, K, V in its own third.
int tc_gemm_bf16(const void* A, const uint16_t* W, const float* bias, void* C, int64_t M, int N,
                 int K, int epi, cudaStream_t s);
// transformer backward (tf_backward.cu)
int64_t tf_bwd_seq_capacity(const ModelConst& mc);
size_t tf_bwd_workspace(const ModelConst& mc, int64_t B);
// phases: 1 recomputes the forward activations into ws, 2 runs the backward from them (same
// bits, B, ws and parameters; B within one recompute pass), 3 both.
int tf_backward(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                const float* g_abs, const float* g_phase, float* grad, void* ws, cudaStream_t s, int phases = 3);
// status of the tensor-core kernels' bounded waits; synchronous, clears the flag
// Head form of the last block's fused MLP (d_model 64): per row the output-head logit of
// LNf(h) and, on rows at position n - 2, h itself for the phase head (the final h is not stored).
struct TcMlpHead {
    const float *lnf_g, *lnf_b, *head_w, *head_b;
    int n;
    float* logit;   // [M]
    float* hph;     // [M / n][64]: h of position n - 2
};
// h += GELU(A . W1d^T + b1) . W2d^T + b2 (compensated bf16 forms), the hidden layer kept on chip;
// with hd, the head form instead.
int tc_mlp_bf16(const void* A, const uint16_t* W1d, const float* b1, const uint16_t* W2d, const float* b2,
                float* h, int64_t M, int D, cudaStream_t s, const TcMlpHead* hd = nullptr);
// h[M, 64] += A . W^T + bias, then a[M, 2*64] = hi|lo of LayerNorm(h; ln_g, ln_b) (compensated
// BF16 transformer, d_model 64): the attention-output GEMM with the next LayerNorm fused in.
int tc_gemm_bf16_resid_ln(const void* A, const uint16_t* W, const float* bias, float* h, void* a_out,
                          const float* ln_g, const float* ln_b, int64_t M, int N, int K, cudaStream_t s,
                          const TcTokTable* h_old = nullptr);
// o = causal attention of (A . Wqkv^T + bqkv) for the compensated d_model-64 transformer with
// head size 16, without writing qkv (R sequences of T <= 64 positions; o hi|lo bf16).
int tc_qkv_attention_bf16(const void* A, const uint16_t* Wd, const float* bqkv, void* o, int64_t R, int T,
                          cudaStream_t s, const TcTokTable* qkv = nullptr);
bool tc_qkv_gather_fits(int T);   // the gather form's table fits its shared memory
int tc_status_take();
// Device address of the status word that bounded device waits set on timeout (read and cleared
// by tc_status_take).
int device_status_ptr(int** out);
// Row-generic pieces of the transformer forward (transformer.cu): C = A . W^T (+ epilogue) of
// block `layer`'s matrix `which`, and the MLP half h += W2 . gelu(W1 . a + b1) + b2.
int tf_gemm(const ModelConst& mc, const TfWeights& w, int which, int layer, const void* A, void* C, int64_t M, int N,
            int K, int epi, const float* bias, cudaStream_t s);
int tf_mlp(const ModelConst& mc, const float* P, const TfWeights& w, int layer, const void* a, void* mid, float* h,
           int64_t M, cudaStream_t s, const TcMlpHead* head = nullptr);
// Attention-output projection with the residual add and LayerNorm 2 in its epilogue (compensated
// BF16, d_model 64 or 128; h_old: the first block's old h from the token-position table, d 64).
int tf_resid_ln(const ModelConst& mc, const float* P, const TfWeights& w, int layer, const void* o, float* h,
                void* a, int64_t M, cudaStream_t s, const TcTokTable* h_old = nullptr);

// Prefix-sharing local energy of the transformer (chains.cu).  Jobs of levels 0 (the samples),
// 1 (one flip) and 2 (two flips) with their per-layer key/value caches, and the leaves (the
// sweep's rows); see chains.cu.
constexpr int64_t CHAIN_MAX_CHUNK = 64;                     // samples per chunk
constexpr int64_t CHAIN_CACHE_BYTES = 24ll << 30;           // key/value caches of one chunk
constexpr int64_t CHAIN_PASS_BYTES = 16ll << 30;            // activations of one pass-B sub-pass (default)
constexpr int CHAIN_MAX_SPLIT = 4096;                       // pass-B sub-passes of one chunk
struct ChainBufs {
    int64_t chunk = 0, rows_cap = 0, jobs_cap = 0, pass_rows = 0;
    unsigned long long *l1 = nullptr, *l2 = nullptr;         // per sample: level-1 flips, level-2 (f1, f2) bits
    int64_t *cnt1 = nullptr, *cnt2 = nullptr, *base1 = nullptr, *base2 = nullptr;
    int32_t* cum2 = nullptr;                                 // per (sample, f1): level-2 jobs before f1
    uint64_t* jbits = nullptr;                               // pass-A jobs
    int32_t *jstart = nullptr, *jpar = nullptr;
    int64_t *jrows = nullptr, *joff = nullptr, *jseg = nullptr;   // jseg: end of the parent's job range
    int32_t *lpar = nullptr, *lstart = nullptr;              // leaves (sweep rows)
    int64_t* lrows = nullptr;
    int32_t* lorder = nullptr;                               // slot -> leaf, leaves with rows grouped by parent
    int64_t *srows = nullptr, *soff = nullptr, *sseg = nullptr;  // per slot: rows, row offset, parent's end
    unsigned long long* hist = nullptr;                      // per parent: leaves (then cursors)
    int64_t* hoff = nullptr;                                 // per parent: first slot; [jobs + 1] = slots
    float* kv = nullptr;                                     // [jobs][layers][n][2d]
    float2* cum = nullptr;                                   // [jobs][n + 1]
    float* logit = nullptr;                                  // [jobs][n]
    float* ph4 = nullptr;                                    // [jobs][4]
    int32_t* rjob = nullptr;                                 // per pass row
    uint8_t* rpos = nullptr;
    uint8_t* rstart = nullptr;                               // per pass row: its job's first own position
    // attention chunks of a pass: per chunk (first row offset, nrows | parent << 32, first tile,
    // end tile); tiles of 16 rows of one job: (row0, rows, job's first row, job start)
    int64_t *ccnt = nullptr, *coff = nullptr, *tcnt = nullptr, *toff = nullptr, *chunks = nullptr;
    int32_t* tiles = nullptr;
    int64_t *split = nullptr, *split_off = nullptr;
    TfBufs tf{};
};
bool chain_supported(const ModelConst& mc);   // head shape and staging fit the prefix-sharing kernels
int64_t chain_jobs_per_sample(const ModelConst& mc, int depth);
int64_t chain_chunk(const ModelConst& mc, int depth);
int64_t chain_pass_rows(const ModelConst& mc, int depth, int64_t chunk, int64_t rows_cap, int64_t pass_bytes);
void chain_layout(Carver& c, const ModelConst& mc, int depth, int64_t chunk, int64_t rows_cap, int64_t pass_bytes,
                  ChainBufs& b);
// Ratio-weighted contributions of the chunk's sweep rows (contrib) and the samples' log psi
// (la_x, ph_x) by prefix sharing at the given depth (0..3).
int chain_local_energy(const ModelConst& mc, const float* P, const TfWeights& w, ChainBufs& b, int depth,
                       const uint64_t* xs, int64_t nb, const int64_t* seg, int64_t seg_stride, const uint64_t* xprime,
                       const float4* S, const int64_t* rows_dev, int64_t rows_max, float* la_x, float* ph_x,
                       float2* contrib, cudaStream_t s);

struct TfCtx {
    const TfWeights* w;
    TfBufs* b;
    bool tok_tables = false;   // b holds this call's first-block tables for T = n (tf_tok_tables)
};

// sampler (sampler.cu)
struct SamplerBufs {
    uint64_t *bitsA, *bitsB;   // cap configurations of `words` uint64 each
    int64_t *cntA, *cntB;
    int64_t* start;      // cap+1
    int64_t* n1;         // cap
    uint64_t* thr;       // cap
    float* p;            // cap
    int64_t* flags0;     // cap
    int64_t* flags1;     // cap
    int64_t* pos0;       // cap+1
    int64_t* pos1;       // cap+1
    int64_t* U;          // device scalars: U[0] current U
    int64_t cap;
    int words = 1;       // uint64 words per configuration
    // incremental transformer forward (all null when the conditionals are recomputed from
    // scratch at every step): QKV slabs, ancestor tables (ping-pong), parent slots
    float* kv = nullptr;
    int32_t *ancA = nullptr, *ancB = nullptr;
    int32_t *par = nullptr, *par2 = nullptr;
};
// Tensor-core GEMMs of the bf16 models' backward (tc_bwd.cu): NT recompute (W [N][K], bias,
// residual), NN input gradients (W [K][N]), TN weight-gradient split-K partials in the layout of
// outer_final_kernel ([z][out][in] then [z][out] column sums when with_bias).
bool tc_bwd_ok(const void* A, int64_t lda, const void* B, int64_t ldb);
int tc_bwd_gemm_nt(const float* A, int64_t lda, const float* W, int64_t ldw, const float* bias, float* C, int64_t ldc,
                   int64_t M, int N, int K, bool resid, cudaStream_t s);
int tc_bwd_gemm_nn(const float* A, int64_t lda, const float* W, int64_t ldw, float* C, int64_t ldc, int64_t M, int N,
                   int K, cudaStream_t s);
int tc_bwd_outer_partial(const float* delta, int64_t ld_d, const float* act, int64_t ld_a, int64_t rows, int out_dim,
                         int in_dim, int64_t nsplit, int64_t per, bool with_bias, float* part, cudaStream_t s);

// Programmatic dependent launch for chains of small kernels on one stream: the kernel may be
// resident before its predecessor finishes and waits in pdl_wait() for the predecessor's
// completion (and memory) before it reads anything the predecessor wrote; pdl_trigger() lets the
// next kernel of the chain launch.  Without the launch attribute both are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

// Unique flipped configurations of a local-energy chunk (dedup.cu): a hash table of up to hcap
// slots, each row's slot, the slots' positions in the unique list, and log psi of the unique rows.
struct DedupBufs {
    uint64_t* table = nullptr;
    int64_t hcap = 0;
    int32_t* id = nullptr;       // per slot: position in the unique list
    unsigned long long* count = nullptr;
    int32_t* slot = nullptr;     // per row
    int32_t* sslot = nullptr;    // per sample of the chunk
    uint64_t* uniq = nullptr;    // per unique row
    float *la_u = nullptr, *ph_u = nullptr;
};
void dedup_layout(Carver& c, int64_t rows_cap, int64_t chunk, DedupBufs& d);
// The distinct values of the rows xp[0, *rows_dev) (rows_dev on the device, at most rows_max) and
// the samples xs[0, nb) into d.uniq (their number into *n_unique; synchronizes s).  max_keys
// bounds the number of distinct values (it sizes the hash table).
int dedup_rows(const uint64_t* xp, const int64_t* rows_dev, int64_t rows_max, const uint64_t* xs, int64_t nb,
               int64_t max_keys, const DedupBufs& d, int64_t* n_unique, cudaStream_t s);
// Per-row contributions <x|P|x'> psi(x')/psi(x) of the chunk, log psi of x' and x from d.la_u / d.ph_u.
int dedup_contrib(const uint64_t* xp, const int64_t* rows_dev, int64_t rows_max, const DedupBufs& d,
                  const uint64_t* xsample, const int64_t* seg, int64_t seg_stride, int64_t nseg, const float4* S,
                  float2* contrib, cudaStream_t s);

// Binds the model-owned cache memory (tf_step_cache_bytes(mc, b.cap) bytes) to b.
void sampler_bind_cache(SamplerBufs& b, const ModelConst& mc, void* mem);
int sampler_layout(Carver& c, int64_t n_samples, int64_t max_unique, SamplerBufs& b, int words = 1);
int run_sampler(const ModelConst& mc, const float* P, int64_t n_samples, int64_t max_unique,
                uint64_t seed, SamplerBufs& b, float* trace, int64_t trace_stride,
                const TfCtx* tf, bool fixed_rows, cudaStream_t s);
int sampler_init(SamplerBufs& b, int64_t n_samples, uint64_t seed, cudaStream_t s);
int sampler_steps(const ModelConst& mc, const float* P, int64_t n_samples, int64_t max_unique,
                  SamplerBufs& b, float* trace, int64_t trace_stride, const TfCtx* tf,
                  bool fixed_rows, cudaStream_t s);
// Parent buffers up to this size run the sampler with fixed-size passes and a CUDA graph.
constexpr int64_t SAMPLER_GRAPH_MAX_CAP = 8192;
// Largest model-owned cache of the incremental transformer sampler; larger buffers recompute
// the prefixes at every step.
constexpr int64_t SAMPLER_CACHE_MAX_BYTES = 2ll << 30;

int launch_copy_samples(const SamplerBufs& b, uint64_t* bits_out, int64_t* counts_out,
                        int64_t n, cudaStream_t s);

}  // namespace nqs
