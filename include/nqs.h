/*
 * nqs.h -- C ABI of the B300 (sm_103a) library for the local-energy hot path of autoregressive
 * neural quantum states over Jordan-Wigner qubit Hamiltonians (Zhao, Stokes, Veerapaneni,
 * "Scalable neural quantum states architecture for quantum chemistry", arXiv 2208.05637).
 *
 * Conventions shared by every call
 *  - A configuration (bitstring) or Pauli mask of n_qubits <= 64 is one uint64, qubit j in bit j;
 *    of 64 < n_qubits <= 128 it is W = 2 consecutive uint64 words, qubit j in bit j % 64 of word
 *    j / 64 (the paper reaches 76 qubits, Table 1).  Arrays of B configurations hold B * W words.
 *    Two-word registers are served by every call with the PRODUCT and MADE models (nqs_sample
 *    then runs its steps as separate launches instead of a captured graph); the transformer and
 *    nqs_local_energy_noalloc take n_qubits <= 64 (NQS_ERR_NQUBITS otherwise).  Spin orbital
 *    j = 2p + s: even qubits are spin up (alpha), odd qubits spin down
 *    (beta) (Eq. hamming_weight_constraint).
 *  - A Pauli string is a pair of masks (x_mask, z_mask): qubit j carries I for (0,0), sigma_1
 *    for (1,0), sigma_3 for (0,1) and sigma_2 for (1,1) (Section 3, Eq. hamiltonpauli).
 *  - Pointers documented as "device" must point to memory of the current CUDA device; "host"
 *    pointers to ordinary host memory.  Bulk device buffers (bits, counts, outputs, gradients,
 *    parameters, workspace) are owned by the caller and must stay alive until the work queued
 *    on the stream has completed.  Handles are owned by the library; *_destroy frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *    are asynchronous on it unless stated otherwise.
 *  - Every call returns NQS_OK (0) or a negative status; no exception or abort crosses the
 *    ABI.  nqs_last_error() gives a message for the calling thread's last failure.
 */
#ifndef NQS_H
#define NQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define NQS_OK               0
#define NQS_ERR_INVALID_ARG (-1)  /* a null pointer, negative size, bad enum, bad mask bit    */
#define NQS_ERR_NQUBITS     (-2)  /* n_qubits outside the supported range                   */
#define NQS_ERR_CAPACITY    (-3)  /* an output buffer is too small; the needed size is set  */
#define NQS_ERR_WORKSPACE   (-4)  /* ws_bytes smaller than nqs_workspace_size() reported      */
#define NQS_ERR_CUDA        (-5)  /* a CUDA runtime call or kernel launch failed             */
#define NQS_ERR_TIMEOUT     (-6)  /* a bounded device-side wait gave up                      */
#define NQS_ERR_NAN         (-7)  /* a non-finite coefficient or parameter was supplied      */
#define NQS_ERR_ALLOC       (-8)  /* library-owned host or device allocation failed          */
#define NQS_ERR_UNSUPPORTED (-9)  /* valid request outside what this build implements        */

typedef struct nqs_ham_s* nqs_ham_t;
typedef struct nqs_model_s* nqs_model_t;

enum nqs_arch { NQS_ARCH_PRODUCT = 0, NQS_ARCH_MADE = 1, NQS_ARCH_TRANSFORMER = 2 };
enum nqs_precision { NQS_PREC_FP32 = 0, NQS_PREC_BF16 = 1 };
enum nqs_op { NQS_OP_SAMPLE = 0, NQS_OP_LOGPSI = 1, NQS_OP_LOCAL_ENERGY = 2, NQS_OP_BACKWARD = 3,
              NQS_OP_TERM_SWEEP = 4 };

/* Model description (Section 4).
 *  arch         NQS_ARCH_*: PRODUCT (pi(x_order[t]=1) = p[t], phase 0), MADE (modulus MADE with
 *               `layers` hidden layers of width `hidden` plus the two-layer phase MLP of
 *               Section 4), TRANSFORMER (decoder-only, d_model = hidden, `layers` blocks,
 *               `heads` heads; not in the paper).
 *  n_qubits     even, 4..128 (PRODUCT, MADE) or 4..64 (TRANSFORMER).  n_up / n_dn: electrons
 *               per spin, the sector of Eq.
 *               hamming_weight_constraint.
 *  precision    NQS_PREC_FP32 or NQS_PREC_BF16 (bf16 tensor-core contractions, fp32
 *               accumulation; transformer only).
 *  compensated  nonzero: TwoSum/Kahan accumulation of coefficient sums, log-probabilities
 *               and the local-energy reduction.
 *  order        order[t] = qubit sampled at step t; a permutation of 0..n_qubits-1.  The
 *               paper's reverse order (Section 4) is order[t] = n_qubits-1-t. */
typedef struct nqs_model_desc {
    int arch;
    int n_qubits;
    int n_up;
    int n_dn;
    int hidden;
    int layers;
    int heads;
    int precision;
    int compensated;
    int order[128];
} nqs_model_desc;

/* ---------------------------------------------------------------- Hamiltonian */

/* Build a Hamiltonian H = sum_k coeff[k] P(x_mask[k], z_mask[k]) (Eq. hamiltonpauli) and run
 * the term-grouping pass (Section 5.1: "unique flippings"): equal (x,z) strings are merged by
 * fp64 summation in input order, exact zeros dropped, strings grouped by x_mask (the flip
 * pattern m), and the phase (-i)^r of Eq. mtx_element (r = popcount(x & z)) folded into each
 * coefficient.  The grouped table is copied to the current device.
 *   n_qubits 1..128; n_terms >= 1; x_mask, z_mask: host arrays of n_terms masks of W words
 *   each (W = 1 for n_qubits <= 64, else 2), coeff: host array of n_terms (all copied; the
 *   caller keeps ownership).  Errors: NQS_ERR_NQUBITS, NQS_ERR_INVALID_ARG (null pointer,
 *   mask bit >= n_qubits), NQS_ERR_NAN (non-finite coefficient), NQS_ERR_ALLOC, NQS_ERR_CUDA.
 *   Synchronous. */
int nqs_ham_create(int n_qubits, int64_t n_terms, const uint64_t* x_mask, const uint64_t* z_mask,
                   const double* coeff, nqs_ham_t* out);

/* Merged term count K' and group count G. */
int nqs_ham_info(nqs_ham_t ham, int64_t* n_terms_merged, int64_t* n_groups);

/* Copy the grouped table to host arrays: grp_mask[G] (ascending; G * W words), grp_offset[G+1]
 * (terms of group g are [grp_offset[g], grp_offset[g+1])), term_z[K'] (ascending within a
 * group; K' * W words) and the
 * phase-folded coefficients c'_k = c_k (-i)^{r_k} as term_c_re[K'], term_c_im[K'].  Any
 * pointer may be NULL to skip that array.  Synchronous. */
int nqs_ham_export(nqs_ham_t ham, uint64_t* grp_mask, int64_t* grp_offset, uint64_t* term_z,
                   double* term_c_re, double* term_c_im);

void nqs_ham_destroy(nqs_ham_t ham);

/* ---------------------------------------------------------------- model */

/* Validate a description and create a model handle (no parameters bound yet).
 * Errors: NQS_ERR_NQUBITS, NQS_ERR_INVALID_ARG, NQS_ERR_UNSUPPORTED (e.g. MADE wider than
 * 256 or a transformer head size other than 16/32), NQS_ERR_ALLOC. */
int nqs_model_create(const nqs_model_desc* desc, nqs_model_t* out);

/* Total number of fp32 parameters of the flat parameter vector. */
int nqs_model_param_count(nqs_model_t model, int64_t* n_params);

/* Number of named parameter tensors, and the name / offset / element count of tensor `index`
 * inside the flat vector.  Weight matrices are row-major [out][in].  *name points to storage
 * owned by the model handle. */
int nqs_model_param_tensors(nqs_model_t model, int* n_tensors);
int nqs_model_param_info(nqs_model_t model, int index, const char** name, int64_t* offset,
                         int64_t* numel);

/* Borrow the caller's device fp32 parameter vector (param_count floats).  Every later call
 * reads it at execution time, so updates (e.g. nqs_adam_step) take effect without rebinding. */
int nqs_model_bind_params(nqs_model_t model, const float* params_device);

/* Prefix reuse of the transformer local energy (Section 5.1's unique flippings carried over to
 * prefixes: the network's row at sampling position t depends on the bits before t only, so a
 * connected x' shares its rows before its first flip with the sample x, and x' with the same
 * first flips share more).  depth 0: every x' evaluated from position 0; 1: x's keys and values
 * reused up to the first flip; 2: also strings carrying each sample's first flip; 3: also its
 * first two flips; -1 (default): automatic -- depth 3, or, when the particle-number sector holds
 * fewer configurations than one 1024-sample chunk has connected rows, the per-chunk hash
 * deduplication of x' instead.  The local energies do not depend on the depth, bit for bit;
 * the workspace does (query nqs_workspace_size after setting it).  Transformer models only
 * (NQS_ERR_UNSUPPORTED otherwise); NQS_ERR_INVALID_ARG outside -1..3. */
int nqs_model_set_prefix_reuse(nqs_model_t model, int depth);

/* Activation bytes of one sub-pass of the prefix-sharing local energy (the leaves are evaluated
 * in sub-passes of about this many bytes of layer activations, about 40 d_model bytes a row).
 * 0 (default): 16 GiB.  Smaller values bound the workspace (query nqs_workspace_size after
 * setting it) at the cost of more, smaller launches; the local energies do not depend on it.
 * Transformer models only (NQS_ERR_UNSUPPORTED otherwise); NQS_ERR_INVALID_ARG if negative.
 * Not part of the paper's method: a memory/throughput setting of this implementation. */
int nqs_model_set_pass_bytes(nqs_model_t model, int64_t bytes);

void nqs_model_destroy(nqs_model_t model);

/* Workspace bytes that `op` (NQS_OP_*) needs for `batch` rows: samples for LOGPSI,
 * LOCAL_ENERGY, BACKWARD and TERM_SWEEP; the nominal sample count N_s for SAMPLE (with
 * max_unique = batch).  ham may be NULL except for LOCAL_ENERGY and TERM_SWEEP.  The
 * workspace is a caller-owned device buffer, 256-byte aligned. */
int nqs_workspace_size(nqs_model_t model, nqs_ham_t ham, int op, int64_t batch, size_t* bytes);

/* ---------------------------------------------------------------- hot path */

/* Unique-sample autoregressive sampling with counts (Section 4, Sampling; Eq. modifier).
 * One buffer entry with count n_samples is doubled on qubit order[k] at step k = 0..n-1; every
 * nominal sample draws u = word 0 of Philox4x32-10(counter (j, k, 0, 0), key (seed lo, seed
 * hi)) and takes bit 1 iff u < floor(p * 2^32), p the fp32 constrained conditional of its
 * parent; zero-count children are dropped and, if more than max_unique entries remain, the top
 * max_unique by (count desc, bits asc) are kept.
 *   bits_out[capacity * W] (device, uint64; W words per configuration) and counts_out[capacity]
 *   (device, int64) receive the U unique samples in ascending order (as W-word integers);
 *   *n_unique (host) receives U.  If U > capacity,
 *   returns NQS_ERR_CAPACITY with *n_unique = U and nothing written.
 *   p_trace (device, may be NULL): p_trace[k * trace_stride + s] receives the fp32
 *   probability used for parent s at step k (parents in ascending bit order);
 *   trace_stride >= min(n_samples, 2*max_unique).
 *   Requires 1 <= n_samples < 2^31 and max_unique >= 1.
 *   Synchronises `stream` once at the end to read U. */
int nqs_sample(nqs_model_t model, int64_t n_samples, int64_t max_unique, uint64_t seed,
               uint64_t* bits_out, int64_t* counts_out, int64_t capacity, int64_t* n_unique,
               float* p_trace, int64_t trace_stride, void* ws, size_t ws_bytes, void* stream);

/* log f(x) = i phi(x) + 1/2 sum log pihat (Section 4) for B device bitstrings:
 * log_abs[B] and phase[B] (device fp32).  Out-of-sector inputs give log_abs = -inf. */
int nqs_logpsi(nqs_model_t model, const uint64_t* bits, int64_t B, float* log_abs, float* phase,
               void* ws, size_t ws_bytes, void* stream);

/* Term sweep alone (Eq. mtx_element on grouped strings): for each sample x_i (device,
 * in the model's sector) and each group g whose flip x' = x_i ^ m_g stays in the sector,
 * S_g(x_i) = sum_{k in g} c'_k (-1)^{popcount(x_i & z_k)}.  A sample outside the sector gets
 * one row, x' = x_i with S = NaN + i NaN.  Rows are written per sample in group order:
 * row_offset[B+1] (device int64), xprime[row] (W words per row), s_re[row], s_im[row] (device;
 * fp32), capacity rows at most.  If the row count exceeds capacity, returns NQS_ERR_CAPACITY
 * with *n_rows = the count and no rows written.  n_up, n_dn: the sector.  Synchronises
 * `stream` once (to size the output). */
int nqs_term_sweep(nqs_ham_t ham, int n_up, int n_dn, int compensated, const uint64_t* bits,
                   int64_t B, int64_t* row_offset, uint64_t* xprime, float* s_re, float* s_im,
                   int64_t capacity, int64_t* n_rows, void* ws, size_t ws_bytes, void* stream);

/* Local energy (Eq. local_energy_auto; Algorithm 1) for B device bitstrings in the model's
 * sector: eloc[2*i], eloc[2*i+1] (device fp32) = Re, Im of
 *   l(x_i) = sum_g S_g(x_i) f(x_i ^ m_g) / f(x_i)
 * over the in-sector flips (out-of-sector flips have f = 0 under the constraint).  A sample
 * outside the sector gets NaN (it has f(x_i) = 0, so l(x_i) is undefined).  The
 * network is evaluated on every connected x' with the ratio-weighted reduction fused into its
 * epilogue.  Synchronises `stream` once per internal sample chunk (to size the x' stream). */
int nqs_local_energy(nqs_ham_t ham, nqs_model_t model, const uint64_t* bits, int64_t B,
                     float* eloc, void* ws, size_t ws_bytes, void* stream);

/* Vector-Jacobian product of log f (Eq. grad): grad_accum[P] (device fp32) +=
 *   sum_i g_log_abs[i] d log|f(x_i)|/d theta + g_phase[i] d phi(x_i)/d theta
 * with the forward recomputed inside (no saved activations).  Deterministic order. */
int nqs_logpsi_backward(nqs_model_t model, const uint64_t* bits, int64_t B,
                        const float* g_log_abs, const float* g_phase, float* grad_accum,
                        void* ws, size_t ws_bytes, void* stream);

/* nqs_logpsi_backward in two calls, so that the forward recompute (phase 1: needs only the
 * parameters and bits) can run on another stream while the local energy and its statistics
 * produce g_log_abs and g_phase; phase 2 then runs the backward from the recomputed activations.
 * Phase 2 must follow phase 1 with the same model, bits, B and workspace, the parameters
 * unchanged, and ordered after it on the device.  Transformer models need B within one recompute
 * pass (else NQS_ERR_UNSUPPORTED: use nqs_logpsi_backward); for the other models phase 1 does
 * nothing and phase 2 is nqs_logpsi_backward.  g_log_abs, g_phase and grad_accum may be NULL in
 * phase 1.  Same results as nqs_logpsi_backward, bit for bit. */
int nqs_logpsi_backward_phase(nqs_model_t model, int phase, const uint64_t* bits, int64_t B,
                              const float* g_log_abs, const float* g_phase, float* grad_accum,
                              void* ws, size_t ws_bytes, void* stream);

/* FP64 energy statistics (Eq. total_energy_sum with sample counts as weights):
 * stats[0..3] (device double) = Re E_bar, Im E_bar, Var = sum w|E - E_bar|^2 / W, W = sum w.
 * If g_abs and g_phase (device fp32, may be NULL) are given they receive the upstream
 * gradients of the VMC surrogate: g_abs[i] = 2 w_i Re(E_i - E_bar) / W and
 * g_phase[i] = 2 w_i Im(E_i) / W (baseline b = Re E_bar of Eq. grad). */
int nqs_energy_stats(const float* eloc, const int64_t* counts, int64_t B, double* stats,
                     float* g_abs, float* g_phase, void* stream);

/* Per-rank pieces of the data-parallel VMC gradient (Section 5: the B*K summands are split over
 * L GPUs and the gradients averaged).  sums[0..3] (device double) = sum_i w_i Re E_i,
 * sum_i w_i Im E_i, sum_i w_i |E_i|^2 and W = sum_i w_i over this rank's B samples (weights =
 * counts).  If the three device fp32 arrays are given they receive the upstream gradients
 * g_abs_e[i] = 2 w_i Re E_i, g_phase_e[i] = 2 w_i Im E_i and g_abs_w[i] = w_i: the backward
 * (nqs_logpsi_backward) with (g_abs_e, g_phase_e) gives the sum `first`, with (g_abs_w, 0) the
 * sum `second`, and after one all-reduce of [sums, first, second] over the ranks the gradient of
 * Eq. grad is (first - 2 Re(E_bar) second) / W with E_bar = (sums[0] + i sums[1]) / W. */
int nqs_energy_sums(const float* eloc, const int64_t* counts, int64_t B, double* sums, float* g_abs_e,
                    float* g_phase_e, float* g_abs_w, void* stream);

/* One Adam update (Section 5.1) in place on device fp32 arrays of n elements; step is the
 * 1-based iteration number. */
int nqs_adam_step(float* params, const float* grad, float* m, float* v, int64_t n, int step,
                  float lr, float beta1, float beta2, float eps, void* stream);

/* Diagnostic: the library's bf16 tensor-core GEMM on its own (the contraction inside the BF16
 * transformer path).  C[M,N] = A[M,K] . W[N,K]^T + bias with A, W bf16 row-major (device,
 * 16-byte aligned, K % 8 == 0), N % 16 == 0, fp32 accumulation; epilogue 0: C fp32 store,
 * 1: C bf16 = gelu_tanh(.), 2: C fp32 += (.), 4: C bf16[M, 2N] = (hi | lo) with hi = bf16(g),
 * lo = bf16(g - hi), g = gelu_tanh(.); bias (device fp32[N]) may be NULL.  Synchronises
 * `stream`; returns NQS_ERR_TIMEOUT if a bounded device wait gave up. */
int nqs_gemm_bf16(const void* A, const void* W, const float* bias, void* C, int64_t M, int N, int K,
                  int epilogue, void* stream);

/* ---------------------------------------------------------------- no-allocation variant */

/* Size of the library's static device scratch used by nqs_local_energy_noalloc (32 MiB). */
#define NQS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* nqs_local_energy without any allocation, for callers that cannot call cudaMalloc (code inside
 * an allocator's or framework's no-allocation region, plugins handed only their input and output
 * buffers, runtimes that reserve all device memory up front).  The paper has no counterpart: it
 * is an interface convenience of this library.
 *   Same arguments and results as nqs_local_energy, minus the workspace: the scratch is one
 *   static device array of NQS_NOALLOC_SCRATCH_BYTES held by every GPU that loads the library
 *   until the process exits.  No cudaMalloc, cudaFree or allocating library routine is called.
 *   Product and MADE models only (NQS_ERR_UNSUPPORTED otherwise).
 *   Limit: the B per-sample log psi values plus one chunk of at least one sample's sweep rows
 *   must fit in the scratch; larger requests return NQS_ERR_CAPACITY with a message.
 *   The first call on a device looks up the scratch's device address (cudaGetSymbolAddress)
 *   with that device current.  Under lazy module loading (CUDA's default since 12.2) that
 *   lookup loads the library's device module, which is when the array is allocated: make the
 *   first call on each device outside any no-allocation region and before any stream capture.
 *   Every call reuses the same
 *   array: calls whose GPU work overlaps (other streams or host threads) race on it and must be
 *   serialised by the caller.  Asynchronous on `stream`. */
int nqs_local_energy_noalloc(nqs_ham_t ham, nqs_model_t model, const uint64_t* bits, int64_t B,
                             float* eloc, void* stream);

/* ---------------------------------------------------------------- diagnostics */

const char* nqs_strerror(int status);
const char* nqs_last_error(void);

/* Per-kernel device timing with CUDA events recorded on the launching stream.  While enabled,
 * each launch of a timed kernel is bracketed by two events; nqs_profile_read() synchronises
 * the recorded events and returns the summed milliseconds and launch count of the kernel
 * named `kernel` ("term_sweep", "eloc_rows", ...).  nqs_profile_reset() clears the records. */
int nqs_profile_enable(int on);
int nqs_profile_reset(void);
int nqs_profile_read(const char* kernel, double* total_ms, int64_t* launches);
/* Summed algorithmic work recorded with the timed launches of `kernel` since the last reset:
 * useful FLOPs and compulsory DRAM bytes (operands read once, results written once) -- for
 * "tf_gemm" 2*M*N*K FLOPs (the compensated split's second pass not counted) and the bytes of A,
 * W, C (and C read back for a residual add); 0 where no figure is attached. */
int nqs_profile_work(const char* kernel, double* flops, double* bytes);

/* Diagnostic: measured issue rates of the SM pipes that bound the term sweep and the fp32
 * network, in instructions per SM per clock cycle: out[0] 32-bit population count (each probe
 * instruction is paired with one logic op), out[1] three-input logic (LOP3), out[2] 32-bit
 * integer add, out[3] fp32 fused multiply-add.  One CTA of 1024 threads per SM runs eight
 * independent chains of the instruction; the rate is the CTA's instruction count over its own
 * elapsed SM cycles (median over the SMs), so it does not depend on the clock frequency.  The
 * paper has no counterpart: these are the denominators of the rooflines of Section 5.1's
 * operator-matrix evaluation on this GPU.  Synchronous; allocates and frees two small device
 * buffers.  per_sm_per_clock: host double[4]. */
int nqs_probe_pipes(double* per_sm_per_clock);

/* Number of kernels this library has launched in the calling process (all streams). */
int64_t nqs_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* NQS_H */
