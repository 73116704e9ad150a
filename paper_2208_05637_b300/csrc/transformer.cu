// Decoder-only transformer wavefunction (used by the larger workloads; not in the paper) in
// layer-wise kernels over a compact activation buffer of R sequences x T positions.
//
//   tokens     [BOS, x_order[0], ..., x_order[T-2]]        (token ids 2, then bits 0/1)
//   h          tok_emb[token] + pos_emb[t]
//   block l    h += Wo . attn(LN1(h))  ;  h += W2 . gelu(W1 . LN2(h))      (pre-LayerNorm)
//   heads      logit_t = LNf(h_t) . head_w + head_b[t];  phase = LNf(h_{n-2}) . phase_w + phase_b
//   log f      1/2 sum_t log pihat_t(x_t) (Hamming-weight constraint as for MADE) + i phase[sel]
//
// Every GEMM is C[M, N] = A[M, K] . W[N, K]^T (+ bias, + epilogue) with M = R*T rows; the four
// block GEMMs run in FP32 on CUDA cores (this file) or in BF16 on the tensor cores
// (tc_gemm.cu, precision NQS_PREC_BF16).  Attention (T <= 64, head size 16/32) runs per
// (sequence, head) on CUDA cores in FP32.  The last kernel applies LNf, the heads and the
// constraint and, for the local energy, multiplies the row's coefficient sum S by
// exp(log|f(x')| - log|f(x)|) e^{i (phi(x') - phi(x))} -- the ratio-weighted reduction is fused
// into the network's epilogue; a per-sample TwoSum pass adds the rows of each sample.
#include "tf_common.cuh"

namespace nqs {

namespace {

// ---------------------------------------------------------------- heads and constraint
// One warp per sequence.  mode 0: (log|f|, phi) per sequence; mode 1: local-energy
// contribution of an x' row; mode 2: sampler conditional at position k = T-1.
struct HeadArgs {
    int mode;
    float* la;                 // mode 0
    float* ph;
    const uint64_t* xsample;   // mode 1: the samples of the chunk
    const float* la_x;
    const float* ph_x;
    const int64_t* seg;        // mode 1: row offsets per sample (stride seg_stride), nseg samples
    int64_t seg_stride, nseg, row0;
    const float4* S;
    float2* contrib;
    float* p_out;              // mode 2
    uint64_t* thr;
    float* trace;
    int step_pos;              // mode 2 with h holding only position step_pos (T = 1), else -1
};

template <int DPL>
__global__ void __launch_bounds__(256)
heads_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
             const float* __restrict__ h, int64_t R, int T, HeadArgs args) {
    const int d = mc.hidden;
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= R) return;
    const uint64_t x = bits[r];
    float hw[DPL], g[DPL], bb[DPL];
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        hw[i] = P[mc.head_w + j]; g[i] = P[mc.lnf_g + j]; bb[i] = P[mc.lnf_b + j];
    }
    const float inv_d = 1.f / (float)d;   // d is a power of two: exact
    auto lnf_row = [&](int t, float (&y)[DPL]) {
        const float* row = h + (r * T + t) * (int64_t)d;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) { y[i] = row[lane + 32 * i]; s += y[i]; }
        const float mu = warp_sum(s) * inv_d;
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) { const float c = y[i] - mu; q += c * c; }
        const float rstd = rsqrtf(fmaf(warp_sum(q), inv_d, LN_EPS));
#pragma unroll
        for (int i = 0; i < DPL; ++i) y[i] = (y[i] - mu) * rstd * g[i] + bb[i];
    };
    if (args.mode == 2) {
        const int k = args.step_pos >= 0 ? args.step_pos : T - 1;
        int ones0 = 0, ones1 = 0;
        for (int t = 0; t < k; ++t) {
            const int b = (int)((x >> mc.order[t]) & 1ull);
            if (mc.order[t] & 1) ones1 += b; else ones0 += b;
        }
        const int sp = mc.order[k] & 1;
        const int c = sp ? ones1 : ones0;
        const int need = sp ? mc.n_dn : mc.n_up;
        float p;
        if (c + mc.after[k] < need) p = 1.f;
        else if (c >= need) p = 0.f;
        else {
            float y[DPL];
            lnf_row(args.step_pos >= 0 ? 0 : k, y);
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < DPL; ++i) a = fmaf(y[i], hw[i], a);
            a = warp_sum(a) + P[mc.head_b + k];
            p = 1.f / (1.f + expf(-a));
        }
        if (lane == 0) {
            args.p_out[r] = p;
            args.thr[r] = (uint64_t)(p * 4294967296.0f);
            if (args.trace) args.trace[r] = p;
        }
        return;
    }
    // full log psi over all n positions
    float acc = 0.f, err = 0.f;
    int ones0 = 0, ones1 = 0;
    bool bad = false;
    float phase = 0.f;
    for (int t = 0; t < mc.n; ++t) {
        const int sp = mc.order[t] & 1;
        const int b = (int)((x >> mc.order[t]) & 1ull);
        const int c = sp ? ones1 : ones0;
        const int need = sp ? mc.n_dn : mc.n_up;
        const bool f1 = c + mc.after[t] < need, f0 = c >= need;
        if (f1) bad |= (b == 0);
        else if (f0) bad |= (b == 1);
        if (!(f1 || f0) || t == mc.n - 2) {
            float y[DPL];
            lnf_row(t, y);
            if (!(f1 || f0)) {
                float a = 0.f;
#pragma unroll
                for (int i = 0; i < DPL; ++i) a = fmaf(y[i], hw[i], a);
                a = warp_sum(a) + P[mc.head_b + t];
                const float lp = logsig(b ? a : -a);
                if (mc.compensated) two_sum_acc(acc, err, lp); else acc += lp;
            }
            if (t == mc.n - 2) {
                const int sel = (int)(((x >> mc.order[mc.n - 2]) & 1ull) * 2 + ((x >> mc.order[mc.n - 1]) & 1ull));
                float a = 0.f;
#pragma unroll
                for (int i = 0; i < DPL; ++i) a = fmaf(y[i], P[mc.phase_w + sel * d + lane + 32 * i], a);
                phase = warp_sum(a) + P[mc.phase_b + sel];
            }
        }
        if (sp) ones1 += b; else ones0 += b;
    }
    const float la = bad ? -INFINITY : 0.5f * (acc + err);
    if (lane != 0) return;
    if (args.mode == 0) {
        args.la[r] = la;
        args.ph[r] = phase;
        return;
    }
    // mode 1: row r of the chunk belongs to the sample whose segment contains row0 + r
    const int64_t grow = args.row0 + r;
    int64_t lo = 0, hi = args.nseg - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (args.seg[mid * args.seg_stride] <= grow) lo = mid; else hi = mid - 1;
    }
    const float4 s4 = args.S[grow];
    const float sre = s4.x + s4.y, sim = s4.z + s4.w;
    float cr = sre, ci = sim;
    if (x != args.xsample[lo]) {
        const float mag = expf(la - args.la_x[lo]);
        float sn, cs;
        sincosf(phase - args.ph_x[lo], &sn, &cs);
        const float rr = mag * cs, ri = mag * sn;
        cr = sre * rr - sim * ri;
        ci = sre * ri + sim * rr;
    }
    args.contrib[grow] = make_float2(cr, ci);
}

// Attention of position k for R prefixes whose keys and values of positions j < k sit in the
// per-step QKV slabs of the sampler cache (slab j holds [cap][3d] for the prefixes of step j;
// anc[r * n + j] is the slot of prefix r's ancestor at step j; position k is row r of slab k).
// One CTA per prefix, one warp per head, lanes over the key positions j = lane, lane + 32
// (k < 64): every lane resolves its ancestor slot, then scores, warp max / sum in the log2
// domain and the weighted value rows summed across the lanes.
template <int MODE, int DH>
__global__ void __launch_bounds__(256)
attention_step_kernel(const float* __restrict__ slab0, int64_t slab_stride, int64_t cap,
                      const int32_t* __restrict__ anc, int n, int k, const int64_t* __restrict__ Udev,
                      int64_t R, int d, int H, void* __restrict__ o) {
    const int lane = threadIdx.x & 31, h = threadIdx.x >> 5;
    const int64_t r = blockIdx.x;
    const int64_t U = min(*Udev, R);
    if (r >= U || h >= H) return;
    const int ld = 3 * d;
    const float scale = rsqrtf((float)DH) * 1.4426950408889634f;   // log2 domain
    const float* own = slab0 + (int64_t)k * slab_stride + r * ld;
    // key rows of this lane's positions (j0 = lane, j1 = lane + 32)
    const float* kr[2] = {nullptr, nullptr};
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        const int j = lane + 32 * h2;
        if (j > k) continue;
        int64_t slot = r;
        if (j < k) {
            slot = anc[r * n + j];
            slot = slot < 0 ? 0 : (slot >= cap ? cap - 1 : slot);
        }
        kr[h2] = slab0 + (int64_t)j * slab_stride + slot * ld;
    }
    float q[DH];
#pragma unroll
    for (int j4 = 0; j4 < DH / 4; ++j4) {
        const float4 x = reinterpret_cast<const float4*>(own + h * DH)[j4];
        q[4 * j4] = x.x * scale; q[4 * j4 + 1] = x.y * scale; q[4 * j4 + 2] = x.z * scale; q[4 * j4 + 3] = x.w * scale;
    }
    float sc[2] = {-INFINITY, -INFINITY};
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2)
        if (kr[h2]) sc[h2] = att_dot<DH>(q, reinterpret_cast<const float4*>(kr[h2] + d + h * DH));
    float m = fmaxf(sc[0], sc[1]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    float e[2], l = 0.f;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) { e[h2] = kr[h2] ? exp2f(sc[h2] - m) : 0.f; l += e[h2]; }
    l = warp_sum(l);
    float acc[DH];
#pragma unroll
    for (int c = 0; c < DH; ++c) acc[c] = 0.f;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        if (!kr[h2]) continue;
        const float4* vr = reinterpret_cast<const float4*>(kr[h2] + 2 * d + h * DH);
#pragma unroll
        for (int j4 = 0; j4 < DH / 4; ++j4) {
            const float4 v4 = vr[j4];
            acc[4 * j4] = fmaf(e[h2], v4.x, acc[4 * j4]);
            acc[4 * j4 + 1] = fmaf(e[h2], v4.y, acc[4 * j4 + 1]);
            acc[4 * j4 + 2] = fmaf(e[h2], v4.z, acc[4 * j4 + 2]);
            acc[4 * j4 + 3] = fmaf(e[h2], v4.w, acc[4 * j4 + 3]);
        }
    }
#pragma unroll
    for (int c = 0; c < DH; ++c) acc[c] = warp_sum(acc[c]);
    if (lane == 0) att_store_row<MODE, DH>(acc, l, o, r, d, h * DH);
}

// Heads of whole sequences from the per-row logits and phase dots left by the fused last MLP
// (modes 0 and 1 of HeadArgs): one warp per sequence, lane l taking positions t = l, l + 32.  A
// lane applies the Hamming-weight constraint at its positions (forced conditionals and
// violations from the same-spin ones before t) and the log-sigmoid of the free ones; the lanes'
// sums are joined with TwoSum (compensated models) or plainly.
__global__ void __launch_bounds__(256)
heads_reduce_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
                    const float* __restrict__ logit, const float* __restrict__ hph, int64_t R, HeadArgs args) {
    const int n = mc.n;
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= R) return;
    const uint64_t x = bits[r];
    float s = 0.f, e = 0.f;
    bool bad = false;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int t = lane + 32 * half;
        if (t >= n) continue;
        const int q = mc.order[t], sp = q & 1;
        const int b = (int)((x >> q) & 1ull);
        int c = 0;
        for (int u = 0; u < t; ++u) {
            const int qu = mc.order[u];
            if ((qu & 1) == sp) c += (int)((x >> qu) & 1ull);
        }
        const int need = sp ? mc.n_dn : mc.n_up;
        const bool f1 = c + mc.after[t] < need, f0 = c >= need;
        if (f1) bad |= (b == 0);
        else if (f0) bad |= (b == 1);
        if (!(f1 || f0)) {
            const float a = logit[r * n + t];
            const float lp = logsig(b ? a : -a);
            if (mc.compensated) two_sum_acc(s, e, lp); else s += lp;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, off), e2 = __shfl_xor_sync(0xffffffffu, e, off);
        if (mc.compensated) { e += e2; two_sum_acc(s, e, s2); }
        else s += s2;
    }
    bad = __any_sync(0xffffffffu, bad);
    // phase head: LNf of h at position n - 2 (d = 64, two features a lane), the selected row
    const int sel = (int)(((x >> mc.order[n - 2]) & 1ull) * 2 + ((x >> mc.order[n - 1]) & 1ull));
    const float2 hv = reinterpret_cast<const float2*>(hph + r * 64)[lane];
    const float mu = warp_sum(hv.x + hv.y) * (1.f / 64.f);
    const float c0 = hv.x - mu, c1 = hv.y - mu;
    const float rstd = rsqrtf(fmaf(warp_sum(fmaf(c0, c0, c1 * c1)), 1.f / 64.f, LN_EPS));
    const int j = 2 * lane;
    const float y0 = c0 * rstd * P[mc.lnf_g + j] + P[mc.lnf_b + j];
    const float y1 = c1 * rstd * P[mc.lnf_g + j + 1] + P[mc.lnf_b + j + 1];
    const float* pw = P + mc.phase_w + sel * 64 + j;
    const float phase = warp_sum(fmaf(y0, pw[0], y1 * pw[1])) + P[mc.phase_b + sel];
    if (lane != 0) return;
    const float la = bad ? -INFINITY : 0.5f * (s + e);
    if (args.mode == 0) {
        args.la[r] = la;
        args.ph[r] = phase;
        return;
    }
    // mode 1: row r of the chunk belongs to the sample whose segment contains row0 + r
    const int64_t grow = args.row0 + r;
    int64_t lo = 0, hi = args.nseg - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (args.seg[mid * args.seg_stride] <= grow) lo = mid; else hi = mid - 1;
    }
    const float4 s4 = args.S[grow];
    const float sre = s4.x + s4.y, sim = s4.z + s4.w;
    float cr = sre, ci = sim;
    if (x != args.xsample[lo]) {
        const float mag = expf(la - args.la_x[lo]);
        float sn, cs;
        sincosf(phase - args.ph_x[lo], &sn, &cs);
        const float rr = mag * cs, ri = mag * sn;
        cr = sre * rr - sim * ri;
        ci = sre * ri + sim * rr;
    }
    args.contrib[grow] = make_float2(cr, ci);
}

// Per-sample sum of the row contributions (TwoSum), one CTA per sample.
__global__ void __launch_bounds__(128)
segment_sum_kernel(const int64_t* __restrict__ seg, int64_t seg_stride, int64_t nseg,
                   const float2* __restrict__ contrib, int compensated, float* __restrict__ eloc) {
    __shared__ float red[4][128];
    for (int64_t i = blockIdx.x; i < nseg; i += gridDim.x) {
        const int64_t r0 = seg[i * seg_stride], r1 = seg[(i + 1) * seg_stride];
        float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const float2 c = contrib[r];
            if (compensated) { two_sum_acc(re, re_e, c.x); two_sum_acc(im, im_e, c.y); }
            else { re += c.x; im += c.y; }
        }
        red[0][threadIdx.x] = re; red[1][threadIdx.x] = re_e;
        red[2][threadIdx.x] = im; red[3][threadIdx.x] = im_e;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) {
                float a = red[0][threadIdx.x], ae = red[1][threadIdx.x] + red[1][threadIdx.x + st];
                two_sum_acc(a, ae, red[0][threadIdx.x + st]);
                red[0][threadIdx.x] = a; red[1][threadIdx.x] = ae;
                float b = red[2][threadIdx.x], be = red[3][threadIdx.x] + red[3][threadIdx.x + st];
                two_sum_acc(b, be, red[2][threadIdx.x + st]);
                red[2][threadIdx.x] = b; red[3][threadIdx.x] = be;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            eloc[2 * i] = red[0][0] + red[1][0];
            eloc[2 * i + 1] = red[2][0] + red[3][0];
        }
        __syncthreads();
    }
}

inline int blocks_for(int64_t rows, int per) { return (int)((rows + per - 1) / per); }

template <class F>
int with_dpl(int d, F&& f) {
    switch (d / 32) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 8: return f(std::integral_constant<int, 8>{});
        default:
            set_error("transformer d_model must be 32, 64, 128 or 256");
            return NQS_ERR_UNSUPPORTED;
    }
}

}  // namespace

// ====================================================================== host side
int64_t tf_seq_capacity(const ModelConst& mc) {
    // Sequences per pass: the pass's activations (h, a, qkv, o and the 4d MLP buffer, about
    // 10*d floats per position) are kept near 1 GB.  Smaller, L2-resident passes lose more to
    // the extra launches than they gain in bandwidth; larger ones leave fewer launch gaps.
    const int64_t per_seq = (int64_t)mc.n * mc.hidden * 10 * 4;
    int64_t R = 64;
    while (R * 2 * per_seq <= (1024ll << 20) && R < 32768) R *= 2;
    return R;
}

void tf_layout(Carver& c, const ModelConst& mc, int64_t R, TfBufs& b) {
    const int64_t M = R * mc.n, d = mc.hidden;
    b.R = R;
    b.h = c.take<float>(M * d);
    b.a = c.take<float>(M * d);          // fp32 or bf16 view
    b.qkv = c.take<float>(M * 3 * d);
    b.o = c.take<float>(M * d);          // fp32 or bf16 view
    b.mid = c.take<float>(M * 4 * d);    // fp32 or bf16 view
    b.logit = c.take<float>(M);
    b.tab_h = c.take<float>(3 * (int64_t)mc.n * d);
    b.tab_qkv = c.take<float>(3 * (int64_t)mc.n * 3 * d);
    b.hph = c.take<float>(R * 64);
    b.fused_heads = false;
}

int tf_gemm(const ModelConst& mc, const TfWeights& w, int which, int layer, const void* A,
            void* C, int64_t M, int N, int K, int epi, const float* bias, cudaStream_t s) {
    // compulsory bytes: A and W read once, C written once (and read once for a residual add)
    const bool bf = mc.precision == NQS_PREC_BF16;
    const double split = (bf && mc.compensated) ? 2.0 : 1.0;
    const double a_el = bf ? 2.0 * split : 4.0, w_el = bf ? 2.0 * split : 4.0;
    const double c_el = epi == TF_EPI_GELU ? (bf ? 2.0 * split : 4.0) : 4.0;   // TF_EPI_SPLIT: 2 x bf16
    const double bytes = (double)M * K * a_el + (double)N * K * w_el +
                         (double)M * N * c_el * (epi == TF_EPI_RESID ? 2.0 : 1.0);
    ProfScope ps("tf_gemm", s, 2.0 * (double)M * N * K, bytes);
    if (bf) {
        // compensated form: A = [A_hi | A_lo] and B = [W | W], so K doubles
        const bool split = mc.compensated != 0;
        const int e = (epi == TF_EPI_GELU && split) ? TF_EPI_GELU2 : epi;
        return tc_gemm_bf16(A, w.bf16 + w.bf16_off[layer][which], bias, C, M, N, split ? 2 * K : K, e, s);
    }
    if (epi == TF_EPI_SPLIT) { set_error("split-layout projection needs a bf16 model"); return NQS_ERR_UNSUPPORTED; }
    const float* W = w.fp32 + w.fp32_off[layer][which];
    dim3 grid((unsigned)((N + SG_BN - 1) / SG_BN), (unsigned)((M + SG_BM - 1) / SG_BM));
    const float* Af = (const float*)A;
    float* Cf = (float*)C;
    switch (epi) {
        case TF_EPI_STORE: sgemm_kernel<float, false, TF_EPI_STORE, float><<<grid, 256, 0, s>>>(Af, W, bias, Cf, M, N, K); break;
        case TF_EPI_GELU: sgemm_kernel<float, false, TF_EPI_GELU, float><<<grid, 256, 0, s>>>(Af, W, bias, Cf, M, N, K); break;
        case TF_EPI_RESID: sgemm_kernel<float, false, TF_EPI_RESID, float><<<grid, 256, 0, s>>>(Af, W, bias, Cf, M, N, K); break;
        default: set_error("bad GEMM epilogue"); return NQS_ERR_INVALID_ARG;
    }
    NQS_LAUNCHED();
    return NQS_OK;
}

// Attention-output projection of block l with the residual add and LayerNorm 2 fused
// (compensated BF16, d_model 64 or 128): h += Wo . o + bo; a = LN2(h).
int tf_resid_ln(const ModelConst& mc, const float* P, const TfWeights& w, int layer, const void* o, float* h,
                void* a, int64_t M, cudaStream_t s, const TcTokTable* h_old) {
    const int d = mc.hidden;
    // A (hi+lo) read, h read (unless it comes from the token-position table) and written,
    // a (hi+lo) written, weights
    const double bytes = (double)M * 2 * d * 2 + (double)M * d * 4 * (h_old ? 1 : 2) + (double)M * 2 * d * 2 +
                         2.0 * d * d * 2;
    ProfScope ps("tf_resid_ln", s, 2.0 * (double)M * d * d, bytes);
    return tc_gemm_bf16_resid_ln(o, w.bf16 + w.bf16_off[layer][TF_WO], P + mc.bo[layer], h, a, P + mc.ln2_g[layer],
                                 P + mc.ln2_b[layer], M, d, 2 * d, s, h_old);
}

// The first block's rows as functions of the (token, position) pair, for positions 0..T-1 of the
// compensated d_model-64 model: h0 = tok_emb[token] + pos_emb[t] and the projection
// LN1_0(h0) . Wqkv^T with the tensor-core operands (hi + lo activations against the bf16
// weights, products summed in fp32; the bias is added where the rows are used).  One CTA of 192
// threads per (token, position); rows that never occur (token 2 past t = 0, tokens 0 and 1 at
// t = 0) are computed too and left unused.
__global__ void __launch_bounds__(192)
tok_table_kernel(ModelConst mc, const float* __restrict__ P, const __nv_bfloat16* __restrict__ Wqkv, int ldw, int T,
                 float* __restrict__ tab_h, float* __restrict__ tab_qkv, int compensated) {
    constexpr int D = 64;
    __shared__ float s_hi[D], s_lo[D];
    const int row = blockIdx.x;                    // token * T + t
    const int tok = row / T, t = row - tok * T;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, c0 = 2 * lane;
        float v[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            v[i] = P[mc.tok_emb + tok * D + c0 + i] + P[mc.pos_emb + t * D + c0 + i];
            tab_h[row * D + c0 + i] = v[i];
        }
        const float inv_d = 1.f / (float)D;
        const float mu = warp_sum(v[0] + v[1]) * inv_d;
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < 2; ++i) { const float c = v[i] - mu; q += c * c; }
        const float rstd = rsqrtf(fmaf(warp_sum(q), inv_d, LN_EPS));
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float y = (v[i] - mu) * rstd * P[mc.ln1_g[0] + c0 + i] + P[mc.ln1_b[0] + c0 + i];
            const float hi = __bfloat162float(__float2bfloat16_rn(y));
            s_hi[c0 + i] = hi;
            s_lo[c0 + i] = compensated ? __bfloat162float(__float2bfloat16_rn(y - hi)) : 0.f;
        }
    }
    __syncthreads();
    const int j = threadIdx.x;                     // output column
    const __nv_bfloat16* wr = Wqkv + (int64_t)j * ldw;
    float acc = 0.f;
#pragma unroll 8
    for (int k = 0; k < D; ++k) {
        const float wk = __bfloat162float(wr[k]);
        acc = fmaf(s_hi[k], wk, acc);
        acc = fmaf(s_lo[k], wk, acc);
    }
    tab_qkv[row * 3 * D + j] = acc;
}

// MLP half of block l: h += W2 . gelu(W1 . a + b1) + b2.  Compensated BF16 models with d_model
// 64 or 128 run it as one fused tensor-core kernel (the 4d hidden layer stays on chip); the
// others as two GEMMs through the mid buffer.
int tf_mlp(const ModelConst& mc, const float* P, const TfWeights& w, int layer, const void* a, void* mid,
           float* h, int64_t M, cudaStream_t s, const TcMlpHead* head) {
    const int d = mc.hidden;
    if (mc.precision == NQS_PREC_BF16 && mc.compensated && (d == 64 || d == 128)) {
        const double flops = 2.0 * 2.0 * (double)M * 4 * d * d;
        // A (hi+lo) read, h read (and written unless the heads are fused), W1 and W2 once
        const double bytes = (double)M * 2 * d * 2 + (double)M * d * 4 * (head ? 1 : 2) + 8.0 * d * d * 2 +
                             (head ? (double)M * 4 : 0.0);
        ProfScope ps("tf_mlp", s, flops, bytes);
        return tc_mlp_bf16(a, w.bf16 + w.bf16_off[layer][TF_W1], P + mc.b1[layer], w.bf16 + w.bf16_off[layer][TF_W2],
                           P + mc.b2[layer], h, M, d, s, head);
    }
    NQS_TRY(tf_gemm(mc, w, TF_W1, layer, a, mid, M, 4 * d, d, TF_EPI_GELU, P + mc.b1[layer], s));
    return tf_gemm(mc, w, TF_W2, layer, mid, h, M, d, 4 * d, TF_EPI_RESID, P + mc.b2[layer], s);
}

int tf_prepare_weights(const ModelConst& mc, const float* P, TfWeights& w, cudaStream_t s) {
    w.fp32 = P;
    for (int l = 0; l < mc.layers; ++l) {
        w.fp32_off[l][TF_WQKV] = mc.wqkv[l];
        w.fp32_off[l][TF_WO] = mc.wo[l];
        w.fp32_off[l][TF_W1] = mc.w1[l];
        w.fp32_off[l][TF_W2] = mc.w2[l];
    }
    if (mc.precision != NQS_PREC_BF16) return NQS_OK;
    if (!w.bf16) { set_error("bf16 weight buffer missing"); return NQS_ERR_INVALID_ARG; }
    const int64_t d = mc.hidden;
    const int dup = mc.compensated ? 1 : 0;
    int64_t off = 0;
    const int64_t rows[4] = {3 * d, d, 4 * d, d}, cols[4] = {d, d, d, 4 * d};
    WconvList wl{};
    wl.dup = dup;
    wl.f32_out = 0;
    for (int l = 0; l < mc.layers; ++l) {
        for (int q = 0; q < 4; ++q) {
            w.bf16_off[l][q] = off;
            const int64_t n = rows[q] * cols[q];
            WconvJob& J = wl.job[wl.njobs++];
            J.src = P + w.fp32_off[l][q];
            J.dst = reinterpret_cast<__nv_bfloat16*>(w.bf16) + off;
            J.start = wl.total;
            J.cols = (int)cols[q];
            wl.total += n;
            off += ((n << dup) + 127) & ~int64_t(127);   // 256-byte aligned matrices
        }
    }
    // all blocks' matrices in one launch
    const int grid = (int)std::min<int64_t>((wl.total + 255) / 256, (int64_t)num_sms() * 8);
    wconv_kernel<<<grid, 256, 0, s>>>(wl);
    NQS_LAUNCHED();
    return NQS_OK;
}

int64_t tf_bf16_weight_elems(const ModelConst& mc) {
    const int64_t d = mc.hidden;
    const int dup = mc.compensated ? 1 : 0;
    int64_t total = 0;
    const int64_t sizes[4] = {3 * d * d, d * d, 4 * d * d, 4 * d * d};
    for (int l = 0; l < mc.layers; ++l)
        for (int q = 0; q < 4; ++q) total += ((sizes[q] << dup) + 127) & ~int64_t(127);
    return total;
}

// Forward of R sequences over their first T positions, leaving the final residual stream in
// b.h.  `bits` are the R configurations.
template <int MODE>
static int tf_forward_mode(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
                           int64_t R, int T, TfBufs& b, cudaStream_t s, bool head_logits) {
    const int d = mc.hidden;
    const int64_t M = R * T;
    b.fused_heads = false;
    return with_dpl(d, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        // algorithmic bytes: an activation element is 4 bytes in every storage form (fp32, or
        // bf16 hi + lo); a plain bf16 form would be 2
        const double act_b = MODE == ACT_BF16 ? 2.0 : 4.0;
        const double ln_bytes = (double)M * d * (4.0 + act_b);       // h read (or written) + a written
        const bool fused_qkv_attention = MODE == ACT_BF16X2 && d == 64 && mc.heads == 4 && T <= 64;
        // the compensated d = 64 forward takes the first block's h and q | k | v rows from tables
        // over the 3T (token, position) pairs; the others embed every row
        const bool tables = fused_qkv_attention && tc_qkv_gather_fits(T);
        TcTokTable tab_qkv, tab_h;
        if (tables) {
            tab_qkv.tab = b.tab_qkv; tab_qkv.bits = bits; tab_qkv.T = T;
            for (int t = 0; t < mc.n; ++t) tab_qkv.order[t] = mc.order[t];
            tab_h = tab_qkv;
            tab_h.tab = b.tab_h;
            ProfScope ps("tf_tok_table", s, 2.0 * 3 * T * 2 * d * 3 * d, 3.0 * T * 4 * d * 4);
            tok_table_kernel<<<3 * T, 192, 0, s>>>(mc, P, reinterpret_cast<const __nv_bfloat16*>(w.bf16 + w.bf16_off[0][TF_WQKV]),
                                                   2 * d, T, b.tab_h, b.tab_qkv, 1);
            NQS_LAUNCHED();
        } else {
            ProfScope ps("tf_layernorm", s, 0.0, ln_bytes);
            embed_ln_kernel<MODE, DPL><<<ln_grid(M), 256, 0, s>>>(mc, P, bits, R, T, 0, b.h, b.a);
            NQS_LAUNCHED();
        }
        for (int l = 0; l < mc.layers; ++l) {
            if (fused_qkv_attention) {
                // A (hi+lo) read unless gathered, o (hi+lo) written, Wqkv
                const bool gather = tables && l == 0;
                ProfScope ps("tf_qkv_attention", s, gather ? 0.0 : 2.0 * (double)M * 3 * d * d,
                             (gather ? (double)R * 8 : (double)M * 2 * d * 2 + 3.0 * d * d * 2) + (double)M * d * act_b);
                NQS_TRY(tc_qkv_attention_bf16(b.a, w.bf16 + w.bf16_off[l][TF_WQKV], P + mc.bqkv[l], b.o, R, T, s,
                                              gather ? &tab_qkv : nullptr));
            } else {
                NQS_TRY(tf_gemm(mc, w, TF_WQKV, l, b.a, b.qkv, M, 3 * d, d, TF_EPI_STORE, P + mc.bqkv[l], s));
                ProfScope ps("tf_attention", s, 0.0, (double)M * 3 * d * 4 + (double)M * d * act_b);
                NQS_CK(launch_attention<MODE>(b.qkv, R, T, d, mc.heads, b.o, s));
                count_launch();
            }
            if (MODE == ACT_BF16X2 && d == 64) {
                NQS_TRY(tf_resid_ln(mc, P, w, l, b.o, b.h, b.a, M, s, tables && l == 0 ? &tab_h : nullptr));
            } else {
                NQS_TRY(tf_gemm(mc, w, TF_WO, l, b.o, b.h, M, d, d, TF_EPI_RESID, P + mc.bo[l], s));
                ProfScope ps("tf_layernorm", s, 0.0, ln_bytes);
                layernorm_kernel<MODE, DPL><<<ln_grid(M), 256, 0, s>>>(b.h, M, d, P + mc.ln2_g[l], P + mc.ln2_b[l], b.a);
                NQS_LAUNCHED();
            }
            // whole sequences of the compensated d = 64 model: the last MLP also applies LNf and
            // the output / phase heads and leaves per-row logits instead of the final h
            const bool fuse_heads = head_logits && l + 1 == mc.layers && T == mc.n && MODE == ACT_BF16X2 && d == 64;
            if (fuse_heads) {
                TcMlpHead hd{P + mc.lnf_g, P + mc.lnf_b, P + mc.head_w, P + mc.head_b, mc.n, b.logit, b.hph};
                NQS_TRY(tf_mlp(mc, P, w, l, b.a, b.mid, b.h, M, s, &hd));
                b.fused_heads = true;
            } else {
                NQS_TRY(tf_mlp(mc, P, w, l, b.a, b.mid, b.h, M, s));
            }
            if (l + 1 < mc.layers) {
                ProfScope ps("tf_layernorm", s, 0.0, ln_bytes);
                layernorm_kernel<MODE, DPL><<<ln_grid(M), 256, 0, s>>>(b.h, M, d, P + mc.ln1_g[l + 1], P + mc.ln1_b[l + 1], b.a);
                NQS_LAUNCHED();
            }
        }
        return NQS_OK;
    });
}

// Forward of R sequences over their first T positions, leaving the final residual stream in
// b.h.  `bits` are the R configurations.
int tf_forward(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
               int64_t R, int T, TfBufs& b, cudaStream_t s, bool head_logits) {
    if (mc.precision != NQS_PREC_BF16) return tf_forward_mode<ACT_F32>(mc, P, w, bits, R, T, b, s, head_logits);
    if (mc.compensated) return tf_forward_mode<ACT_BF16X2>(mc, P, w, bits, R, T, b, s, head_logits);
    return tf_forward_mode<ACT_BF16>(mc, P, w, bits, R, T, b, s, head_logits);
}

// Position k of R prefixes (bits) for the sampler, with the keys and values of positions < k
// read from the cache (kc) and those of position k written into slab k: the forward of one
// position per prefix, leaving its final residual stream in b.h (R rows).
template <int MODE>
static int tf_step_mode(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
                        int64_t R, int k, const TfStepCache& kc, TfBufs& b, cudaStream_t s) {
    const int d = mc.hidden, H = mc.heads, dh = d / H;
    const int64_t layer_stride = (int64_t)mc.n * kc.cap * 3 * d;   // slabs of one layer
    const int64_t slab_stride = kc.cap * 3 * d;
    return with_dpl(d, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        embed_ln_kernel<MODE, DPL><<<ln_grid(R), 256, 0, s>>>(mc, P, bits, R, 1, k, b.h, b.a);
        NQS_LAUNCHED();
        for (int l = 0; l < mc.layers; ++l) {
            float* slab0 = kc.kv + l * layer_stride;
            NQS_TRY(tf_gemm(mc, w, TF_WQKV, l, b.a, slab0 + k * slab_stride, R, 3 * d, d, TF_EPI_STORE,
                            P + mc.bqkv[l], s));
            {
                ProfScope ps("tf_step_attention", s);
                const unsigned grid = (unsigned)R;                // one CTA per prefix, one warp per head
                if (dh == 16)
                    attention_step_kernel<MODE, 16><<<grid, 32 * H, 0, s>>>(slab0, slab_stride, kc.cap, kc.anc, mc.n, k,
                                                                            kc.Udev, R, d, H, b.o);
                else
                    attention_step_kernel<MODE, 32><<<grid, 32 * H, 0, s>>>(slab0, slab_stride, kc.cap, kc.anc, mc.n, k,
                                                                            kc.Udev, R, d, H, b.o);
                NQS_LAUNCHED();
            }
            if (MODE == ACT_BF16X2 && d == 64) {
                NQS_TRY(tf_resid_ln(mc, P, w, l, b.o, b.h, b.a, R, s));
            } else {
                NQS_TRY(tf_gemm(mc, w, TF_WO, l, b.o, b.h, R, d, d, TF_EPI_RESID, P + mc.bo[l], s));
                layernorm_kernel<MODE, DPL><<<ln_grid(R), 256, 0, s>>>(b.h, R, d, P + mc.ln2_g[l], P + mc.ln2_b[l], b.a);
                NQS_LAUNCHED();
            }
            NQS_TRY(tf_mlp(mc, P, w, l, b.a, b.mid, b.h, R, s));
            if (l + 1 < mc.layers) {
                layernorm_kernel<MODE, DPL><<<ln_grid(R), 256, 0, s>>>(b.h, R, d, P + mc.ln1_g[l + 1], P + mc.ln1_b[l + 1], b.a);
                NQS_LAUNCHED();
            }
        }
        return NQS_OK;
    });
}

int tf_step(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits, int64_t R, int k,
            const TfStepCache& kc, TfBufs& b, cudaStream_t s) {
    if (R > kc.cap) { set_error("sampler step: more prefixes than the cache holds"); return NQS_ERR_CAPACITY; }
    if (mc.precision != NQS_PREC_BF16) return tf_step_mode<ACT_F32>(mc, P, w, bits, R, k, kc, b, s);
    if (mc.compensated) return tf_step_mode<ACT_BF16X2>(mc, P, w, bits, R, k, kc, b, s);
    return tf_step_mode<ACT_BF16>(mc, P, w, bits, R, k, kc, b, s);
}

int64_t tf_step_cache_bytes(const ModelConst& mc, int64_t cap) {
    const int64_t slabs = (int64_t)mc.n * mc.layers * cap * 3 * mc.hidden * (int64_t)sizeof(float);
    const int64_t anc = 2 * cap * (int64_t)mc.n * (int64_t)sizeof(int32_t);
    const int64_t par = 2 * cap * (int64_t)sizeof(int32_t);
    return slabs + anc + par + 5 * 256;   // five 256-byte aligned pieces
}

int tf_heads(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t R, int T,
             const TfBufs& b, const HeadArgsHost& ha, cudaStream_t s) {
    HeadArgs a{};
    a.mode = ha.mode; a.la = ha.la; a.ph = ha.ph; a.xsample = ha.xsample; a.la_x = ha.la_x;
    a.ph_x = ha.ph_x; a.seg = ha.seg; a.seg_stride = ha.seg_stride; a.nseg = ha.nseg;
    a.row0 = ha.row0; a.S = ha.S; a.contrib = ha.contrib; a.p_out = ha.p_out; a.thr = ha.thr;
    a.trace = ha.trace;
    a.step_pos = ha.step_pos;
    return with_dpl(mc.hidden, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        if (b.fused_heads && a.mode != 2 && T == mc.n) {
            // the last MLP left the per-row logits and phase dots: constraint, log-sigmoid and ratio
            ProfScope ps("tf_heads", s, 0.0, (double)R * T * 4 + (double)R * 64 * 4);
            heads_reduce_kernel<<<blocks_for(R, 8), 256, 0, s>>>(mc, P, bits, b.logit, b.hph, R, a);
            NQS_LAUNCHED();
            return NQS_OK;
        }
        ProfScope ps("tf_heads", s, 0.0, (double)R * T * mc.hidden * 4);
        heads_kernel<DPL><<<blocks_for(R, 8), 256, 0, s>>>(mc, P, bits, b.h, R, T, a);
        NQS_LAUNCHED();
        return NQS_OK;
    });
}

int tf_segment_sum(const int64_t* seg, int64_t seg_stride, int64_t nseg, const float2* contrib,
                   int compensated, float* eloc, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>(nseg, (int64_t)num_sms() * 8);
    segment_sum_kernel<<<grid, 128, 0, s>>>(seg, seg_stride, nseg, contrib, compensated, eloc);
    NQS_LAUNCHED();
    return NQS_OK;
}

int tf_tok_tables(const ModelConst& mc, const float* P, const TfWeights& w, int T, float* tab_h, float* tab_qkv,
                  cudaStream_t s) {
    if (mc.hidden != 64 || mc.precision != NQS_PREC_BF16 || T < 1 || T > mc.n) {
        set_error("token-position tables: d_model 64 bf16 models only");
        return NQS_ERR_UNSUPPORTED;
    }
    const int ldw = mc.compensated ? 2 * mc.hidden : mc.hidden;
    ProfScope ps("tf_tok_table", s);
    tok_table_kernel<<<3 * T, 192, 0, s>>>(mc, P, reinterpret_cast<const __nv_bfloat16*>(w.bf16 + w.bf16_off[0][TF_WQKV]),
                                           ldw, T, tab_h, tab_qkv, mc.compensated ? 1 : 0);
    NQS_LAUNCHED();
    return NQS_OK;
}

int tf_logpsi(const ModelConst& mc, const float* P, const TfWeights& w, const uint64_t* bits,
              int64_t B, float* la, float* ph, TfBufs& b, cudaStream_t s) {
    for (int64_t lo = 0; lo < B; lo += b.R) {
        const int64_t R = std::min(b.R, B - lo);
        NQS_TRY(tf_forward(mc, P, w, bits + lo, R, mc.n, b, s, true));
        HeadArgsHost ha{};
        ha.mode = 0; ha.la = la + lo; ha.ph = ph + lo;
        NQS_TRY(tf_heads(mc, P, bits + lo, R, mc.n, b, ha, s));
    }
    return NQS_OK;
}

}  // namespace nqs
