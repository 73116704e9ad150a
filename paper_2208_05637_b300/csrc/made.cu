// Row-wise wavefunction models evaluated one configuration per thread in FP32 (paper
// Section 4): the MADE modulus sub-model with the two-layer phase MLP, and the product model.
//
//   log f(x) = i phi(x) + 1/2 sum_t log pihat_t(x_t | x_<t)          (Section 4, Architecture)
//
// Positions t follow the sampling order (position t holds qubit order[t]); inputs are spins
// +-1.  MADE connectivity (Germain et al.): input degree t+1, hidden degree (k mod (n-1)) + 1,
// hidden <- input iff deg_h >= t+1, hidden <- hidden iff deg >= deg, output t <- hidden iff
// deg_h < t+1.  The masks are multiplied into the shared-memory copy of the weights once per
// CTA, so the per-row loops are plain FMAs over float4 weight rows (broadcast reads).
// Hamming-weight constraint (Eq. modifier): at position t with spin s, c ones of spin s so far
// and r spin-s positions left after t, the bit is forced to 1 if c + r < n_s and to 0 if
// c >= n_s; forced positions contribute log 1 = 0 and a mismatch gives log|f| = -inf.
#include "nqs_internal.h"

namespace nqs {
namespace {

__device__ __forceinline__ float logsig(float v) { return fminf(v, 0.f) - log1pf(expf(-fabsf(v))); }

__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
}

// The configuration's bits in sampling order (bit t = x_{order[t]}), in the configuration's own
// width (one word for n <= 64, two for n <= 128).
template <class BT>
__device__ __forceinline__ BT to_positions(const BT& x, const ModelConst& mc, int upto) {
    BT xo = bits_zero<BT>();
    for (int t = 0; t < upto; ++t)
        if (qbit(x, mc.order[t])) xo = with_bit(xo, t);
    return xo;
}

// ------------------------------------------------------------------ shared-memory image
struct MadeLay {
    int W[MADE_MAX_LAYERS], b[MADE_MAX_LAYERS];
    int Wout, bout, P0, pb0, P1, pb1, total;
};

__host__ __device__ inline int r4(int v) { return (v + 3) & ~3; }

__host__ __device__ inline MadeLay made_layout(const ModelConst& mc, int H) {
    MadeLay L{};
    int o = 0;
    const int n = mc.n;
    L.W[0] = o; o += n * H;                    // W0^T [n][H], masked
    L.b[0] = o; o += H;
    for (int l = 1; l < mc.layers; ++l) {      // W_l [H][H], masked
        L.W[l] = o; o += H * H;
        L.b[l] = o; o += H;
    }
    L.Wout = o; o += n * H;                    // [n][H], masked
    L.bout = o; o += r4(n);
    L.P0 = o; o += (n - 2) * H;                // P0^T [n-2][H]
    L.pb0 = o; o += H;
    L.P1 = o; o += 4 * H;                      // [4][H]
    L.pb1 = o; o += 4;
    L.total = o;
    return L;
}

__host__ __device__ inline int made_deg(int k, int n) { return k % (n - 1) + 1; }

template <int H>
struct MadeRow {
    static size_t smem_bytes(const ModelConst& mc) { return (size_t)made_layout(mc, H).total * 4; }

    __device__ static void stage(float* sm, const float* __restrict__ P, const ModelConst& mc) {
        const MadeLay L = made_layout(mc, H);
        const int n = mc.n, hid = mc.hidden;
        for (int i = threadIdx.x; i < L.total; i += blockDim.x) sm[i] = 0.f;
        __syncthreads();
        for (int i = threadIdx.x; i < hid * n; i += blockDim.x) {
            const int k = i / n, t = i % n;
            if (t < made_deg(k, n)) sm[L.W[0] + t * H + k] = P[mc.made_W[0] + i];
        }
        for (int k = threadIdx.x; k < hid; k += blockDim.x) {
            sm[L.b[0] + k] = P[mc.made_b[0] + k];
            sm[L.pb0 + k] = P[mc.ph_b0 + k];
        }
        for (int l = 1; l < mc.layers; ++l) {
            for (int i = threadIdx.x; i < hid * hid; i += blockDim.x) {
                const int k = i / hid, kp = i % hid;
                if (made_deg(kp, n) <= made_deg(k, n)) sm[L.W[l] + k * H + kp] = P[mc.made_W[l] + i];
            }
            for (int k = threadIdx.x; k < hid; k += blockDim.x) sm[L.b[l] + k] = P[mc.made_b[l] + k];
        }
        for (int i = threadIdx.x; i < n * hid; i += blockDim.x) {
            const int t = i / hid, k = i % hid;
            if (made_deg(k, n) < t + 1) sm[L.Wout + t * H + k] = P[mc.made_Wout + i];
        }
        for (int t = threadIdx.x; t < n; t += blockDim.x) sm[L.bout + t] = P[mc.made_bout + t];
        for (int i = threadIdx.x; i < hid * (n - 2); i += blockDim.x) {
            const int k = i / (n - 2), t = i % (n - 2);
            sm[L.P0 + t * H + k] = P[mc.ph_W0 + i];
        }
        for (int i = threadIdx.x; i < 4 * hid; i += blockDim.x) {
            const int j = i / hid, k = i % hid;
            sm[L.P1 + j * H + k] = P[mc.ph_W1 + i];
        }
        for (int j = threadIdx.x; j < 4; j += blockDim.x) sm[L.pb1 + j] = P[mc.ph_b1 + j];
    }

    // h <- relu(first layer) for position bits xo
    template <class PB>
    __device__ static void first_layer(const float* sm, const MadeLay& L, const ModelConst& mc,
                                       const PB& xo, float (&h)[H]) {
        float z[H];
#pragma unroll
        for (int k = 0; k < H; ++k) z[k] = sm[L.b[0] + k];
        for (int t = 0; t < mc.n; ++t) {
            const float s = qbit(xo, t) ? 1.f : -1.f;
            const float4* w = reinterpret_cast<const float4*>(sm + L.W[0] + t * H);
#pragma unroll
            for (int k4 = 0; k4 < H / 4; ++k4) {
                const float4 v = w[k4];
                z[4 * k4 + 0] = fmaf(v.x, s, z[4 * k4 + 0]);
                z[4 * k4 + 1] = fmaf(v.y, s, z[4 * k4 + 1]);
                z[4 * k4 + 2] = fmaf(v.z, s, z[4 * k4 + 2]);
                z[4 * k4 + 3] = fmaf(v.w, s, z[4 * k4 + 3]);
            }
        }
#pragma unroll
        for (int k = 0; k < H; ++k) h[k] = fmaxf(z[k], 0.f);
    }

    // h <- last hidden layer of the modulus MADE for position bits xo
    template <class PB>
    __device__ static void hidden(const float* sm, const MadeLay& L, const ModelConst& mc,
                                  const PB& xo, float (&h)[H]) {
        first_layer(sm, L, mc, xo, h);
        float z[H];
        for (int l = 1; l < mc.layers; ++l) {
#pragma unroll
            for (int k = 0; k < H; ++k) {
                float a = sm[L.b[l] + k];
                const float4* w = reinterpret_cast<const float4*>(sm + L.W[l] + k * H);
#pragma unroll
                for (int k4 = 0; k4 < H / 4; ++k4) {
                    const float4 v = w[k4];
                    a = fmaf(v.x, h[4 * k4 + 0], a);
                    a = fmaf(v.y, h[4 * k4 + 1], a);
                    a = fmaf(v.z, h[4 * k4 + 2], a);
                    a = fmaf(v.w, h[4 * k4 + 3], a);
                }
                z[k] = a;
            }
#pragma unroll
            for (int k = 0; k < H; ++k) h[k] = fmaxf(z[k], 0.f);
        }
    }

    __device__ static float logit(const float* sm, const MadeLay& L, const float (&h)[H], int t) {
        float a = sm[L.bout + t];
        const float4* w = reinterpret_cast<const float4*>(sm + L.Wout + t * H);
#pragma unroll
        for (int k4 = 0; k4 < H / 4; ++k4) {
            const float4 v = w[k4];
            a = fmaf(v.x, h[4 * k4 + 0], a);
            a = fmaf(v.y, h[4 * k4 + 1], a);
            a = fmaf(v.z, h[4 * k4 + 2], a);
            a = fmaf(v.w, h[4 * k4 + 3], a);
        }
        return a;
    }

    // phase MLP output selected by the last two positions; hp receives the hidden layer
    template <class PB>
    __device__ static float phase(const float* sm, const MadeLay& L, const ModelConst& mc,
                                  const PB& xo, float (&hp)[H]) {
#pragma unroll
        for (int k = 0; k < H; ++k) hp[k] = sm[L.pb0 + k];
        for (int t = 0; t < mc.n - 2; ++t) {
            const float s = qbit(xo, t) ? 1.f : -1.f;
            const float4* w = reinterpret_cast<const float4*>(sm + L.P0 + t * H);
#pragma unroll
            for (int k4 = 0; k4 < H / 4; ++k4) {
                const float4 v = w[k4];
                hp[4 * k4 + 0] = fmaf(v.x, s, hp[4 * k4 + 0]);
                hp[4 * k4 + 1] = fmaf(v.y, s, hp[4 * k4 + 1]);
                hp[4 * k4 + 2] = fmaf(v.z, s, hp[4 * k4 + 2]);
                hp[4 * k4 + 3] = fmaf(v.w, s, hp[4 * k4 + 3]);
            }
        }
#pragma unroll
        for (int k = 0; k < H; ++k) hp[k] = fmaxf(hp[k], 0.f);
        const int sel = qbit(xo, mc.n - 2) * 2 + qbit(xo, mc.n - 1);
        float a = sm[L.pb1 + sel];
        const float4* w = reinterpret_cast<const float4*>(sm + L.P1 + sel * H);
#pragma unroll
        for (int k4 = 0; k4 < H / 4; ++k4) {
            const float4 v = w[k4];
            a = fmaf(v.x, hp[4 * k4 + 0], a);
            a = fmaf(v.y, hp[4 * k4 + 1], a);
            a = fmaf(v.z, hp[4 * k4 + 2], a);
            a = fmaf(v.w, hp[4 * k4 + 3], a);
        }
        return a;
    }

    template <class BT>
    __device__ static void logpsi(const float* sm, const ModelConst& mc, const BT& x, float& la,
                                  float& ph) {
        const MadeLay L = made_layout(mc, H);
        const BT xo = to_positions(x, mc, mc.n);
        float h[H];
        hidden(sm, L, mc, xo, h);
        float acc = 0.f, err = 0.f;
        int ones0 = 0, ones1 = 0;
        bool bad = false;
        for (int t = 0; t < mc.n; ++t) {
            const int sp = mc.order[t] & 1;
            const int b = qbit(xo, t);
            const int c = sp ? ones1 : ones0;
            const int need = sp ? mc.n_dn : mc.n_up;
            if (c + mc.after[t] < need) bad |= (b == 0);
            else if (c >= need) bad |= (b == 1);
            else {
                const float l = logit(sm, L, h, t);
                const float lp = logsig(b ? l : -l);
                if (mc.compensated) two_sum_acc(acc, err, lp); else acc += lp;
            }
            if (sp) ones1 += b; else ones0 += b;
        }
        la = bad ? -INFINITY : 0.5f * (acc + err);
        ph = phase(sm, L, mc, xo, h);
    }

    // unconstrained pi(x_{order[k]} = 1 | prefix) for prefix position bits xo (positions < k)
    template <class PB>
    __device__ static float p1(const float* sm, const ModelConst& mc, const PB& xo, int k) {
        const MadeLay L = made_layout(mc, H);
        float h[H];
        hidden(sm, L, mc, xo, h);
        const float l = logit(sm, L, h, k);
        return 1.f / (1.f + expf(-l));
    }
};

struct ProductRow {
    static size_t smem_bytes(const ModelConst& mc) { return (size_t)r4(mc.n) * 4; }
    __device__ static void stage(float* sm, const float* __restrict__ P, const ModelConst& mc) {
        for (int t = threadIdx.x; t < mc.n; t += blockDim.x) sm[t] = fminf(fmaxf(P[mc.p_prob + t], 0.f), 1.f);
    }
    template <class BT>
    __device__ static void logpsi(const float* sm, const ModelConst& mc, const BT& x, float& la,
                                  float& ph) {
        float acc = 0.f, err = 0.f;
        int ones0 = 0, ones1 = 0;
        bool bad = false;
        for (int t = 0; t < mc.n; ++t) {
            const int sp = mc.order[t] & 1;
            const int b = qbit(x, mc.order[t]);
            const int c = sp ? ones1 : ones0;
            const int need = sp ? mc.n_dn : mc.n_up;
            if (c + mc.after[t] < need) bad |= (b == 0);
            else if (c >= need) bad |= (b == 1);
            else {
                const float lp = b ? logf(sm[t]) : log1pf(-sm[t]);
                if (mc.compensated) two_sum_acc(acc, err, lp); else acc += lp;
            }
            if (sp) ones1 += b; else ones0 += b;
        }
        la = bad ? -INFINITY : 0.5f * (acc + err);
        ph = 0.f;
    }
    template <class PB>
    __device__ static float p1(const float* sm, const ModelConst&, const PB&, int k) { return sm[k]; }
};

// ------------------------------------------------------------------ kernels
template <class R, class BT>
__global__ void __launch_bounds__(128)
logpsi_rows_kernel(ModelConst mc, const float* __restrict__ P, const BT* __restrict__ bits,
                   int64_t B, float* __restrict__ la, float* __restrict__ ph) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    R::stage(sm, P, mc);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B;
         i += (int64_t)gridDim.x * blockDim.x) {
        float a, p;
        R::logpsi(sm, mc, bits[i], a, p);
        la[i] = a;
        ph[i] = p;
    }
}

// One CTA per sample: evaluate the model on every connected x' of the sample and reduce
//   E_loc(x) = sum_r S_r exp(log|f(x'_r)| - log|f(x)|) e^{i (phi(x'_r) - phi(x))}
// with the ratio-weighted (optionally TwoSum-compensated) complex reduction fused in.
template <class R, class BT>
__global__ void __launch_bounds__(128)
eloc_rows_kernel(ModelConst mc, const float* __restrict__ P, const BT* __restrict__ bits,
                 int64_t B, const float* __restrict__ la_x, const float* __restrict__ ph_x,
                 const int64_t* __restrict__ off, int64_t ntiles,
                 const BT* __restrict__ xprime, const float4* __restrict__ S,
                 float* __restrict__ eloc) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    __shared__ float red[4][128];
    R::stage(sm, P, mc);
    __syncthreads();
    for (int64_t i = blockIdx.x; i < B; i += gridDim.x) {
        const int64_t r0 = off[i * ntiles], r1 = off[(i + 1) * ntiles];
        const BT x = bits[i];
        const float lai = la_x[i], phi = ph_x[i];
        float re = 0.f, re_e = 0.f, im = 0.f, im_e = 0.f;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
            const BT xp = xprime[r];
            const float4 s = S[r];
            const float sre = s.x + s.y, sim = s.z + s.w;
            float cr = sre, ci = sim;
            if (xp != x) {
                float la2, ph2;
                R::logpsi(sm, mc, xp, la2, ph2);
                const float mag = expf(la2 - lai);
                float sn, cs;
                sincosf(ph2 - phi, &sn, &cs);
                const float rr = mag * cs, ri = mag * sn;
                cr = sre * rr - sim * ri;
                ci = sre * ri + sim * rr;
            }
            if (mc.compensated) { two_sum_acc(re, re_e, cr); two_sum_acc(im, im_e, ci); }
            else { re += cr; im += ci; }
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

// Sampler conditional at step k for each parent prefix: constrained pihat, its 2^32 threshold,
// and a reset of the per-parent ones counter.
template <class R, class BT>
__global__ void __launch_bounds__(128)
cond_rows_kernel(ModelConst mc, const float* __restrict__ P, int k,
                 const BT* __restrict__ bits, const int64_t* __restrict__ Udev,
                 float* __restrict__ p_out, uint64_t* __restrict__ thr, float* __restrict__ trace) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    R::stage(sm, P, mc);
    __syncthreads();
    const int64_t U = *Udev;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < U;
         s += (int64_t)gridDim.x * blockDim.x) {
        const BT xo = to_positions(bits[s], mc, k);
        int ones0 = 0, ones1 = 0;
        for (int t = 0; t < k; ++t) {
            const int b = qbit(xo, t);
            if (mc.order[t] & 1) ones1 += b; else ones0 += b;
        }
        const int sp = mc.order[k] & 1;
        const int c = sp ? ones1 : ones0;
        const int need = sp ? mc.n_dn : mc.n_up;
        float p;
        if (c + mc.after[k] < need) p = 1.f;
        else if (c >= need) p = 0.f;
        else p = R::p1(sm, mc, xo, k);
        p_out[s] = p;
        thr[s] = (uint64_t)(p * 4294967296.0f);   // exact: scaling by 2^32, then floor
        if (trace) trace[s] = p;
    }
}

// ------------------------------------------------------------------ MADE backward
struct ActLay {
    int u, h0, hp, dout, dz0, dpo, dzp, ld;
};

__host__ __device__ inline ActLay act_layout(const ModelConst& mc) {
    ActLay a{};
    const int n = mc.n, hid = mc.hidden, L = mc.layers;
    a.u = 0;
    a.h0 = n;                       // h_l at h0 + l*hid
    a.hp = n + L * hid;
    a.dout = a.hp + hid;
    a.dz0 = a.dout + n;             // dz_l at dz0 + l*hid
    a.dpo = a.dz0 + L * hid;
    a.dzp = a.dpo + 4;
    a.ld = r4(a.dzp + hid);
    return a;
}

template <int H, class BT>
__global__ void __launch_bounds__(128)
made_backward_kernel(ModelConst mc, const float* __restrict__ P, const BT* __restrict__ bits,
                     int64_t B, const float* __restrict__ g_abs, const float* __restrict__ g_phase,
                     float* __restrict__ acts, int64_t ld) {
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    MadeRow<H>::stage(sm, P, mc);
    __syncthreads();
    const MadeLay L = made_layout(mc, H);
    const ActLay A = act_layout(mc);
    const int n = mc.n, hid = mc.hidden;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B;
         i += (int64_t)gridDim.x * blockDim.x) {
        float* row = acts + i * ld;
        const BT xo = to_positions(bits[i], mc, n);
        for (int t = 0; t < n; ++t) row[A.u + t] = qbit(xo, t) ? 1.f : -1.f;
        // forward, storing every hidden layer (outer loops over units stay rolled; the
        // inner loops over the previous layer are unrolled against register arrays)
        float h[H];
        MadeRow<H>::first_layer(sm, L, mc, xo, h);
#pragma unroll
        for (int k = 0; k < H; ++k)
            if (k < hid) row[A.h0 + k] = h[k];
        for (int l = 1; l < mc.layers; ++l) {
            for (int k = 0; k < hid; ++k) {
                float a = sm[L.b[l] + k];
                const float4* w = reinterpret_cast<const float4*>(sm + L.W[l] + k * H);
#pragma unroll
                for (int k4 = 0; k4 < H / 4; ++k4) {
                    const float4 v = w[k4];
                    a = fmaf(v.x, h[4 * k4 + 0], a);
                    a = fmaf(v.y, h[4 * k4 + 1], a);
                    a = fmaf(v.z, h[4 * k4 + 2], a);
                    a = fmaf(v.w, h[4 * k4 + 3], a);
                }
                row[A.h0 + l * hid + k] = fmaxf(a, 0.f);
            }
#pragma unroll
            for (int k = 0; k < H; ++k) h[k] = k < hid ? row[A.h0 + l * hid + k] : 0.f;
        }
        // output deltas d(g_abs * log|f|)/d logit_t = g_abs/2 (x_t - sigmoid(l_t)) on free t
        const float ga = g_abs[i];
        float dh[H];
#pragma unroll
        for (int k = 0; k < H; ++k) dh[k] = 0.f;
        int ones0 = 0, ones1 = 0;
        for (int t = 0; t < n; ++t) {
            const int sp = mc.order[t] & 1;
            const int b = qbit(xo, t);
            const int c = sp ? ones1 : ones0;
            const int need = sp ? mc.n_dn : mc.n_up;
            float d = 0.f;
            if (!(c + mc.after[t] < need) && !(c >= need)) {
                const float l = MadeRow<H>::logit(sm, L, h, t);
                d = 0.5f * ga * ((float)b - 1.f / (1.f + expf(-l)));
            }
            row[A.dout + t] = d;
            const float4* wo = reinterpret_cast<const float4*>(sm + L.Wout + t * H);
#pragma unroll
            for (int k4 = 0; k4 < H / 4; ++k4) {
                const float4 v = wo[k4];
                dh[4 * k4 + 0] = fmaf(d, v.x, dh[4 * k4 + 0]);
                dh[4 * k4 + 1] = fmaf(d, v.y, dh[4 * k4 + 1]);
                dh[4 * k4 + 2] = fmaf(d, v.z, dh[4 * k4 + 2]);
                dh[4 * k4 + 3] = fmaf(d, v.w, dh[4 * k4 + 3]);
            }
            if (sp) ones1 += b; else ones0 += b;
        }
        // back through the hidden stack
        const int Lh = mc.layers;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            dh[k] = h[k] > 0.f ? dh[k] : 0.f;
            if (k < hid) row[A.dz0 + (Lh - 1) * hid + k] = dh[k];
        }
        for (int l = Lh - 1; l >= 1; --l) {
            float dp[H];
#pragma unroll
            for (int kp = 0; kp < H; ++kp) dp[kp] = 0.f;
            for (int k = 0; k < hid; ++k) {
                const float d = row[A.dz0 + l * hid + k];
                const float4* w = reinterpret_cast<const float4*>(sm + L.W[l] + k * H);
#pragma unroll
                for (int k4 = 0; k4 < H / 4; ++k4) {
                    const float4 v = w[k4];
                    dp[4 * k4 + 0] = fmaf(d, v.x, dp[4 * k4 + 0]);
                    dp[4 * k4 + 1] = fmaf(d, v.y, dp[4 * k4 + 1]);
                    dp[4 * k4 + 2] = fmaf(d, v.z, dp[4 * k4 + 2]);
                    dp[4 * k4 + 3] = fmaf(d, v.w, dp[4 * k4 + 3]);
                }
            }
#pragma unroll
            for (int kp = 0; kp < H; ++kp) {
                if (kp < hid) {
                    const float hv = row[A.h0 + (l - 1) * hid + kp];
                    row[A.dz0 + (l - 1) * hid + kp] = hv > 0.f ? dp[kp] : 0.f;
                }
            }
        }
        // phase sub-model
        const float gp = g_phase[i];
        float hp[H];
        MadeRow<H>::phase(sm, L, mc, xo, hp);
        const int sel = qbit(xo, n - 2) * 2 + qbit(xo, n - 1);
        for (int j = 0; j < 4; ++j) row[A.dpo + j] = j == sel ? gp : 0.f;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            if (k < hid) {
                row[A.hp + k] = hp[k];
                row[A.dzp + k] = hp[k] > 0.f ? gp * sm[L.P1 + sel * H + k] : 0.f;
            }
        }
    }
}

template <class BT>
__global__ void product_backward_kernel(ModelConst mc, const float* __restrict__ P,
                                        const BT* __restrict__ bits, int64_t B,
                                        const float* __restrict__ g_abs, float* __restrict__ grad) {
    __shared__ float red[256];
    const int t = blockIdx.x;   // position
    const float p = fminf(fmaxf(P[mc.p_prob + t], 0.f), 1.f);
    const int sp = mc.order[t] & 1;
    const int need = sp ? mc.n_dn : mc.n_up;
    float acc = 0.f;
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
        const BT x = bits[i];
        int c = 0;
        for (int u = 0; u < t; ++u)
            if ((mc.order[u] & 1) == sp) c += qbit(x, mc.order[u]);
        if (!(c + mc.after[t] < need) && !(c >= need)) {
            const int b = qbit(x, mc.order[t]);
            acc += 0.5f * g_abs[i] * (b ? 1.f / p : -1.f / (1.f - p));
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[mc.p_prob + t] += red[0];
}

// ------------------------------------------------------------------ dispatch helpers
template <class K>
int prep_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    }
    return NQS_OK;
}

template <class F>
int with_row_model(const ModelConst& mc, F&& f) {
    if (mc.arch == NQS_ARCH_PRODUCT) return f(ProductRow{});
    if (mc.arch == NQS_ARCH_MADE) {
        if (mc.hidden <= 16) return f(MadeRow<16>{});
        return f(MadeRow<64>{});
    }
    set_error("row-wise kernels serve the product and MADE models only");
    return NQS_ERR_UNSUPPORTED;
}

inline int grid_for(int64_t work, int per) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + per - 1) / per, (int64_t)num_sms() * 16));
}

}  // namespace

int launch_logpsi_rows(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                       float* la, float* ph, cudaStream_t s) {
    return with_row_model(mc, [&](auto row) -> int {
        using R = decltype(row);
        const size_t sm = R::smem_bytes(mc);
        ProfScope ps("logpsi_rows", s);
        if (words_of(mc.n) == 2) {
            NQS_TRY(prep_smem(logpsi_rows_kernel<R, U128>, sm));
            logpsi_rows_kernel<R, U128><<<grid_for(B, 128), 128, sm, s>>>(mc, P, reinterpret_cast<const U128*>(bits),
                                                                           B, la, ph);
        } else {
            NQS_TRY(prep_smem(logpsi_rows_kernel<R, uint64_t>, sm));
            logpsi_rows_kernel<R, uint64_t><<<grid_for(B, 128), 128, sm, s>>>(mc, P, bits, B, la, ph);
        }
        NQS_LAUNCHED();
        return NQS_OK;
    });
}

int launch_eloc_rows(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                     const float* la_x, const float* ph_x, const int64_t* off, int64_t ntiles,
                     const uint64_t* xprime, const float4* S, float* eloc, cudaStream_t s) {
    return with_row_model(mc, [&](auto row) -> int {
        using R = decltype(row);
        const size_t sm = R::smem_bytes(mc);
        const int grid = (int)std::min<int64_t>(B, (int64_t)num_sms() * 8);
        if (words_of(mc.n) == 2) {
            NQS_TRY(prep_smem(eloc_rows_kernel<R, U128>, sm));
            eloc_rows_kernel<R, U128><<<grid, 128, sm, s>>>(mc, P, reinterpret_cast<const U128*>(bits), B, la_x, ph_x,
                                                            off, ntiles, reinterpret_cast<const U128*>(xprime), S, eloc);
        } else {
            NQS_TRY(prep_smem(eloc_rows_kernel<R, uint64_t>, sm));
            eloc_rows_kernel<R, uint64_t><<<grid, 128, sm, s>>>(mc, P, bits, B, la_x, ph_x, off, ntiles, xprime, S, eloc);
        }
        NQS_LAUNCHED();
        return NQS_OK;
    });
}

int launch_cond_rows(const ModelConst& mc, const float* P, int k, const uint64_t* bits,
                     const int64_t* U, int64_t cap, float* p_out, uint64_t* thr, float* trace,
                     cudaStream_t s) {
    return with_row_model(mc, [&](auto row) -> int {
        using R = decltype(row);
        const size_t sm = R::smem_bytes(mc);
        if (words_of(mc.n) == 2) {
            NQS_TRY(prep_smem(cond_rows_kernel<R, U128>, sm));
            cond_rows_kernel<R, U128><<<grid_for(cap, 128), 128, sm, s>>>(mc, P, k, reinterpret_cast<const U128*>(bits), U,
                                                                           p_out, thr, trace);
        } else {
            NQS_TRY(prep_smem(cond_rows_kernel<R, uint64_t>, sm));
            cond_rows_kernel<R, uint64_t><<<grid_for(cap, 128), 128, sm, s>>>(mc, P, k, bits, U, p_out, thr, trace);
        }
        NQS_LAUNCHED();
        return NQS_OK;
    });
}

int64_t made_act_stride(const ModelConst& mc) { return act_layout(mc).ld; }

int launch_made_backward(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                         const float* g_abs, const float* g_phase, float* acts, int64_t ld,
                         cudaStream_t s) {
    auto go = [&](auto kernel, auto b, size_t sm) -> int {
        NQS_TRY(prep_smem(kernel, sm));
        kernel<<<grid_for(B, 128), 128, sm, s>>>(mc, P, b, B, g_abs, g_phase, acts, ld);
        NQS_LAUNCHED();
        return NQS_OK;
    };
    const U128* b2 = reinterpret_cast<const U128*>(bits);
    if (words_of(mc.n) == 2) {
        if (mc.hidden <= 16) return go(made_backward_kernel<16, U128>, b2, MadeRow<16>::smem_bytes(mc));
        return go(made_backward_kernel<64, U128>, b2, MadeRow<64>::smem_bytes(mc));
    }
    if (mc.hidden <= 16) return go(made_backward_kernel<16, uint64_t>, bits, MadeRow<16>::smem_bytes(mc));
    return go(made_backward_kernel<64, uint64_t>, bits, MadeRow<64>::smem_bytes(mc));
}

int made_grad_reduce(const ModelConst& mc, const float* acts, int64_t ld, int64_t B, float* grad,
                     cudaStream_t s) {
    const ActLay A = act_layout(mc);
    const int n = mc.n, hid = mc.hidden, L = mc.layers;
    NQS_TRY(launch_outer_grad(acts + A.dout, ld, acts + A.h0 + (L - 1) * hid, ld, B, n, hid, 3, n,
                              grad + mc.made_Wout, grad + mc.made_bout, s));
    for (int l = L - 1; l >= 1; --l)
        NQS_TRY(launch_outer_grad(acts + A.dz0 + l * hid, ld, acts + A.h0 + (l - 1) * hid, ld, B,
                                  hid, hid, 2, n, grad + mc.made_W[l], grad + mc.made_b[l], s));
    NQS_TRY(launch_outer_grad(acts + A.dz0, ld, acts + A.u, ld, B, hid, n, 1, n,
                              grad + mc.made_W[0], grad + mc.made_b[0], s));
    NQS_TRY(launch_outer_grad(acts + A.dpo, ld, acts + A.hp, ld, B, 4, hid, 0, n,
                              grad + mc.ph_W1, grad + mc.ph_b1, s));
    NQS_TRY(launch_outer_grad(acts + A.dzp, ld, acts + A.u, ld, B, hid, n - 2, 0, n,
                              grad + mc.ph_W0, grad + mc.ph_b0, s));
    return NQS_OK;
}

int launch_product_backward(const ModelConst& mc, const float* P, const uint64_t* bits,
                            int64_t B, const float* g_abs, float* grad, cudaStream_t s) {
    ProfScope ps("product_backward", s);
    if (words_of(mc.n) == 2)
        product_backward_kernel<U128><<<mc.n, 256, 0, s>>>(mc, P, reinterpret_cast<const U128*>(bits), B, g_abs, grad);
    else
        product_backward_kernel<uint64_t><<<mc.n, 256, 0, s>>>(mc, P, bits, B, g_abs, grad);
    NQS_LAUNCHED();
    return NQS_OK;
}

}  // namespace nqs
