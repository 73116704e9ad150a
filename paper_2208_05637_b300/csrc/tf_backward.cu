// Hand-written backward of the transformer wavefunction (paper Eq. grad, via the surrogate
// sum_i g_abs_i log|f(x_i)| + g_phase_i phi(x_i)), with the forward recomputed inside
// (activation recomputation) in chunks of R sequences.  FP32 on CUDA cores; for BF16 models
// the recomputed forward uses the same bf16-rounded weights and GEMM input activations as the
// tensor-core forward, and the backward treats the rounding as identity (straight-through).
//
// Per chunk: forward with every block's activations saved; heads + final LayerNorm backward;
// then for each block, last to first: MLP (W2, GELU, W1, LN2) and attention (Wo, softmax
// attention, Wqkv, LN1) backward; finally the embeddings.  Weight gradients are reductions
// over all rows of the chunk, done in fixed order (split-K partials reduced in order), so
// results are bit-reproducible run to run.
#include <memory>

#include "tf_common.cuh"

#include <mutex>

namespace nqs {
namespace {

__device__ __forceinline__ float gelu_grad(float x) {
    const float k = 0.7978845608028654f;
    const float u = k * (x + 0.044715f * x * x * x);
    const float th = tanhf(u);
    return 0.5f * (1.f + th) + 0.5f * x * (1.f - th * th) * k * (1.f + 3.f * 0.044715f * x * x);
}


__global__ void embed_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
                             int64_t R, int T, float* __restrict__ h) {
    const int d = mc.hidden;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < R * T * d;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / d;
        const int j = (int)(i % d);
        const int64_t r = row / T;
        const int t = (int)(row % T);
        const int tok = t == 0 ? 2 : (int)((bits[r] >> mc.order[t - 1]) & 1ull);
        h[i] = P[mc.tok_emb + tok * d + j] + P[mc.pos_emb + t * d + j];
    }
}

template <int MODE>
__global__ void gelu_fwd_kernel(const float* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        store_mode<MODE>(y + i, 0, 1, 0, gelu_tanh(x[i]));
}

__global__ void gelu_bwd_kernel(const float* __restrict__ x, float* __restrict__ g, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] *= gelu_grad(x[i]);
}

// LayerNorm backward, one warp per row: out = res + dLN/dx (x, g; dy), and gx = dy * xhat for
// the gain gradient.
template <int DPL>
__global__ void __launch_bounds__(256)
ln_bwd_kernel(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ dy,
              const float* __restrict__ res, float* __restrict__ out, float* __restrict__ gx,
              int64_t M, int d) {
    const int lane = threadIdx.x & 31;
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= M) return;
    float v[DPL], dyv[DPL];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) { v[i] = x[row * d + lane + 32 * i]; s += v[i]; }
    const float mu = warp_sum(s) * (1.f / (float)d);
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) { v[i] -= mu; q += v[i] * v[i]; }
    const float rstd = rsqrtf(fmaf(warp_sum(q), 1.f / (float)d, LN_EPS));
    float m1 = 0.f, m2 = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        v[i] *= rstd;                                   // xhat
        dyv[i] = dy[row * d + j];
        const float dx = dyv[i] * g[j];
        m1 += dx;
        m2 += dx * v[i];
    }
    m1 = warp_sum(m1) * (1.f / (float)d);
    m2 = warp_sum(m2) * (1.f / (float)d);
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        const float dx = dyv[i] * g[j];
        out[row * d + j] = res[row * d + j] + rstd * (dx - m1 - v[i] * m2);
        gx[row * d + j] = dyv[i] * v[i];
    }
}

// Heads + final LayerNorm backward, one warp per (sequence, position).  Writes dh (gradient wrt the final
// residual stream), dy rows and dy*xhat rows of LNf, the LNf outputs hf, the logit deltas dl
// and the one-hot phase deltas dph.
template <int DPL>
__global__ void __launch_bounds__(256)
heads_bwd_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ bits,
                 const float* __restrict__ h, int64_t R, const float* __restrict__ g_abs,
                 const float* __restrict__ g_phase, float* __restrict__ dh, float* __restrict__ dyo,
                 float* __restrict__ gx, float* __restrict__ hf, float* __restrict__ dl,
                 float* __restrict__ dph) {
    const int d = mc.hidden, n = mc.n;
    const int lane = threadIdx.x & 31;
    // one warp per (sequence, position) row: the rows run in parallel, the constraint's counts of
    // earlier same-spin ones come from the configuration directly
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= R * n) return;
    const int64_t r = row / n;
    const int t = (int)(row - r * n);
    const uint64_t x = bits[r];
    const float ga = g_abs[r], gp = g_phase[r];
    const int sel = (int)(((x >> mc.order[n - 2]) & 1ull) * 2 + ((x >> mc.order[n - 1]) & 1ull));
    if (t == 0 && lane < 4) dph[r * 4 + lane] = lane == sel ? gp : 0.f;
    {
        const int sp = mc.order[t] & 1;
        const int b = (int)((x >> mc.order[t]) & 1ull);
        int c = 0;
        for (int u = 0; u < t; ++u)
            if ((mc.order[u] & 1) == sp) c += (int)((x >> mc.order[u]) & 1ull);
        const int need = sp ? mc.n_dn : mc.n_up;
        const bool free_t = !(c + mc.after[t] < need) && !(c >= need);
        float v[DPL];
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) { v[i] = h[row * d + lane + 32 * i]; s += v[i]; }
        const float mu = warp_sum(s) * (1.f / (float)d);
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) { v[i] -= mu; q += v[i] * v[i]; }
        const float rstd = rsqrtf(fmaf(warp_sum(q), 1.f / (float)d, LN_EPS));
        float y[DPL];
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
            const int j = lane + 32 * i;
            v[i] *= rstd;
            y[i] = v[i] * P[mc.lnf_g + j] + P[mc.lnf_b + j];
            hf[row * d + j] = y[i];
            a = fmaf(y[i], P[mc.head_w + j], a);
        }
        a = warp_sum(a) + P[mc.head_b + t];
        const float delta = free_t ? 0.5f * ga * ((float)b - 1.f / (1.f + expf(-a))) : 0.f;
        if (lane == 0) dl[row] = delta;
        float dyv[DPL];
        float m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
            const int j = lane + 32 * i;
            dyv[i] = delta * P[mc.head_w + j] + (t == n - 2 ? gp * P[mc.phase_w + sel * d + j] : 0.f);
            const float dx = dyv[i] * P[mc.lnf_g + j];
            m1 += dx;
            m2 += dx * v[i];
        }
        m1 = warp_sum(m1) * (1.f / (float)d);
        m2 = warp_sum(m2) * (1.f / (float)d);
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
            const int j = lane + 32 * i;
            const float dx = dyv[i] * P[mc.lnf_g + j];
            dh[row * d + j] = rstd * (dx - m1 - v[i] * m2);
            dyo[row * d + j] = dyv[i];
            gx[row * d + j] = dyv[i] * v[i];
        }
    }
}

// Attention backward per (sequence, head), dynamic shared memory; DH = head size.  Threads map
// to (row, column) pairs by shifts and strided loops (no divisions in the loops).
template <int DH>
__global__ void __launch_bounds__(128)
attention_bwd_kernel(const float* __restrict__ qkv, const float* __restrict__ dout, int T, int d,
                     float* __restrict__ dqkv) {
    extern __shared__ float sm[];
    constexpr int LD = DH + 1;
    const int lp = T + 1;
    float* q = sm;
    float* k = q + T * LD;
    float* v = k + T * LD;
    float* go = v + T * LD;
    float* p = go + T * LD;
    float* dp = p + T * lp;
    const int64_t r = blockIdx.x;
    const int hd = blockIdx.y;
    const float scale = rsqrtf((float)DH);
    for (int i = threadIdx.x; i < T * DH; i += blockDim.x) {
        const int t = i / DH, j = i % DH;              // DH is a power of two: shifts
        const float* row = qkv + (r * T + t) * (int64_t)(3 * d);
        q[t * LD + j] = row[hd * DH + j];
        k[t * LD + j] = row[d + hd * DH + j];
        v[t * LD + j] = row[2 * d + hd * DH + j];
        go[t * LD + j] = dout[(r * T + t) * (int64_t)d + hd * DH + j];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // scores and dP: warp w takes rows t = w, w + nw, ...; lane the keys u = lane, lane + 32, ...
    for (int t = warp; t < T; t += nw) {
        float qt[DH], gt[DH];
#pragma unroll
        for (int j = 0; j < DH; ++j) { qt[j] = q[t * LD + j]; gt[j] = go[t * LD + j]; }
        for (int u = lane; u < T; u += 32) {
            float sc = -INFINITY, g = 0.f;
            if (u <= t) {
                sc = 0.f;
#pragma unroll
                for (int j = 0; j < DH; ++j) { sc = fmaf(qt[j], k[u * LD + j], sc); g = fmaf(gt[j], v[u * LD + j], g); }
                sc *= scale;
            }
            p[t * lp + u] = sc;
            dp[t * lp + u] = g;
        }
    }
    __syncwarp();
    for (int t = warp; t < T; t += nw) {
        float mx = -INFINITY;
        for (int u = lane; u <= t; u += 32) mx = fmaxf(mx, p[t * lp + u]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        float s = 0.f;
        for (int u = lane; u <= t; u += 32) { const float e = expf(p[t * lp + u] - mx); p[t * lp + u] = e; s += e; }
        s = warp_sum(s);
        const float inv = 1.f / s;
        float pd = 0.f;
        for (int u = lane; u <= t; u += 32) { p[t * lp + u] *= inv; pd += p[t * lp + u] * dp[t * lp + u]; }
        pd = warp_sum(pd);
        for (int u = lane; u <= t; u += 32) dp[t * lp + u] = p[t * lp + u] * (dp[t * lp + u] - pd);   // dS
        for (int u = t + 1 + lane; u < T; u += 32) { p[t * lp + u] = 0.f; dp[t * lp + u] = 0.f; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * DH; i += blockDim.x) {
        const int t = i / DH, j = i % DH;
        float dq = 0.f, dk = 0.f, dv = 0.f;
        // causal: dS[t][u] and P[t][u] vanish for u > t
        for (int u = 0; u <= t; ++u) dq = fmaf(dp[t * lp + u], k[u * LD + j], dq);   // dS[t][u] k[u]
        for (int u = t; u < T; ++u) {
            dk = fmaf(dp[u * lp + t], q[u * LD + j], dk);      // dS[u][t] q[u]
            dv = fmaf(p[u * lp + t], go[u * LD + j], dv);      // P[u][t] dO[u]
        }
        float* row = dqkv + (r * T + t) * (int64_t)(3 * d);
        row[hd * DH + j] = dq * scale;
        row[d + hd * DH + j] = dk * scale;
        row[2 * d + hd * DH + j] = dv;
    }
}

// Head sizes other than the template's.
__global__ void __launch_bounds__(128)
attention_bwd_any_kernel(const float* __restrict__ qkv, const float* __restrict__ dout, int T, int d,
                         int dh, float* __restrict__ dqkv) {
    extern __shared__ float sm[];
    const int ld = dh + 1, lp = T + 1;
    float* q = sm;
    float* k = q + T * ld;
    float* v = k + T * ld;
    float* go = v + T * ld;
    float* p = go + T * ld;
    float* dp = p + T * lp;
    const int64_t r = blockIdx.x;
    const int hd = blockIdx.y;
    const float scale = rsqrtf((float)dh);
    for (int i = threadIdx.x; i < T * dh; i += blockDim.x) {
        const int t = i / dh, j = i % dh;
        const float* row = qkv + (r * T + t) * (int64_t)(3 * d);
        q[t * ld + j] = row[hd * dh + j];
        k[t * ld + j] = row[d + hd * dh + j];
        v[t * ld + j] = row[2 * d + hd * dh + j];
        go[t * ld + j] = dout[(r * T + t) * (int64_t)d + hd * dh + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
        const int t = i / T, u = i % T;
        float s = -INFINITY, g = 0.f;
        if (u <= t) {
            s = 0.f;
            for (int j = 0; j < dh; ++j) { s = fmaf(q[t * ld + j], k[u * ld + j], s); g = fmaf(go[t * ld + j], v[u * ld + j], g); }
            s *= scale;
        }
        p[t * lp + u] = s;
        dp[t * lp + u] = g;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = warp; t < T; t += blockDim.x >> 5) {
        float mx = -INFINITY;
        for (int u = lane; u <= t; u += 32) mx = fmaxf(mx, p[t * lp + u]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        float s = 0.f;
        for (int u = lane; u <= t; u += 32) { const float e = expf(p[t * lp + u] - mx); p[t * lp + u] = e; s += e; }
        s = warp_sum(s);
        const float inv = 1.f / s;
        float pd = 0.f;
        for (int u = lane; u <= t; u += 32) { p[t * lp + u] *= inv; pd += p[t * lp + u] * dp[t * lp + u]; }
        pd = warp_sum(pd);
        for (int u = lane; u <= t; u += 32) dp[t * lp + u] = p[t * lp + u] * (dp[t * lp + u] - pd);   // dS
        for (int u = t + 1 + lane; u < T; u += 32) { p[t * lp + u] = 0.f; dp[t * lp + u] = 0.f; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * dh; i += blockDim.x) {
        const int t = i / dh, j = i % dh;
        float dq = 0.f, dk = 0.f, dv = 0.f;
        for (int u = 0; u < T; ++u) {
            dq = fmaf(dp[t * lp + u], k[u * ld + j], dq);
            dk = fmaf(dp[u * lp + t], q[u * ld + j], dk);
            dv = fmaf(p[u * lp + t], go[u * ld + j], dv);
        }
        float* row = dqkv + (r * T + t) * (int64_t)(3 * d);
        row[hd * dh + j] = dq * scale;
        row[d + hd * dh + j] = dk * scale;
        row[2 * d + hd * dh + j] = dv;
    }
}

// ---------------------------------------------------------------- deterministic reductions
// Column sums of one or two matrices X0, X1 (same shape; blockIdx.z picks one): stage 1 sums
// chunks of CS_ROWS rows per column, stage 2 adds the chunk sums in chunk order.
constexpr int CS_ROWS = 128;
__global__ void colsum_partial_kernel(const float* __restrict__ X0, const float* __restrict__ X1, int64_t ld,
                                      int64_t M, int ncols, float* __restrict__ part) {
    __shared__ float red[8][33];
    const float* X = blockIdx.z ? X1 : X0;
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * CS_ROWS;
    float s = 0.f;
    if (c < ncols)
        for (int64_t r = r0 + threadIdx.y; r < min(M, r0 + CS_ROWS); r += 8) s += X[r * ld + c];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < ncols) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
        part[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * ncols + c] = t;
    }
}

// Stage 2: one warp per (matrix, column); lane l adds chunks l, l + 32, ... in order, then a
// fixed shuffle tree (deterministic).
__global__ void colsum_final_kernel(const float* __restrict__ part, int nchunks, int ncols, int nmat,
                                    float* __restrict__ out0, float* __restrict__ out1) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= nmat * ncols) return;
    const int z = e / ncols, c = e % ncols;
    float s = 0.f;
    for (int i = lane; i < nchunks; i += 32) s += part[((int64_t)z * nchunks + i) * ncols + c];
    s = warp_sum(s);
    if (lane == 0) (z ? out1 : out0)[c] += s;
}

// Weight (and bias) gradients of a dense layer, split over row ranges: partial z holds
//   dW[o][i] = sum_b delta[b][o] act[b][i]   and   db[o] = sum_b delta[b][o]
// over rows b of its range, at part + z * (out_dim * in_dim + out_dim) (weights, then bias).
// 64 x 64 output tiles, 16 rows per shared-memory stage (the next stage is fetched into
// registers while the current one is used), 4 x 4 outputs per thread.
constexpr int OP_B = 64, OP_K = 16;
__global__ void __launch_bounds__(256)
outer_partial_kernel(const float* __restrict__ delta, int64_t ld_d, const float* __restrict__ act,
                     int64_t ld_a, int64_t M, int out_dim, int in_dim, int64_t rows_per_split,
                     float* __restrict__ part) {
    __shared__ __align__(16) float sd[2][OP_K][OP_B + 4];
    __shared__ __align__(16) float sa[2][OP_K][OP_B + 4];
    const int o0 = blockIdx.y * OP_B, i0 = blockIdx.x * OP_B;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t b_lo = (int64_t)blockIdx.z * rows_per_split;
    const int64_t b_hi = min(M, b_lo + rows_per_split);
    // fetch roles: rows (tid >> 6) + 4 q, column tid & 63
    const int fr = tid >> 6, fc = tid & 63;
    float rd[4], ra[4];
    auto fetch = [&](int64_t b0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t b = b0 + fr + 4 * q;
            rd[q] = (b < b_hi && o0 + fc < out_dim) ? delta[b * ld_d + o0 + fc] : 0.f;
            ra[q] = (b < b_hi && i0 + fc < in_dim) ? act[b * ld_a + i0 + fc] : 0.f;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sd[buf][fr + 4 * q][fc] = rd[q];
            sa[buf][fr + 4 * q][fc] = ra[q];
        }
    };
    float acc[4][4] = {};
    float accb[4] = {0.f, 0.f, 0.f, 0.f};
    fetch(b_lo);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int64_t b0 = b_lo; b0 < b_hi; b0 += OP_K) {
        const bool more = b0 + OP_K < b_hi;
        if (more) fetch(b0 + OP_K);
#pragma unroll
        for (int kk = 0; kk < OP_K; ++kk) {
            const float4 dv = *reinterpret_cast<const float4*>(&sd[buf][kk][ty * 4]);
            const float4 av = *reinterpret_cast<const float4*>(&sa[buf][kk][tx * 4]);
            const float dq[4] = {dv.x, dv.y, dv.z, dv.w}, aq[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                accb[q] += dq[q];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[q][j] = fmaf(dq[q], aq[j], acc[q][j]);
            }
        }
        if (more) {
            stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    const int64_t stride = (int64_t)out_dim * in_dim + out_dim;
    float* pz = part + (int64_t)blockIdx.z * stride;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int o = o0 + ty * 4 + q;
        if (o >= out_dim) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + tx * 4 + j;
            if (i < in_dim) pz[(int64_t)o * in_dim + i] = acc[q][j];
        }
        if (blockIdx.x == 0 && tx == 0) pz[(int64_t)out_dim * in_dim + o] = accb[q];
    }
}

// Stage 2: dW += sum of the partials (in split order); db += its sums when db is given.
__global__ void outer_final_kernel(const float* __restrict__ part, int nsplit, int out_dim, int in_dim,
                                   float* __restrict__ dW, float* __restrict__ db) {
    const int64_t nw = (int64_t)out_dim * in_dim, stride = nw + out_dim;
    const int64_t n = db ? stride : nw;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
#pragma unroll 8
        for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * stride + e];
        if (e < nw) dW[e] += s;
        else db[e - nw] += s;
    }
}

// Embedding gradients, deterministic two-stage sums.  Stage 1: CTA (position t, chunk of
// EB_ROWS sequences), thread j = column: the chunk's sums of dh[., t, j] over the sequences
// whose token at t is 0 (or the start token, t = 0) and over those whose token is 1.
constexpr int EB_ROWS = 64;
__global__ void embed_bwd_partial_kernel(ModelConst mc, const uint64_t* __restrict__ bits,
                                         const float* __restrict__ dh, int64_t R, float* __restrict__ part) {
    const int d = mc.hidden, n = mc.n;
    const int t = blockIdx.x, j = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * EB_ROWS, r1 = min(R, r0 + EB_ROWS);
    if (j >= d) return;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
    for (int64_t r = r0; r < r1; ++r) {            // unrolled: the loads fly together, the sums keep their order
        const float g = dh[(r * n + t) * d + j];
        const bool one = t > 0 && ((bits[r] >> mc.order[t - 1]) & 1ull);
        if (one) s1 += g; else s0 += g;
    }
    float* out = part + (((int64_t)blockIdx.y * n + t) * 2) * d;   // [chunk][t][token 0/1][d]
    out[j] = s0;
    out[d + j] = s1;
}

// Stage 2: pos_emb[t] += sum over chunks of both sums; tok_emb[0/1] += sums over chunks and
// positions t >= 1; tok_emb[2] (start token) += the position-0 sums.
__global__ void embed_bwd_final_kernel(ModelConst mc, const float* __restrict__ part, int nchunks,
                                       float* __restrict__ grad) {
    const int d = mc.hidden, n = mc.n;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (n + 3) * d) return;
    const int j = e % d;
    auto at = [&](int c, int t, int k) { return part[(((int64_t)c * n + t) * 2 + k) * d + j]; };
    float s = 0.f;
    if (e < n * d) {
        const int t = e / d;
#pragma unroll 8
        for (int c = 0; c < nchunks; ++c) s += at(c, t, 0) + at(c, t, 1);
        grad[mc.pos_emb + e] += s;
        return;
    }
    const int k = e / d - n;   // token id
    if (k == 2) {
#pragma unroll 8
        for (int c = 0; c < nchunks; ++c) s += at(c, 0, 0);
    } else {
        for (int c = 0; c < nchunks; ++c)
#pragma unroll 8
            for (int t = 1; t < n; ++t) s += at(c, t, k);
    }
    grad[mc.tok_emb + k * d + j] += s;
}

inline int gs(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16)); }

template <class F>
int with_dpl_b(int d, F&& f) {
    switch (d / 32) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 8: return f(std::integral_constant<int, 8>{});
        default: set_error("transformer d_model must be 32, 64, 128 or 256"); return NQS_ERR_UNSUPPORTED;
    }
}

struct BwdBufs {
    int64_t R, M, nsplit, part_elems;
    float** Hin;     // L+1 x [M d]
    float** Hmid;    // L
    void** A1;       // L x [M d] (T_ACT)
    float** QKV;     // L x [M 3d]
    void** O;        // L x [M d] (T_ACT)
    void** A2;       // L
    float** MPRE;    // L x [M 4d]
    void** MM;       // L x [M 4d] (T_ACT)
    // gradients, one buffer per block and use, so that the weight-gradient reductions (a side
    // stream) only read buffers that the main chain never writes again within a chunk
    float* dH[TF_MAX_LAYERS + 1];                  // w.r.t. Hin[l]
    float *dHmid[TF_MAX_LAYERS], *dBig[TF_MAX_LAYERS], *dQKV[TF_MAX_LAYERS];
    float *dSa[TF_MAX_LAYERS], *dSb[TF_MAX_LAYERS], *dSc[TF_MAX_LAYERS];   // into LN2, attention, LN1
    float *GXa[TF_MAX_LAYERS], *GXc[TF_MAX_LAYERS];                        // LN2, LN1 gain terms
    float *dSh, *GXh, *HF, *DL, *DPH, *part, *part_e, *Wr;
};

int64_t bwd_per_seq_floats(const ModelConst& mc) {
    const int64_t n = mc.n, d = mc.hidden, L = mc.layers;
    return n * (d * (L + 1) + L * (d + 3 * d + d + d + 4 * d + 4 * d + d) + d * (L + 1) + L * 13 * d + 3 * d + 1) + 4;
}

void bwd_layout(Carver& c, const ModelConst& mc, int64_t R, BwdBufs& b, float** ptrs, void** vptrs) {
    const int64_t n = mc.n, d = mc.hidden, L = mc.layers, M = R * n;
    b.R = R; b.M = M;
    b.Hin = ptrs; b.Hmid = ptrs + (L + 1); b.QKV = b.Hmid + L; b.MPRE = b.QKV + L;
    b.A1 = vptrs; b.O = vptrs + L; b.A2 = b.O + L; b.MM = b.A2 + L;
    for (int l = 0; l <= L; ++l) b.Hin[l] = c.take<float>(M * d);
    for (int l = 0; l < L; ++l) {
        b.Hmid[l] = c.take<float>(M * d);
        b.A1[l] = c.take<float>(M * d);
        b.QKV[l] = c.take<float>(M * 3 * d);
        b.O[l] = c.take<float>(M * d);
        b.A2[l] = c.take<float>(M * d);
        b.MPRE[l] = c.take<float>(M * 4 * d);
        b.MM[l] = c.take<float>(M * 4 * d);
    }
    for (int l = 0; l <= L; ++l) b.dH[l] = c.take<float>(M * d);
    for (int l = 0; l < L; ++l) {
        b.dHmid[l] = c.take<float>(M * d);
        b.dBig[l] = c.take<float>(M * 4 * d);
        b.dQKV[l] = c.take<float>(M * 3 * d);
        b.dSa[l] = c.take<float>(M * d);
        b.dSb[l] = c.take<float>(M * d);
        b.dSc[l] = c.take<float>(M * d);
        b.GXa[l] = c.take<float>(M * d);
        b.GXc[l] = c.take<float>(M * d);
    }
    b.dSh = c.take<float>(M * d);
    b.GXh = c.take<float>(M * d);
    b.HF = c.take<float>(M * d);
    b.DL = c.take<float>(M);
    b.DPH = c.take<float>(R * 4);
    b.nsplit = std::max<int64_t>(1, std::min<int64_t>(256, (M + 255) / 256));   // ~256 rows per split
    b.part_elems = std::max<int64_t>(b.nsplit * (4 * d * d + 4 * d), ((M + CS_ROWS - 1) / CS_ROWS) * 4 * d);
    b.part_elems = std::max<int64_t>(b.part_elems, 2 * ((M + CS_ROWS - 1) / CS_ROWS) * d);
    b.part_elems = std::max<int64_t>(b.part_elems, ((R + EB_ROWS - 1) / EB_ROWS) * n * 2 * d);
    b.part = c.take<float>(b.part_elems);
    b.part_e = c.take<float>(((R + EB_ROWS - 1) / EB_ROWS) * n * 2 * d);
    b.Wr = c.take<float>(12 * d * d * L);
}

}  // namespace

int64_t tf_bwd_seq_capacity(const ModelConst& mc) {
    const int64_t per = bwd_per_seq_floats(mc) * 4;
    int64_t R = 16;
    while (R * 2 * per <= (512ll << 20) && R < 4096) R *= 2;
    return R;
}

size_t tf_bwd_workspace(const ModelConst& mc, int64_t B) {
    Carver c(nullptr);
    float* ptrs[3 * TF_MAX_LAYERS + 2];
    void* vptrs[4 * TF_MAX_LAYERS];
    BwdBufs b;
    bwd_layout(c, mc, std::max<int64_t>(1, std::min(B, tf_bwd_seq_capacity(mc))), b, ptrs, vptrs);
    return c.used;
}

template <int MODE>
int tf_backward_mode(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                     const float* g_abs, const float* g_phase, float* grad, void* ws, cudaStream_t s, int phases);

int tf_backward(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                const float* g_abs, const float* g_phase, float* grad, void* ws, cudaStream_t s, int phases) {
    if (phases != 3 && B > tf_bwd_seq_capacity(mc)) {
        set_error("two-phase backward: the batch exceeds one recompute pass");
        return NQS_ERR_UNSUPPORTED;
    }
    if (mc.precision != NQS_PREC_BF16) return tf_backward_mode<ACT_F32>(mc, P, bits, B, g_abs, g_phase, grad, ws, s, phases);
    if (mc.compensated) return tf_backward_mode<ACT_F32_Q2>(mc, P, bits, B, g_abs, g_phase, grad, ws, s, phases);
    return tf_backward_mode<ACT_F32_Q1>(mc, P, bits, B, g_abs, g_phase, grad, ws, s, phases);
}

// The weight-gradient reductions run on a library-owned side stream, ordered after the main
// chain's producers by events (one stream and two events per device, created on first use).
struct BwdSide {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
static int bwd_side(BwdSide*& out) {
    static BwdSide sides[16];
    static std::mutex mu;
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 16) { set_error("backward side stream: device index out of range"); return NQS_ERR_UNSUPPORTED; }
    std::lock_guard<std::mutex> lk(mu);
    BwdSide& b = sides[dev];
    if (!b.st) {
        NQS_CK(cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking));
        NQS_CK(cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming));
        NQS_CK(cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming));
    }
    out = &b;
    return NQS_OK;
}

// MODE: how the recomputed forward stores GEMM input activations (fp32 values equal to the
// ones the forward of this precision feeds its GEMMs).
// phases: 1 recompute the forward into the workspace, 2 the backward from it, 3 both.
template <int MODE>
int tf_backward_mode(const ModelConst& mc, const float* P, const uint64_t* bits, int64_t B,
                     const float* g_abs, const float* g_phase, float* grad, void* ws, cudaStream_t s, int phases) {
    const int n = mc.n, d = mc.hidden, dh = d / mc.heads, L = mc.layers;
    const bool bf = mc.precision == NQS_PREC_BF16;
    float* ptrs[3 * TF_MAX_LAYERS + 2];
    void* vptrs[4 * TF_MAX_LAYERS];
    Carver c(ws);
    BwdBufs b;
    bwd_layout(c, mc, std::max<int64_t>(1, std::min(B, tf_bwd_seq_capacity(mc))), b, ptrs, vptrs);

    // weights used by the GEMMs: the fp32 masters, or their bf16-rounded values (BF16 models)
    const float* W[TF_MAX_LAYERS][4];
    const int64_t wsz[4] = {3ll * d * d, 1ll * d * d, 4ll * d * d, 4ll * d * d};
    {
        int64_t off = 0;
        WconvList wl{};
        wl.f32_out = 1;
        for (int l = 0; l < L; ++l) {
            const int64_t src[4] = {mc.wqkv[l], mc.wo[l], mc.w1[l], mc.w2[l]};
            const int cols[4] = {d, d, d, 4 * d};
            for (int q = 0; q < 4; ++q) {
                if (bf) {
                    WconvJob& J = wl.job[wl.njobs++];
                    J.src = P + src[q];
                    J.dst = b.Wr + off;
                    J.start = wl.total;
                    J.cols = cols[q];
                    wl.total += wsz[q];
                    W[l][q] = b.Wr + off;
                    off += wsz[q];
                } else {
                    W[l][q] = P + src[q];
                }
            }
        }
        if (bf && (phases & 1)) {   // all blocks' bf16-rounded copies in one launch
            wconv_kernel<<<gs(wl.total), 256, 0, s>>>(wl);
            NQS_LAUNCHED();
        }
    }

    // bf16 models: the GEMMs on the tensor cores (split fp32 operands); fp32 models: SIMT
    const bool tc = bf;
    auto gemm_nt = [&](auto* A, const float* Wm, const float* bias, float* C, int64_t M, int N, int K,
                       int epi) -> int {
        using TA = std::remove_cv_t<std::remove_pointer_t<decltype(A)>>;
        if constexpr (std::is_same<TA, float>::value) {
            if (tc && tc_bwd_ok(A, K, Wm, K))
                return tc_bwd_gemm_nt(A, K, Wm, K, bias, C, N, M, N, K, epi == TF_EPI_RESID, s);
        }
        dim3 grid((unsigned)((N + SG_BN - 1) / SG_BN), (unsigned)((M + SG_BM - 1) / SG_BM));
        if (epi == TF_EPI_STORE) sgemm_kernel<TA, false, TF_EPI_STORE, float><<<grid, 256, 0, s>>>(A, Wm, bias, C, M, N, K);
        else sgemm_kernel<TA, false, TF_EPI_RESID, float><<<grid, 256, 0, s>>>(A, Wm, bias, C, M, N, K);
        NQS_LAUNCHED();
        return NQS_OK;
    };
    auto gemm_nn = [&](const float* A, const float* Wm, float* C, int64_t M, int N, int K) -> int {
        if (tc && N % 4 == 0 && tc_bwd_ok(A, K, Wm, N)) return tc_bwd_gemm_nn(A, K, Wm, N, C, N, M, N, K, s);
        dim3 grid((unsigned)((N + SG_BN - 1) / SG_BN), (unsigned)((M + SG_BM - 1) / SG_BM));
        sgemm_kernel<float, true, TF_EPI_STORE, float><<<grid, 256, 0, s>>>(A, Wm, nullptr, C, M, N, K);
        NQS_LAUNCHED();
        return NQS_OK;
    };
    // the gradient reductions below run on the side stream ss, each after a fork() that orders it
    // behind everything the main stream has issued so far; b.part is theirs alone
    BwdSide* side = nullptr;
    NQS_TRY(bwd_side(side));
    cudaStream_t ss = side->st;
    auto fork = [&]() -> int {
        NQS_CK(cudaEventRecord(side->fork, s));
        NQS_CK(cudaStreamWaitEvent(ss, side->fork, 0));
        return NQS_OK;
    };
    auto join = [&]() -> int {
        NQS_CK(cudaEventRecord(side->join, ss));
        NQS_CK(cudaStreamWaitEvent(s, side->join, 0));
        return NQS_OK;
    };
    // column sums of X0 (and X1) into out0 (and out1)
    auto colsum = [&](const float* X0, const float* X1, int64_t ld, int64_t M, int ncols, float* out0,
                      float* out1) -> int {
        const int nch = (int)((M + CS_ROWS - 1) / CS_ROWS);
        const int nmat = X1 ? 2 : 1;
        colsum_partial_kernel<<<dim3((ncols + 31) / 32, nch, nmat), dim3(32, 8), 0, ss>>>(X0, X1, ld, M, ncols, b.part);
        NQS_LAUNCHED();
        colsum_final_kernel<<<(nmat * ncols + 7) / 8, 256, 0, ss>>>(b.part, nch, ncols, nmat, out0, out1);
        NQS_LAUNCHED();
        return NQS_OK;
    };
    // dW += delta^T act and (if db) db += column sums of delta
    auto outer = [&](const float* delta, int64_t ld_d, const float* act, int64_t ld_a, int64_t M, int out_dim,
                     int in_dim, float* dW, float* db) -> int {
        const int64_t stride = (int64_t)out_dim * in_dim + out_dim;
        const int64_t ns = std::max<int64_t>(1, std::min<int64_t>(b.nsplit, b.part_elems / stride));
        const int64_t per = (M + ns - 1) / ns;
        if (tc && out_dim >= 64 && out_dim % 4 == 0 && in_dim % 4 == 0 && tc_bwd_ok(delta, ld_d, act, ld_a)) {
            NQS_TRY(tc_bwd_outer_partial(delta, ld_d, act, ld_a, M, out_dim, in_dim, ns, per, db != nullptr, b.part, ss));
        } else {
            dim3 grid((unsigned)((in_dim + OP_B - 1) / OP_B), (unsigned)((out_dim + OP_B - 1) / OP_B), (unsigned)ns);
            outer_partial_kernel<<<grid, 256, 0, ss>>>(delta, ld_d, act, ld_a, M, out_dim, in_dim, per, b.part);
            NQS_LAUNCHED();
        }
        outer_final_kernel<<<gs(stride), 256, 0, ss>>>(b.part, (int)ns, out_dim, in_dim, dW, db);
        NQS_LAUNCHED();
        return NQS_OK;
    };

    return with_dpl_b(d, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        const size_t att_smem = (size_t)(4 * n * (dh + 1) + 2 * n * (n + 1)) * sizeof(float);
        if (att_smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(attention_bwd_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)att_smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(attention_bwd_any_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)att_smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
        }
        for (int64_t lo = 0; lo < B; lo += b.R) {
            const int64_t R = std::min(b.R, B - lo);
            const int64_t M = R * n;
            const uint64_t* xb = bits + lo;
            if (phases & 1) {
            // ---- forward with saved activations
            auto ps_fwd = std::make_unique<ProfScope>("bwd_recompute", s);
            embed_kernel<<<gs(M * d), 256, 0, s>>>(mc, P, xb, R, n, b.Hin[0]);
            NQS_LAUNCHED();
            auto ln_fwd = [&](const float* hsrc, const float* g, const float* bb, void* dst) -> int {
                layernorm_kernel<MODE, DPL><<<ln_grid(M), 256, 0, s>>>(hsrc, M, d, g, bb, dst);
                NQS_LAUNCHED();
                return NQS_OK;
            };
            NQS_TRY(ln_fwd(b.Hin[0], P + mc.ln1_g[0], P + mc.ln1_b[0], b.A1[0]));
            for (int l = 0; l < L; ++l) {
                NQS_TRY(gemm_nt((const float*)b.A1[l], W[l][TF_WQKV], P + mc.bqkv[l], b.QKV[l], M, 3 * d, d, TF_EPI_STORE));
                NQS_CK(launch_attention<MODE>(b.QKV[l], R, n, d, mc.heads, b.O[l], s));
                count_launch();
                NQS_CK(cudaMemcpyAsync(b.Hmid[l], b.Hin[l], M * d * sizeof(float), cudaMemcpyDeviceToDevice, s));
                NQS_TRY(gemm_nt((const float*)b.O[l], W[l][TF_WO], P + mc.bo[l], b.Hmid[l], M, d, d, TF_EPI_RESID));
                NQS_TRY(ln_fwd(b.Hmid[l], P + mc.ln2_g[l], P + mc.ln2_b[l], b.A2[l]));
                NQS_TRY(gemm_nt((const float*)b.A2[l], W[l][TF_W1], P + mc.b1[l], b.MPRE[l], M, 4 * d, d, TF_EPI_STORE));
                gelu_fwd_kernel<MODE><<<gs(M * 4 * d), 256, 0, s>>>(b.MPRE[l], (float*)b.MM[l], M * 4 * d);
                NQS_LAUNCHED();
                NQS_CK(cudaMemcpyAsync(b.Hin[l + 1], b.Hmid[l], M * d * sizeof(float), cudaMemcpyDeviceToDevice, s));
                NQS_TRY(gemm_nt((const float*)b.MM[l], W[l][TF_W2], P + mc.b2[l], b.Hin[l + 1], M, d, 4 * d, TF_EPI_RESID));
                if (l + 1 < L) NQS_TRY(ln_fwd(b.Hin[l + 1], P + mc.ln1_g[l + 1], P + mc.ln1_b[l + 1], b.A1[l + 1]));
            }
            ps_fwd.reset();
            }
            if (!(phases & 2)) continue;
            // ---- heads and final LayerNorm
            auto ps_heads = std::make_unique<ProfScope>("bwd_heads", s);
            heads_bwd_kernel<DPL><<<(int)((M + 7) / 8), 256, 0, s>>>(mc, P, xb, b.Hin[L], R, g_abs + lo, g_phase + lo,
                                                                      b.dH[L], b.dSh, b.GXh, b.HF, b.DL, b.DPH);
            NQS_LAUNCHED();
            NQS_TRY(fork());
            NQS_TRY(outer(b.DL, 1, b.HF, d, M, 1, d, grad + mc.head_w, nullptr));
            NQS_TRY(colsum(b.DL, nullptr, n, R, n, grad + mc.head_b, nullptr));
            NQS_TRY(outer(b.DPH, 4, b.HF + (int64_t)(n - 2) * d, (int64_t)n * d, R, 4, d, grad + mc.phase_w,
                          grad + mc.phase_b));
            NQS_TRY(colsum(b.GXh, b.dSh, d, M, d, grad + mc.lnf_g, grad + mc.lnf_b));
            ps_heads.reset();
            // ---- blocks, last to first (weight gradients on the side stream)
            for (int l = L - 1; l >= 0; --l) {
                // MLP: Hin[l+1] = Hmid + gelu(A2 W1^T + b1) W2^T + b2
                auto ps_mlp = std::make_unique<ProfScope>("bwd_mlp", s);
                NQS_TRY(outer(b.dH[l + 1], d, (const float*)b.MM[l], 4 * d, M, d, 4 * d, grad + mc.w2[l], grad + mc.b2[l]));
                NQS_TRY(gemm_nn(b.dH[l + 1], W[l][TF_W2], b.dBig[l], M, 4 * d, d));
                gelu_bwd_kernel<<<gs(M * 4 * d), 256, 0, s>>>(b.MPRE[l], b.dBig[l], M * 4 * d);
                NQS_LAUNCHED();
                NQS_TRY(fork());
                NQS_TRY(outer(b.dBig[l], 4 * d, (const float*)b.A2[l], d, M, 4 * d, d, grad + mc.w1[l], grad + mc.b1[l]));
                NQS_TRY(gemm_nn(b.dBig[l], W[l][TF_W1], b.dSa[l], M, d, 4 * d));
                ln_bwd_kernel<DPL><<<(int)((M + 7) / 8), 256, 0, s>>>(b.Hmid[l], P + mc.ln2_g[l], b.dSa[l], b.dH[l + 1],
                                                                       b.dHmid[l], b.GXa[l], M, d);
                NQS_LAUNCHED();
                NQS_TRY(fork());
                NQS_TRY(colsum(b.GXa[l], b.dSa[l], d, M, d, grad + mc.ln2_g[l], grad + mc.ln2_b[l]));
                ps_mlp.reset();
                // attention: Hmid = Hin + attn(A1 Wqkv^T + bqkv) Wo^T + bo
                ProfScope ps_att("bwd_attention", s);
                NQS_TRY(outer(b.dHmid[l], d, (const float*)b.O[l], d, M, d, d, grad + mc.wo[l], grad + mc.bo[l]));
                NQS_TRY(gemm_nn(b.dHmid[l], W[l][TF_WO], b.dSb[l], M, d, d));
                if (dh == 16)
                    attention_bwd_kernel<16><<<dim3((unsigned)R, (unsigned)mc.heads), 128, att_smem, s>>>(b.QKV[l], b.dSb[l], n, d,
                                                                                                        b.dQKV[l]);
                else
                    attention_bwd_any_kernel<<<dim3((unsigned)R, (unsigned)mc.heads), 128, att_smem, s>>>(b.QKV[l], b.dSb[l], n, d, dh,
                                                                                                        b.dQKV[l]);
                NQS_LAUNCHED();
                NQS_TRY(fork());
                NQS_TRY(outer(b.dQKV[l], 3 * d, (const float*)b.A1[l], d, M, 3 * d, d, grad + mc.wqkv[l], grad + mc.bqkv[l]));
                NQS_TRY(gemm_nn(b.dQKV[l], W[l][TF_WQKV], b.dSc[l], M, d, 3 * d));
                ln_bwd_kernel<DPL><<<(int)((M + 7) / 8), 256, 0, s>>>(b.Hin[l], P + mc.ln1_g[l], b.dSc[l], b.dHmid[l], b.dH[l],
                                                                       b.GXc[l], M, d);
                NQS_LAUNCHED();
                NQS_TRY(fork());
                NQS_TRY(colsum(b.GXc[l], b.dSc[l], d, M, d, grad + mc.ln1_g[l], grad + mc.ln1_b[l]));
            }
            {
                ProfScope ps_emb("bwd_embed", s);
                const int nch = (int)((R + EB_ROWS - 1) / EB_ROWS);
                embed_bwd_partial_kernel<<<dim3(n, nch), d, 0, s>>>(mc, xb, b.dH[0], R, b.part_e);
                NQS_LAUNCHED();
                embed_bwd_final_kernel<<<((n + 3) * d + 255) / 256, 256, 0, s>>>(mc, b.part_e, nch, grad);
                NQS_LAUNCHED();
            }
            // the side stream's reductions are done before the next chunk reuses the buffers and
            // before the caller reads the gradient
            NQS_TRY(join());
        }
        return NQS_OK;
    });
}

}  // namespace nqs
