// Prefix-sharing local energy for the transformer wavefunction.
//
// Every connected x' = x ^ m of a sample x agrees with x on the sampling positions before its
// first flipped bit, and x' that share their first flips agree further: the transformer's row at
// position t depends on the bits at positions < t only, so all those rows are equal (the same
// autoregressive structure the sampler uses to reuse its keys and values; the local-energy
// counterpart of the paper's unique flippings, Section 5.1, applied to prefixes).  With flips at
// positions f1 < f2 < f3 < ... (sampling order) the work is organised as jobs, each a string
// whose rows are computed from some position `start` on, with the keys and values of the
// positions before `start` read from a parent job's cache:
//
//   level 0   the sample x itself: all n rows (start 0), no parent
//   level 1   x with flip f1 (prefix depth >= 2): rows f1+1 .. n-1, parent x
//   level 2   x with flips f1, f2 (depth 3): rows f2+1 .. n-1, parent the level-1 job of f1
//   leaves    every x' row of the term sweep: rows from one past the first flip its parent
//             does not carry (depth 3: f3 + 1 for three or more flips, f2 + 1 for two; depth
//             2: f2 + 1; depth 1: f1 + 1 with parent x; depth 0: from position 0, no parent)
//
// Pass A evaluates levels 0-2 together, layer by layer, and stores each job's keys and values of
// every layer for all n positions (positions before `start` copied from the parent, level by
// level) together with its per-position output logits, the TwoSum prefix sums of its
// log-probabilities and its phase-head outputs.  Pass B evaluates the leaves in sub-passes of
// bounded row count against those caches, and turns each leaf's log psi into its ratio-weighted
// contribution S(x, x') psi(x')/psi(x).  A leaf's log|psi| is its parent's prefix sum up to the
// branch position, plus the parent's logit at the branch position with the leaf's own bit, plus
// the terms of its own rows.  Rows are computed by the same kernels whatever their job, and a
// row's keys and values are the same numbers whether they come from a cache or from its own
// pass, so the local energies do not depend on the prefix depth, bit for bit.
#include "tf_common.cuh"

namespace nqs {
namespace {

// The flip mask m as a mask over sampling positions.
__device__ __forceinline__ uint64_t pos_mask(const ModelConst& mc, uint64_t m) {
    uint64_t pm = 0;
    while (m) {
        const int q = __ffsll((long long)m) - 1;
        m &= m - 1;
        pm |= 1ull << mc.pos[q];
    }
    return pm;
}

__device__ __forceinline__ int ctz64(uint64_t v) { return __ffsll((long long)v) - 1; }
__device__ __forceinline__ uint64_t below(int f) { return f >= 64 ? ~0ull : ((1ull << f) - 1ull); }

// Sample of sweep row r: the segment of the chunk's row offsets (stride seg_stride) holding r.
__device__ __forceinline__ int64_t seg_of(const int64_t* __restrict__ seg, int64_t stride, int64_t nseg, int64_t r) {
    int64_t lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (seg[mid * stride] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- job construction
__global__ void ch_mark_kernel(ModelConst mc, const uint64_t* __restrict__ xs, int64_t nb, const int64_t* __restrict__ seg,
                               int64_t seg_stride, const uint64_t* __restrict__ xprime, const int64_t* __restrict__ rows_dev,
                               int64_t rows_max, int depth, unsigned long long* __restrict__ l1,
                               unsigned long long* __restrict__ l2) {
    const int64_t rows = min(*rows_dev, rows_max);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = seg_of(seg, seg_stride, nb, r);
        const uint64_t m = xs[i] ^ xprime[r];
        if (!m) continue;
        const uint64_t pm = pos_mask(mc, m);
        const int k = __popcll(pm);
        const int f1 = ctz64(pm);
        if (depth >= 2 && k >= 2) atomicOr(l1 + i, 1ull << f1);
        if (depth >= 3 && k >= 3) atomicOr(l2 + i * 64 + f1, 1ull << ctz64(pm & (pm - 1)));
    }
}

// One warp per sample: level-1 and level-2 chain counts and the per-f1 prefix of level-2 chains.
__global__ void ch_count_kernel(const unsigned long long* __restrict__ l1, const unsigned long long* __restrict__ l2,
                                int64_t nb, int64_t* __restrict__ cnt1, int64_t* __restrict__ cnt2,
                                int32_t* __restrict__ cum2) {
    const int lane = threadIdx.x & 31;
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= nb) return;
    const int c0 = __popcll(l2[i * 64 + lane]), c1 = __popcll(l2[i * 64 + 32 + lane]);
    int v0 = c0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v0, d);
        if (lane >= d) v0 += y;
    }
    const int tot0 = __shfl_sync(0xffffffffu, v0, 31);
    int v1 = c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v1, d);
        if (lane >= d) v1 += y;
    }
    cum2[i * 64 + lane] = v0 - c0;
    cum2[i * 64 + 32 + lane] = tot0 + v1 - c1;
    if (lane == 31) {
        cnt2[i] = tot0 + v1;
        cnt1[i] = __popcll(l1[i]);
    }
}

__device__ __forceinline__ int64_t l1_id(int64_t nb, const int64_t* base1, const unsigned long long* l1, int64_t i, int f1) {
    return nb + base1[i] + __popcll(l1[i] & below(f1));
}
__device__ __forceinline__ int64_t l2_id(int64_t nb, const int64_t* base1, const int64_t* base2, const int32_t* cum2,
                                         const unsigned long long* l2, int64_t i, int f1, int f2) {
    return nb + base1[nb] + base2[i] + cum2[i * 64 + f1] + __popcll(l2[i * 64 + f1] & below(f2));
}

// Thread per (sample, position f): the level-0 job at f = 0, the level-1 job of flip f and the
// level-2 jobs (f, f2).
__global__ void ch_jobs_kernel(ModelConst mc, const uint64_t* __restrict__ xs, int64_t nb,
                               const unsigned long long* __restrict__ l1, const unsigned long long* __restrict__ l2,
                               const int64_t* __restrict__ base1, const int64_t* __restrict__ base2,
                               const int32_t* __restrict__ cum2, uint64_t* __restrict__ jbits, int32_t* __restrict__ jstart,
                               int32_t* __restrict__ jpar, int64_t* __restrict__ jrows, int64_t* __restrict__ jseg) {
    const int n = mc.n;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nb * n) return;
    const int64_t i = idx / n;
    const int f = (int)(idx - i * n);
    const uint64_t x = xs[i];
    // jseg[j]: one past the last job with j's parent (jobs of one parent are consecutive)
    if (f == 0) { jbits[i] = x; jstart[i] = 0; jpar[i] = -1; jrows[i] = n; jseg[i] = nb; }
    if (!((l1[i] >> f) & 1ull)) return;
    const int64_t id1 = l1_id(nb, base1, l1, i, f);
    const uint64_t x1 = x ^ (1ull << mc.order[f]);
    jbits[id1] = x1; jstart[id1] = f + 1; jpar[id1] = (int32_t)i; jrows[id1] = n - f - 1;
    jseg[id1] = nb + base1[i + 1];
    uint64_t w = l2[i * 64 + f];
    const int64_t end2 = nb + base1[nb] + base2[i] + cum2[i * 64 + f] + __popcll(w);
    while (w) {
        const int f2 = ctz64(w);
        w &= w - 1;
        const int64_t id2 = l2_id(nb, base1, base2, cum2, l2, i, f, f2);
        jbits[id2] = x1 ^ (1ull << mc.order[f2]); jstart[id2] = f2 + 1; jpar[id2] = (int32_t)id1; jrows[id2] = n - f2 - 1;
        jseg[id2] = end2;
    }
}

// Per sweep row: the leaf's parent job and first own position (n: the diagonal row, no rows).
__global__ void ch_leaf_kernel(ModelConst mc, const uint64_t* __restrict__ xs, int64_t nb, const int64_t* __restrict__ seg,
                               int64_t seg_stride, const uint64_t* __restrict__ xprime, const int64_t* __restrict__ rows_dev,
                               int64_t rows_max, int depth, const unsigned long long* __restrict__ l1,
                               const unsigned long long* __restrict__ l2, const int64_t* __restrict__ base1,
                               const int64_t* __restrict__ base2, const int32_t* __restrict__ cum2,
                               int32_t* __restrict__ lpar, int32_t* __restrict__ lstart, int64_t* __restrict__ lrows) {
    const int n = mc.n;
    const int64_t rows = min(*rows_dev, rows_max);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = seg_of(seg, seg_stride, nb, r);
        const uint64_t m = xs[i] ^ xprime[r];
        int64_t par = -1;
        int start = n;
        if (m) {
            const uint64_t pm = pos_mask(mc, m);
            const int k = __popcll(pm);
            const int f1 = ctz64(pm);
            const uint64_t r1 = pm & (pm - 1);
            if (depth <= 0) { start = 0; }
            else if (depth == 1 || k < 2) { par = i; start = f1 + 1; }
            else {
                const int f2 = ctz64(r1);
                if (depth == 2 || k < 3) { par = l1_id(nb, base1, l1, i, f1); start = f2 + 1; }
                else { par = l2_id(nb, base1, base2, cum2, l2, i, f1, f2); start = ctz64(r1 & (r1 - 1)) + 1; }
            }
        }
        lpar[r] = (int32_t)par;
        lstart[r] = start;
        lrows[r] = n - start;
    }
}

// Row table of a pass over slots [i0, i1): slot i is job (or leaf) id = order ? order[i] : i,
// whose rows [off[i] - base, ...) are its positions start[id] .. n-1.
__global__ void ch_rows_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ order,
                               const int32_t* __restrict__ start, int64_t i0, int64_t i1, int64_t base, int n,
                               int32_t* __restrict__ rjob, uint8_t* __restrict__ rpos, uint8_t* __restrict__ rstart) {
    for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t id = order ? order[i] : i;
        const int64_t q0 = off[i] - base;
        const int s0 = start[id];
        for (int t = s0; t < n; ++t) {
            rjob[q0 + t - s0] = (int32_t)id;
            rpos[q0 + t - s0] = (uint8_t)t;
            rstart[q0 + t - s0] = (uint8_t)s0;
        }
    }
}

// Leaves with own rows grouped by parent (a counting sort; the order inside a parent's group
// is whatever the atomics give, which no result depends on): histogram, then scatter.
__global__ void ch_hist_kernel(const int32_t* __restrict__ lpar, const int64_t* __restrict__ lrows,
                               const int64_t* __restrict__ rows_dev, int64_t rows_max, int64_t jobs,
                               unsigned long long* __restrict__ hist) {
    const int64_t rows = min(*rows_dev, rows_max);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        if (lrows[r] <= 0) continue;
        const int64_t bkt = lpar[r] >= 0 ? lpar[r] : jobs;
        atomicAdd(hist + bkt, 1ull);
    }
}

__global__ void ch_scatter_kernel(const int32_t* __restrict__ lpar, const int64_t* __restrict__ lrows,
                                  const int64_t* __restrict__ rows_dev, int64_t rows_max, int64_t jobs,
                                  const int64_t* __restrict__ hoff, unsigned long long* __restrict__ cursor,
                                  int32_t* __restrict__ order, int64_t* __restrict__ srows, int64_t* __restrict__ sseg) {
    const int64_t rows = min(*rows_dev, rows_max);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        if (lrows[r] <= 0) continue;
        const int64_t bkt = lpar[r] >= 0 ? lpar[r] : jobs;
        const int64_t slot = hoff[bkt] + (int64_t)atomicAdd(cursor + bkt, 1ull);
        order[slot] = (int32_t)r;
        srows[slot] = lrows[r];
        sseg[slot] = hoff[bkt + 1];      // one past the parent's last slot
    }
}

// Sub-pass boundaries of the leaves: split[k] = first leaf whose row offset is >= k * cap.
__global__ void ch_split_kernel(const int64_t* __restrict__ off, const int64_t* __restrict__ rows_dev, int64_t rows_max,
                                int64_t cap, int nsplit, int64_t* __restrict__ split, int64_t* __restrict__ split_off) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nsplit) return;
    const int64_t rows = min(*rows_dev, rows_max);
    int64_t lo = 0, hi = rows;
    if (k == nsplit) lo = rows;
    else {
        const int64_t target = (int64_t)k * cap;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] < target) lo = mid + 1; else hi = mid;
        }
    }
    split[k] = lo;
    split_off[k] = off[lo];
}

// Chunks of a pass for the attention: consecutive slots of one parent whose rows fit `cap`
// rows, packed greedily from each parent segment's first slot.  Pass 1 counts a segment's
// chunks at its first slot, pass 2 writes [first slot, end slot) of each chunk at the scanned
// offset; the chunk count lands in *n_chunks (device).
__device__ __forceinline__ bool ch_seg_first(const int64_t* __restrict__ segend, int64_t i, int64_t i0) {
    return i == i0 || segend[i] != segend[i - 1];
}

__global__ void ch_chunk_count_kernel(const int64_t* __restrict__ off, const int64_t* __restrict__ segend,
                                      const int64_t* __restrict__ n_dev, int64_t i0, int64_t i1, int cap,
                                      int64_t* __restrict__ cnt, int64_t* __restrict__ tcnt) {
    const int64_t e1 = n_dev ? min(i1, *n_dev) : i1;
    for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e1; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0, t = 0;
        if (ch_seg_first(segend, i, i0)) {
            const int64_t se = min(segend[i], e1);
            int64_t a = i;
            while (a < se) {
                int64_t e = a + 1;
                while (e < se && off[e + 1] - off[a] <= cap) ++e;
                ++c;
                a = e;
            }
            for (int64_t j = i; j < se; ++j) t += (off[j + 1] - off[j] + 15) >> 4;
        }
        cnt[i - i0] = c;
        tcnt[i - i0] = t;
    }
}

// Chunk records (first row offset, rows | parent << 32, first tile, end tile) and the 16-row
// tiles of each job: (row0, rows, job's first row, job start), rows relative to the chunk.
__global__ void ch_chunk_write_kernel(const int64_t* __restrict__ off, const int64_t* __restrict__ segend,
                                      const int64_t* __restrict__ n_dev, int64_t i0, int64_t i1, int cap,
                                      const int64_t* __restrict__ coff, const int64_t* __restrict__ toff,
                                      const int32_t* __restrict__ order, const int32_t* __restrict__ start,
                                      const int32_t* __restrict__ par, int64_t* __restrict__ chunks,
                                      int32_t* __restrict__ tiles) {
    const int64_t e1 = n_dev ? min(i1, *n_dev) : i1;
    for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e1; i += (int64_t)gridDim.x * blockDim.x) {
        if (!ch_seg_first(segend, i, i0)) continue;
        const int64_t se = min(segend[i], e1);
        int64_t a = i, k = coff[i - i0], t = toff[i - i0];
        while (a < se) {
            int64_t e = a + 1;
            while (e < se && off[e + 1] - off[a] <= cap) ++e;
            const int32_t p0 = par[order ? order[a] : a];
            chunks[4 * k] = off[a];
            chunks[4 * k + 1] = (int64_t)(((uint64_t)(uint32_t)p0 << 32) | (uint64_t)(off[e] - off[a]));
            chunks[4 * k + 2] = t;
            for (int64_t j = a; j < e; ++j) {
                const int first = (int)(off[j] - off[a]), rows = (int)(off[j + 1] - off[j]);
                const int st = start[order ? order[j] : j];
                for (int r0 = 0; r0 < rows; r0 += 16, ++t) {
                    tiles[4 * t] = first + r0;
                    tiles[4 * t + 1] = min(16, rows - r0);
                    tiles[4 * t + 2] = first;
                    tiles[4 * t + 3] = st;
                }
            }
            chunks[4 * k + 3] = t;
            ++k;
            a = e;
        }
    }
}

// ---------------------------------------------------------------- forward pieces
// Embedding + first LayerNorm of the pass's rows: row q is position rpos[q] of job rjob[q].
template <int MODE, int DPL>
__global__ void __launch_bounds__(256)
ch_embed_ln_kernel(ModelConst mc, const float* __restrict__ P, const uint64_t* __restrict__ jbits,
                   const int32_t* __restrict__ rjob, const uint8_t* __restrict__ rpos, int64_t M,
                   float* __restrict__ h, void* __restrict__ a) {
    const int d = mc.hidden;
    const int lane = threadIdx.x & 31, col0 = lane * DPL;
    const int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * LN_ROWS;
    if (base >= M) return;
    float v[LN_ROWS][DPL];
    int64_t rows[LN_ROWS];
#pragma unroll
    for (int r = 0; r < LN_ROWS; ++r) {
        rows[r] = base + r;
        const int64_t q = rows[r] < M ? rows[r] : M - 1;
        const int t = rpos[q];
        const int tok = t == 0 ? 2 : (int)((jbits[rjob[q]] >> mc.order[t - 1]) & 1ull);
        float e[DPL], p[DPL];
        load_row<DPL>(P + mc.tok_emb + tok * d + col0, e);
        load_row<DPL>(P + mc.pos_emb + t * d + col0, p);
#pragma unroll
        for (int i = 0; i < DPL; ++i) v[r][i] = e[i] + p[i];
        if (rows[r] < M) store_floats<DPL>(h + rows[r] * d + col0, v[r]);
    }
    ln_rows_store<MODE, DPL>(v, rows, M, d, col0, P + mc.ln1_g[0], P + mc.ln1_b[0], a);
}

// Keys and values of layer l of jobs [j0, j1) for all n positions into their caches: positions
// before `start` from the parent's cache, the others from the job's own rows of the pass.
// Cache of job j, layer l: kv + ((j * L + l) * n + p) * 2d (keys then values).
__global__ void __launch_bounds__(256)
ch_cache_fill_kernel(float* __restrict__ kv, int L, int l, int n, int d, int64_t j0, int64_t j1,
                     const int32_t* __restrict__ jstart, const int32_t* __restrict__ jpar,
                     const int64_t* __restrict__ joff, const float* __restrict__ qkv) {
    const int per_pos = d / 2;   // float4 chunks of K|V per position
    for (int64_t j = j0 + blockIdx.x; j < j1; j += gridDim.x) {
        const int s0 = jstart[j];
        const int64_t par = jpar[j];
        float4* dst = reinterpret_cast<float4*>(kv + ((j * L + l) * (int64_t)n) * 2 * d);
        const float4* pre = par >= 0 ? reinterpret_cast<const float4*>(kv + ((par * L + l) * (int64_t)n) * 2 * d) : nullptr;
        for (int e = threadIdx.x; e < n * per_pos; e += blockDim.x) {
            const int p = e / per_pos, c = e - p * per_pos;
            dst[e] = p < s0 ? pre[e]
                            : reinterpret_cast<const float4*>(qkv + (joff[j] + p - s0) * (int64_t)(3 * d) + d)[c];
        }
    }
}

// Causal attention of the pass's rows over a list of chunks (consecutive slots of one parent
// whose rows fit the staging buffer).  CTAs take chunks interleaved, so the CTAs running at any
// moment work on neighbouring chunks and share their parents' caches in L2.  For each chunk and
// group of HG heads a CTA stages in shared memory (cp.async) the group's keys and values of the
// parent at all n positions and of the chunk's own rows; then each warp takes a (block of 32
// rows, head) item -- lane = row -- and runs the online softmax over keys 0..t in the log2
// domain, in blocks of KB keys: keys before the row's job start from the staged parent, the
// job's own keys from its staged rows.  Lanes of a block share most keys, so a key load is a
// broadcast; rows are padded so neighbouring rows sit on other banks.
constexpr int CH_ATT_THREADS = 128;
constexpr int CH_ATT_HG = 2;                            // heads per staging group

template <int MODE, int DH, int H>
__global__ void __launch_bounds__(CH_ATT_THREADS, 6)
ch_attention_kernel(const float* __restrict__ qkv, void* __restrict__ o, int n, const int64_t* __restrict__ chunks,
                    const int64_t* __restrict__ n_chunks, int64_t row_base, const uint8_t* __restrict__ rpos,
                    const uint8_t* __restrict__ rstart, const float* __restrict__ kv, int L, int l) {
    extern __shared__ __align__(16) float ch_att_sm[];
    constexpr int D = H * DH;
    constexpr int HG = H < CH_ATT_HG ? H : CH_ATT_HG;   // heads per staging group
    constexpr int KVP = 2 * DH + 4;                     // a head's (key, value) slice, padded
    constexpr int RS = HG * KVP + 4;                    // one position / row of the group (rows on other banks)
    constexpr int ld = 3 * D;
    constexpr int C4 = HG * DH / 2;                     // float4 chunks of the group's K|V of one position
    float* sp = ch_att_sm;                              // parent: [n][RS]
    float* so = ch_att_sm + n * RS;                     // chunk rows: [rows][RS]
    const float scale = rsqrtf((float)DH) * 1.4426950408889634f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = CH_ATT_THREADS / 32;
    const int64_t nck = *n_chunks;
    for (int64_t wi = blockIdx.x; wi < nck * (H / HG); wi += gridDim.x) {
        const int64_t ck = wi / (H / HG);
        const int h0 = (int)(wi % (H / HG)) * HG;
        const int64_t r_lo = chunks[4 * ck] - row_base;
        const uint64_t rec = (uint64_t)chunks[4 * ck + 1];
        const int32_t p0 = (int32_t)(uint32_t)(rec >> 32);
        const int nrows = (int)(uint32_t)rec;
        for (int c = threadIdx.x; c < nrows * C4; c += blockDim.x) {
            const int r = c / C4, w = c % C4;
            const int kvsel = w / (C4 / 2), col = 4 * (w % (C4 / 2));      // col within the group's heads
            cp_async16(so + r * RS + (col / DH) * KVP + kvsel * DH + (col % DH),
                       qkv + (r_lo + r) * ld + D + kvsel * D + h0 * DH + col);
        }
        if (p0 >= 0) {
            const float* pre = kv + (((int64_t)p0 * L + l) * (int64_t)n) * 2 * D;
            for (int c = threadIdx.x; c < n * C4; c += blockDim.x) {
                const int p = c / C4, w = c % C4;
                const int kvsel = w / (C4 / 2), col = 4 * (w % (C4 / 2));
                cp_async16(sp + p * RS + (col / DH) * KVP + kvsel * DH + (col % DH),
                           pre + (int64_t)p * 2 * D + kvsel * D + h0 * DH + col);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        const int nblk = (nrows + 31) / 32;
        for (int it = warp; it < nblk * HG; it += NW) {
            const int blk = it / HG, hl = it % HG, hh = h0 + hl;
            const int rr = blk * 32 + lane;
            const bool act = rr < nrows;
            const int rc = act ? rr : nrows - 1;
            const int64_t q = r_lo + rc;
            const int t = rpos[q];
            const int s0 = rstart[q];
            const int own0 = rc - (t - s0);             // chunk row of the job's position s0
            int tmax = act ? t : -1;
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o2));
            float qv[DH], acc[DH];
            const float4* qs = reinterpret_cast<const float4*>(qkv + q * ld + hh * DH);
#pragma unroll
            for (int j4 = 0; j4 < DH / 4; ++j4) {
                const float4 x = __ldg(qs + j4);
                qv[4 * j4] = x.x * scale; qv[4 * j4 + 1] = x.y * scale;
                qv[4 * j4 + 2] = x.z * scale; qv[4 * j4 + 3] = x.w * scale;
            }
#pragma unroll
            for (int c = 0; c < DH; ++c) acc[c] = 0.f;
            float m = -INFINITY, lsum = 0.f;
            constexpr int KB = 8;
            const float* sph = sp + hl * KVP;
            const float* soh = so + hl * KVP;
            for (int pk = 0; pk <= tmax; pk += KB) {
                const float* kp[KB];
                bool ok[KB];
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    const int p = pk + j;
                    ok[j] = act && p <= t;
                    // masked keys read the chunk's first row, the same address in every lane
                    kp[j] = !ok[j] ? soh : (p < s0 ? sph + p * RS : soh + (own0 + p - s0) * RS);
                }
                float sc[KB];
                float bm = -INFINITY;
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    sc[j] = ok[j] ? att_dot<DH>(qv, reinterpret_cast<const float4*>(kp[j])) : -INFINITY;
                    bm = fmaxf(bm, sc[j]);
                }
                if (bm > m) {
                    const float c = ex2_approx(m - bm);    // 0 on the first block
                    lsum *= c;
#pragma unroll
                    for (int c2 = 0; c2 < DH; ++c2) acc[c2] *= c;
                    m = bm;
                }
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    const float ev = ok[j] ? ex2_approx(sc[j] - m) : 0.f;
                    lsum += ev;
                    const float4* vr = reinterpret_cast<const float4*>(kp[j] + DH);
#pragma unroll
                    for (int j4 = 0; j4 < DH / 4; ++j4) {
                        const float4 v4 = vr[j4];
                        acc[4 * j4] = fmaf(ev, v4.x, acc[4 * j4]);
                        acc[4 * j4 + 1] = fmaf(ev, v4.y, acc[4 * j4 + 1]);
                        acc[4 * j4 + 2] = fmaf(ev, v4.z, acc[4 * j4 + 2]);
                        acc[4 * j4 + 3] = fmaf(ev, v4.w, acc[4 * j4 + 3]);
                    }
                }
            }
            if (act) att_store_row<MODE, DH>(acc, lsum, o, q, D, hh * DH);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- attention on the mma.sync path
// The same causal attention for the bf16 forms with head size 16, on the tensor path (mma.sync
// m16n8k16, bf16 operands, fp32 accumulate) with every product in the compensated form
// x y ~ x_hi y_hi + x_hi y_lo + x_lo y_hi (hi = bf16(x), lo = bf16(x - hi)).  The projection
// writes q, k and v already split (the split layout of tc_gemm_bf16: [Q hi | Q lo | K hi | K lo |
// V hi | V lo] per row; the caches hold [K hi | K lo | V hi | V lo] per position), so staging is
// a plain asynchronous copy.  A CTA takes (chunk, head) items, interleaved over the grid, and
// stages the next item (cp.async, double-buffered) while it computes the current one.  A warp
// takes a tile of up to 16 consecutive rows of ONE job from the chunk's tile table and runs the
// online softmax over key positions in steps of 16 (positions 16 k .. 16 k + 15 for every row,
// whatever its job): the keys of a step are gathered by ldmatrix from per-lane row addresses,
// position p from the staged parent when p < start and from the job's own staged row
// otherwise, so the arithmetic of a row is the same whichever job (and prefix depth) it is
// computed in -- the local energies stay independent of the prefix depth bit for bit.
// Positions after a row's own are masked (their weights are exactly 0).
// Fragment layouts (PTX ISA, m16n8k16 .bf16; g = lane / 4, c = lane % 4): A {(g, 2c..2c+1),
// (g+8, 2c..), (g, 2c+8..), (g+8, 2c+8..)}; B {(k 2c..2c+1, n g), (k 2c+8.., n g)}; C {(g, 2c),
// (g, 2c+1), (g+8, 2c), (g+8, 2c+1)}.
// Staging buffer: key slots of 128 bytes = eight 16-byte segments (K hi dims 0-7, 8-15, K lo
// 0-7, 8-15, V hi 0-7, 8-15, V lo 0-7, 8-15), segment s of slot k at position s ^ (k & 7) so
// that eight consecutive slots read by one ldmatrix sit on distinct banks; slots [0, n) hold the
// parent's positions, slot n + r the chunk's row r (then 15 zeroed slots, read only under the
// mask).  Then the chunk's query rows (hi 0-7, hi 8-15, lo 0-7, lo 8-15 and 16 bytes of padding
// per row: eight consecutive rows on distinct banks) and its tile table.
constexpr int CHM_THREADS = 128;
constexpr int CHM_MAX_TILES = 64;      // 16-row tiles of one chunk (chunk rows <= 64)
constexpr int CHM_QSTRIDE = 80;        // bytes per staged query row

__host__ __device__ inline int chm_buf_bytes(int n, int cap) {
    const int b = (n + cap + 15) * 128 + cap * CHM_QSTRIDE + CHM_MAX_TILES * 16;
    return (b + 127) & ~127;
}

__device__ __forceinline__ void chm_split2(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&hh);
    lo = *reinterpret_cast<const uint32_t*>(&ll);
}

__device__ __forceinline__ void chm_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                 "{%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += a b in the compensated form (small terms first)
__device__ __forceinline__ void chm_mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                                         uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    chm_mma(d, al, bh0, bh1);
    chm_mma(d, ah, bl0, bl1);
    chm_mma(d, ah, bh0, bh1);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void cp_async16_s(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Byte offset of segment `seg` of key slot `slot`.
__device__ __forceinline__ uint32_t chm_seg(int slot, int seg) {
    return (uint32_t)(((slot << 3) + (seg ^ (slot & 7))) << 4);
}

template <int MODE>
__device__ __forceinline__ void chm_store2(void* o, int64_t row, int D, int col, float x, float y) {
    __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(o);
    uint32_t hi, lo;
    chm_split2(x, y, hi, lo);
    if (MODE == ACT_BF16X2) {
        *reinterpret_cast<uint32_t*>(b + row * 2 * D + col) = hi;
        *reinterpret_cast<uint32_t*>(b + row * 2 * D + D + col) = lo;
    } else {
        *reinterpret_cast<uint32_t*>(b + row * D + col) = hi;
    }
}

struct ChmItem {
    int64_t r_lo;       // chunk's first row within the pass
    int nrows, p0;      // chunk rows, parent job (-1: none)
    int t0, nt;         // tiles: first (in the pass's list), count
};

__device__ __forceinline__ ChmItem chm_item(const int64_t* __restrict__ chunks, int64_t ck, int64_t row_base) {
    const longlong2 a = __ldg(reinterpret_cast<const longlong2*>(chunks + 4 * ck));
    const longlong2 b = __ldg(reinterpret_cast<const longlong2*>(chunks + 4 * ck + 2));
    ChmItem it;
    it.r_lo = a.x - row_base;
    it.nrows = (int)(uint32_t)(uint64_t)a.y;
    it.p0 = (int)(uint32_t)((uint64_t)a.y >> 32);
    it.t0 = (int)b.x;
    it.nt = (int)min(b.y - b.x, (long long)CHM_MAX_TILES);   // a chunk's rows (and tiles) are <= 64
    return it;
}

template <int H>
__device__ __forceinline__ void chm_stage(const ChmItem& it, int hh, uint32_t kb, uint32_t qb, uint32_t tb,
                                          const uint16_t* __restrict__ qkv, const uint16_t* __restrict__ kv,
                                          const int32_t* __restrict__ tiles, int n, int L, int l) {
    constexpr int D = H * 16, RW = 6 * D;
    // own rows: eight key/value segments (K hi at 2D, K lo 3D, V hi 4D, V lo 5D) and four query
    // segments (Q hi at 0, Q lo at D) per row
    for (int u = threadIdx.x; u < it.nrows * 12; u += CHM_THREADS) {
        const int r = u / 12, k = u - 12 * r;
        const uint16_t* row = qkv + (it.r_lo + r) * RW + hh * 16;
        if (k < 8) cp_async16_s(kb + chm_seg(n + r, k), row + 2 * D + (k >> 1) * D + (k & 1) * 8);
        else cp_async16_s(qb + r * CHM_QSTRIDE + (k - 8) * 16, row + ((k - 8) >> 1) * D + (k & 1) * 8);
    }
    for (int u = threadIdx.x; u < 15 * 8; u += CHM_THREADS)
        asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(kb + chm_seg(n + it.nrows + (u >> 3), u & 7)),
                     "r"(0u) : "memory");
    if (it.p0 >= 0) {
        const uint16_t* pre = kv + (((int64_t)it.p0 * L + l) * (int64_t)n) * 4 * D + hh * 16;
        for (int u = threadIdx.x; u < n * 8; u += CHM_THREADS) {
            const int p = u >> 3, k = u & 7;
            cp_async16_s(kb + chm_seg(p, k), pre + (int64_t)p * 4 * D + (k >> 1) * D + (k & 1) * 8);
        }
    }
    for (int u = threadIdx.x; u < it.nt; u += CHM_THREADS) cp_async16_s(tb + u * 16, tiles + 4 * (int64_t)(it.t0 + u));
}

template <int MODE, int H>
__global__ void __launch_bounds__(CHM_THREADS, 5)
ch_attention_mma_kernel(const uint16_t* __restrict__ qkv, void* __restrict__ o, int n, int cap,
                        const int64_t* __restrict__ chunks, const int64_t* __restrict__ n_chunks,
                        const int32_t* __restrict__ tiles, int64_t row_base, const uint16_t* __restrict__ kv, int L,
                        int l) {
    extern __shared__ __align__(128) uint8_t chm_sm[];
    __shared__ int grab[2];
    constexpr int DH = 16, D = H * DH;
    const int BUF = chm_buf_bytes(n, cap);
    const uint32_t sm0 = ((uint32_t)__cvta_generic_to_shared(chm_sm) + 127u) & ~127u;   // 128-byte aligned buffers
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, c = lane & 3, mj = lane >> 3, rr = lane & 7;
    const float scale = 0.25f * 1.4426950408889634f;                // rsqrt(16) log2(e)
    const int64_t items = *n_chunks * H;
    const int64_t G = gridDim.x;
    int64_t wi = blockIdx.x;
    if (wi >= items) return;
    ChmItem cur = chm_item(chunks, wi / H, row_base), nxt{};
    if (wi + G < items) nxt = chm_item(chunks, (wi + G) / H, row_base);
    chm_stage<H>(cur, (int)(wi % H), sm0, sm0 + (n + cap + 15) * 128, sm0 + (n + cap + 15) * 128 + cap * CHM_QSTRIDE,
                 qkv, kv, tiles, n, L, l);
    if (threadIdx.x == 0) grab[0] = 0;
    cp_async_commit();
    for (int k = 0; wi < items; ++k, wi += G) {
        const int b = k & 1;
        const int64_t wn = wi + G, wn2 = wi + 2 * G;
        ChmItem nx2{};
        if (wn2 < items) nx2 = chm_item(chunks, wn2 / H, row_base);
        const uint32_t kb1 = sm0 + (b ^ 1) * BUF;
        if (wn < items) {
            chm_stage<H>(nxt, (int)(wn % H), kb1, kb1 + (n + cap + 15) * 128,
                         kb1 + (n + cap + 15) * 128 + cap * CHM_QSTRIDE, qkv, kv, tiles, n, L, l);
            if (threadIdx.x == 0) grab[b ^ 1] = 0;
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        // compute item wi from buffer b
        const int hh = (int)(wi % H);
        const uint32_t kb = sm0 + b * BUF, qb = kb + (n + cap + 15) * 128, tb = qb + cap * CHM_QSTRIDE;
        for (;;) {
            int ti = 0;
            if (lane == 0) ti = atomicAdd(&grab[b], 1);
            ti = __shfl_sync(0xffffffffu, ti, 0);
            if (ti >= cur.nt) break;
            int row0, cnt, own0, st;
            asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(row0), "=r"(cnt), "=r"(own0), "=r"(st) : "r"(tb + ti * 16));
            const int t0 = st + (row0 - own0);                 // position of the tile's first row
            const int tlast = t0 + cnt - 1;
            const int ta = g < cnt ? t0 + g : tlast;           // padding rows mirror the last row
            const int tb2 = g + 8 < cnt ? t0 + g + 8 : tlast;
            uint32_t qh[4], ql[4];
            {
                const int qr = row0 + min(rr + 8 * (mj & 1), cnt - 1);
                ldsm_x4(qb + qr * CHM_QSTRIDE + (mj >> 1) * 16, qh);
                ldsm_x4(qb + qr * CHM_QSTRIDE + (2 + (mj >> 1)) * 16, ql);
            }
            float O[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            // running maxima of the raw scores q.k (the scale is folded into the exponent) and sums
            float m[2] = {-INFINITY, -INFINITY}, lsum[2] = {0.f, 0.f};
            // per-lane ldmatrix rows: K (matrices: keys 0-7 / 8-15 x dims 0-7 / 8-15), V transposed;
            // position p sits in parent slot p (p < start) or own slot n + own0 + p - start, and
            // one step (+16 positions) moves either by 16 slots = 2048 bytes (the swizzle repeats
            // every 8 slots).  The lo segment of a hi segment s is s + 2, stored at (s + 2) ^ (slot
            // & 7) = (s ^ (slot & 7)) ^ 2: the hi address with bit 5 flipped (buffers are
            // 128-byte aligned).
            const int pk0 = rr + 8 * (mj >> 1), pv0 = rr + 8 * (mj & 1);
            const uint32_t kpar = kb + chm_seg(pk0, mj & 1), vpar = kb + chm_seg(pv0, 4 + (mj >> 1));
            const int ok0 = n + own0 - st;                     // own slot of position p: ok0 + p (>= 1)
            const uint32_t kown = kb + chm_seg(ok0 + pk0, mj & 1);
            const uint32_t vown = kb + chm_seg(ok0 + pv0, 4 + (mj >> 1));
            for (int pb = 0; pb <= tlast; pb += 16) {
                const uint32_t ka = (pb + pk0 < st ? kpar : kown) + (uint32_t)pb * 128;
                const uint32_t va = (pb + pv0 < st ? vpar : vown) + (uint32_t)pb * 128;
                uint32_t kh[4], kl[4];
                ldsm_x4(ka, kh);
                ldsm_x4(ka ^ 32u, kl);           // K lo
                float S[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                chm_mma3(S[0], qh, ql, kh[0], kh[1], kl[0], kl[1]);
                chm_mma3(S[1], qh, ql, kh[2], kh[3], kl[2], kl[3]);
                if (pb + 15 > t0) {               // the causal edge runs through this step
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int ee = 0; ee < 2; ++ee) {
                            const int p = pb + 8 * nt + 2 * c + ee;
                            if (p > ta) S[nt][ee] = -INFINITY;
                            if (p > tb2) S[nt][2 + ee] = -INFINITY;
                        }
                }
                float mx[2];
                mx[0] = fmaxf(fmaxf(S[0][0], S[0][1]), fmaxf(S[1][0], S[1][1]));
                mx[1] = fmaxf(fmaxf(S[0][2], S[0][3]), fmaxf(S[1][2], S[1][3]));
                float ms[2];
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    mx[hf] = fmaxf(mx[hf], __shfl_xor_sync(0xffffffffu, mx[hf], 1));
                    mx[hf] = fmaxf(mx[hf], __shfl_xor_sync(0xffffffffu, mx[hf], 2));
                    if (mx[hf] > m[hf]) {
                        const float cr = ex2_approx((m[hf] - mx[hf]) * scale);   // 0 on the first step
                        lsum[hf] *= cr;
                        O[0][2 * hf] *= cr; O[0][2 * hf + 1] *= cr;
                        O[1][2 * hf] *= cr; O[1][2 * hf + 1] *= cr;
                        m[hf] = mx[hf];
                    }
                    ms[hf] = -m[hf] * scale;
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int ee = 0; ee < 2; ++ee) {
                        S[nt][ee] = ex2_approx(fmaf(S[nt][ee], scale, ms[0]));
                        S[nt][2 + ee] = ex2_approx(fmaf(S[nt][2 + ee], scale, ms[1]));
                        lsum[0] += S[nt][ee];
                        lsum[1] += S[nt][2 + ee];
                    }
                uint32_t ph[4], pl[4];
                chm_split2(S[0][0], S[0][1], ph[0], pl[0]);
                chm_split2(S[0][2], S[0][3], ph[1], pl[1]);
                chm_split2(S[1][0], S[1][1], ph[2], pl[2]);
                chm_split2(S[1][2], S[1][3], ph[3], pl[3]);
                uint32_t vh[4], vl[4];
                ldsm_x4_t(va, vh);
                ldsm_x4_t(va ^ 32u, vl);         // V lo
                chm_mma3(O[0], ph, pl, vh[0], vh[1], vl[0], vl[1]);
                chm_mma3(O[1], ph, pl, vh[2], vh[3], vl[2], vl[3]);
            }
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                lsum[hf] += __shfl_xor_sync(0xffffffffu, lsum[hf], 1);
                lsum[hf] += __shfl_xor_sync(0xffffffffu, lsum[hf], 2);
            }
            const float ia = 1.f / lsum[0], ib = 1.f / lsum[1];
#pragma unroll
            for (int n2 = 0; n2 < 2; ++n2) {
                const int col = hh * DH + 8 * n2 + 2 * c;
                if (g < cnt) chm_store2<MODE>(o, cur.r_lo + row0 + g, D, col, O[n2][0] * ia, O[n2][1] * ia);
                if (g + 8 < cnt) chm_store2<MODE>(o, cur.r_lo + row0 + g + 8, D, col, O[n2][2] * ib, O[n2][3] * ib);
            }
        }
        __syncthreads();
        cur = nxt;
        nxt = nx2;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- heads
// LNf of row `row` and its output-head logit at position t (the whole warp; every lane gets it).
template <int DPL>
__device__ __forceinline__ void lnf_row(const ModelConst& mc, const float* __restrict__ P, const float* __restrict__ h,
                                        int64_t row, int lane, float (&y)[DPL]) {
    const int d = mc.hidden;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) { y[i] = h[row * d + lane + 32 * i]; s += y[i]; }
    const float inv_d = 1.f / (float)d;
    const float mu = warp_sum(s) * inv_d;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) { const float c = y[i] - mu; q += c * c; }
    const float rstd = rsqrtf(fmaf(warp_sum(q), inv_d, LN_EPS));
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        y[i] = (y[i] - mu) * rstd * P[mc.lnf_g + j] + P[mc.lnf_b + j];
    }
}

// Two rows at once, each with exactly the arithmetic of lnf_row / head_logit (the same butterfly
// per value), so that the two rows' reductions overlap instead of following each other.
__device__ __forceinline__ void warp_sum2(float& a, float& b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
}

template <int DPL>
__device__ __forceinline__ void lnf_row2(const ModelConst& mc, const float* __restrict__ P, const float* __restrict__ h,
                                         int64_t row0, int64_t row1, int lane, float (&y0)[DPL], float (&y1)[DPL]) {
    const int d = mc.hidden;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        y0[i] = h[row0 * d + lane + 32 * i]; s0 += y0[i];
        y1[i] = h[row1 * d + lane + 32 * i]; s1 += y1[i];
    }
    const float inv_d = 1.f / (float)d;
    warp_sum2(s0, s1);
    const float mu0 = s0 * inv_d, mu1 = s1 * inv_d;
    float q0 = 0.f, q1 = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const float c0 = y0[i] - mu0, c1 = y1[i] - mu1;
        q0 += c0 * c0;
        q1 += c1 * c1;
    }
    warp_sum2(q0, q1);
    const float r0 = rsqrtf(fmaf(q0, inv_d, LN_EPS)), r1 = rsqrtf(fmaf(q1, inv_d, LN_EPS));
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const int j = lane + 32 * i;
        const float g = P[mc.lnf_g + j], bb = P[mc.lnf_b + j];
        y0[i] = (y0[i] - mu0) * r0 * g + bb;
        y1[i] = (y1[i] - mu1) * r1 * g + bb;
    }
}

template <int DPL>
__device__ __forceinline__ void head_logit2(const ModelConst& mc, const float* __restrict__ P, const float (&y0)[DPL],
                                            const float (&y1)[DPL], int lane, int t, float& a0, float& a1) {
    a0 = 0.f; a1 = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) {
        const float w = P[mc.head_w + lane + 32 * i];
        a0 = fmaf(y0[i], w, a0);
        a1 = fmaf(y1[i], w, a1);
    }
    warp_sum2(a0, a1);
    a0 += P[mc.head_b + t];
    a1 += P[mc.head_b + t + 1];
}

template <int DPL>
__device__ __forceinline__ float head_logit(const ModelConst& mc, const float* __restrict__ P, const float (&y)[DPL],
                                            int lane, int t) {
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) a = fmaf(y[i], P[mc.head_w + lane + 32 * i], a);
    return warp_sum(a) + P[mc.head_b + t];
}

template <int DPL>
__device__ __forceinline__ float phase_dot(const ModelConst& mc, const float* __restrict__ P, const float (&y)[DPL],
                                           int lane, int sel) {
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < DPL; ++i) a = fmaf(y[i], P[mc.phase_w + sel * mc.hidden + lane + 32 * i], a);
    return warp_sum(a) + P[mc.phase_b + sel];
}

// Hamming-weight constraint of position t given the same-spin ones before it (Eq. modifier):
// 1 forced one, -1 forced zero, 0 free.
__device__ __forceinline__ int forced_at(const ModelConst& mc, int t, int ones_same) {
    const int need = (mc.order[t] & 1) ? mc.n_dn : mc.n_up;
    if (ones_same + mc.after[t] < need) return 1;
    if (ones_same >= need) return -1;
    return 0;
}

// Log-probability term of position t with bit b: 0 when forced and consistent, -inf when forced
// and violated, log-sigmoid of the logit otherwise.
__device__ __forceinline__ float lp_term(int forced, int b, float logit) {
    if (forced == 1) return b ? 0.f : -INFINITY;
    if (forced == -1) return b ? -INFINITY : 0.f;
    return logsig(b ? logit : -logit);
}

struct ChainView {   // per pass-A job: full-view arrays
    float2* cum;     // [jobs][n + 1] TwoSum prefix sums of the log-probability terms
    float* logit;    // [jobs][n]
    float* ph4;      // [jobs][4] phase-head outputs of the row at position n - 2
};

__device__ __forceinline__ void add_lp(float& s, float& e, bool& bad, float lp, int compensated) {
    if (lp == -INFINITY) { bad = true; return; }
    if (compensated) two_sum_acc(s, e, lp); else s += lp;
}

// Pass-A heads of jobs [j0, j1) of one level (their parents' views complete): one warp per job.
// Level-0 jobs also give the samples' log|psi| and phase.
template <int DPL>
__global__ void __launch_bounds__(256)
ch_chain_heads_kernel(ModelConst mc, const float* __restrict__ P, const float* __restrict__ h, int64_t j0, int64_t j1,
                      const uint64_t* __restrict__ jbits, const int32_t* __restrict__ jstart,
                      const int32_t* __restrict__ jpar, const int64_t* __restrict__ joff, ChainView V,
                      int64_t nb, float* __restrict__ la_x, float* __restrict__ ph_x) {
    const int n = mc.n, lane = threadIdx.x & 31;
    const int64_t j = j0 + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= j1) return;
    const uint64_t x = jbits[j];
    const int s0 = jstart[j];
    const int64_t par = jpar[j];
    float2* cum = V.cum + j * (int64_t)(n + 1);
    float* lg = V.logit + j * (int64_t)n;
    // inherited positions
    for (int t = lane; t < s0 && par >= 0; t += 32) {
        cum[t] = V.cum[par * (n + 1) + t];
        lg[t] = V.logit[par * (int64_t)n + t];
    }
    float s = 0.f, e = 0.f;
    bool bad = false;
    int ones[2] = {0, 0};
    for (int t = 0; t < s0 - 1; ++t) ones[mc.order[t] & 1] += (int)((x >> mc.order[t]) & 1ull);
    if (par >= 0 && s0 >= 1) {
        const float2 c = V.cum[par * (n + 1) + s0 - 1];
        s = c.x; e = c.y;
        bad = c.x == -INFINITY;
        const int t = s0 - 1, b = (int)((x >> mc.order[t]) & 1ull);
        add_lp(s, e, bad, lp_term(forced_at(mc, t, ones[mc.order[t] & 1]), b, V.logit[par * (int64_t)n + t]),
               mc.compensated);
        ones[mc.order[t] & 1] += b;
    }
    if (lane == 0) cum[s0] = bad ? make_float2(-INFINITY, 0.f) : make_float2(s, e);
    for (int t = s0; t < n; ++t) {
        float y[DPL];
        lnf_row<DPL>(mc, P, h, joff[j] + t - s0, lane, y);
        const float a = head_logit<DPL>(mc, P, y, lane, t);
        const int b = (int)((x >> mc.order[t]) & 1ull);
        add_lp(s, e, bad, lp_term(forced_at(mc, t, ones[mc.order[t] & 1]), b, a), mc.compensated);
        ones[mc.order[t] & 1] += b;
        if (t == n - 2) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float ph = phase_dot<DPL>(mc, P, y, lane, k);
                if (lane == 0) V.ph4[j * 4 + k] = ph;
            }
        }
        if (lane == 0) {
            lg[t] = a;
            cum[t + 1] = bad ? make_float2(-INFINITY, 0.f) : make_float2(s, e);
        }
    }
    if (s0 > n - 2 && lane < 4) V.ph4[j * 4 + lane] = V.ph4[par * 4 + lane];
    if (j < nb && lane == 0) {   // a sample (its phase-head outputs were written by this lane)
        la_x[j] = bad ? -INFINITY : 0.5f * (s + e);
        const int sel = (int)(((x >> mc.order[n - 2]) & 1ull) * 2 + ((x >> mc.order[n - 1]) & 1ull));
        ph_x[j] = V.ph4[j * 4 + sel];
    }
}

// Pass-B heads: one warp per leaf; the leaf's log psi from its parent's view and its own rows,
// then its ratio-weighted contribution S f(x')/f(x) (the diagonal row: S).  With `order`, the
// leaves of slots [i0, i1) of a sub-pass (own rows from slot offsets soff - row_base); without,
// every leaf r in [i0, i1) that has no own rows (the diagonal, and branches at the last position).
template <int DPL>
__global__ void __launch_bounds__(256)
ch_leaf_heads_kernel(ModelConst mc, const float* __restrict__ P, const float* __restrict__ h, int64_t i0, int64_t i1,
                     const int32_t* __restrict__ order, const int64_t* __restrict__ soff, int64_t row_base,
                     const uint64_t* __restrict__ xprime, const int32_t* __restrict__ lstart,
                     const int32_t* __restrict__ lpar, const int64_t* __restrict__ lrows, ChainView V,
                     const uint64_t* __restrict__ xs, int64_t nb, const int64_t* __restrict__ seg, int64_t seg_stride,
                     const float* __restrict__ la_x, const float* __restrict__ ph_x, const float4* __restrict__ S,
                     float2* __restrict__ contrib, const int64_t* __restrict__ rows_dev) {
    const int n = mc.n, lane = threadIdx.x & 31;
    const int64_t slot = i0 + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (slot >= i1) return;
    if (!order && (slot >= *rows_dev || lrows[slot] > 0)) return;
    const int64_t r = order ? order[slot] : slot;
    const int64_t i = seg_of(seg, seg_stride, nb, r);
    const uint64_t x = xprime[r];
    const float4 s4 = S[r];
    const float sre = s4.x + s4.y, sim = s4.z + s4.w;
    if (x == xs[i]) {
        if (lane == 0) contrib[r] = make_float2(sre, sim);
        return;
    }
    const int s0 = lstart[r];
    const int64_t par = lpar[r];
    float s = 0.f, e = 0.f;
    bool bad = false;
    int ones[2] = {0, 0};
    for (int t = 0; t < s0 - 1; ++t) ones[mc.order[t] & 1] += (int)((x >> mc.order[t]) & 1ull);
    if (par >= 0 && s0 >= 1) {
        const float2 c = V.cum[par * (n + 1) + s0 - 1];
        s = c.x; e = c.y;
        bad = c.x == -INFINITY;
        const int t = s0 - 1, b = (int)((x >> mc.order[t]) & 1ull);
        add_lp(s, e, bad, lp_term(forced_at(mc, t, ones[mc.order[t] & 1]), b, V.logit[par * (int64_t)n + t]),
               mc.compensated);
        ones[mc.order[t] & 1] += b;
    }
    const int sel = (int)(((x >> mc.order[n - 2]) & 1ull) * 2 + ((x >> mc.order[n - 1]) & 1ull));
    float phase = s0 > n - 2 ? V.ph4[par * 4 + sel] : 0.f;
    const int64_t q0 = order ? soff[slot] - row_base : 0;
    int t = s0;
    for (; t + 1 < n; t += 2) {          // two positions per iteration, accumulated in order
        float y0[DPL], y1[DPL], a0, a1;
        lnf_row2<DPL>(mc, P, h, q0 + t - s0, q0 + t + 1 - s0, lane, y0, y1);
        head_logit2<DPL>(mc, P, y0, y1, lane, t, a0, a1);
        const int b0 = (int)((x >> mc.order[t]) & 1ull);
        add_lp(s, e, bad, lp_term(forced_at(mc, t, ones[mc.order[t] & 1]), b0, a0), mc.compensated);
        ones[mc.order[t] & 1] += b0;
        if (t == n - 2) phase = phase_dot<DPL>(mc, P, y0, lane, sel);
        const int b1 = (int)((x >> mc.order[t + 1]) & 1ull);
        add_lp(s, e, bad, lp_term(forced_at(mc, t + 1, ones[mc.order[t + 1] & 1]), b1, a1), mc.compensated);
        ones[mc.order[t + 1] & 1] += b1;
        if (t + 1 == n - 2) phase = phase_dot<DPL>(mc, P, y1, lane, sel);
    }
    if (t < n) {
        float y[DPL];
        lnf_row<DPL>(mc, P, h, q0 + t - s0, lane, y);
        const float a = head_logit<DPL>(mc, P, y, lane, t);
        const int b = (int)((x >> mc.order[t]) & 1ull);
        add_lp(s, e, bad, lp_term(forced_at(mc, t, ones[mc.order[t] & 1]), b, a), mc.compensated);
        ones[mc.order[t] & 1] += b;
        if (t == n - 2) phase = phase_dot<DPL>(mc, P, y, lane, sel);
    }
    if (lane != 0) return;
    const float la = bad ? -INFINITY : 0.5f * (s + e);
    const float mag = expf(la - la_x[i]);
    float sn, cs;
    sincosf(phase - ph_x[i], &sn, &cs);
    const float rr = mag * cs, ri = mag * sn;
    contrib[r] = make_float2(sre * rr - sim * ri, sre * ri + sim * rr);
}

template <class F>
int with_dpl_c(int d, F&& f) {
    switch (d / 32) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 8: return f(std::integral_constant<int, 8>{});
        default: set_error("d_model must be 32, 64, 128 or 256"); return NQS_ERR_UNSUPPORTED;
    }
}

// Rows of one attention chunk at most (a chunk holds whole jobs of one parent; a job has <= n rows).
inline int ch_chunk_cap(int n) { return std::max(n, 48); }

inline int grid_for(int64_t n, int per, int cap_per_sm = 16) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, (int64_t)num_sms() * cap_per_sm));
}

template <int MODE, int DH, int H>
size_t ch_attention_smem(int n) {
    constexpr int HG = H < CH_ATT_HG ? H : CH_ATT_HG;
    return (size_t)(n + ch_chunk_cap(n)) * (HG * (2 * DH + 4) + 4) * sizeof(float);
}

template <int MODE, int DH, int H>
int ch_attention_launch(const ModelConst& mc, const float* qkv, void* o, const int64_t* chunks, const int64_t* n_chunks,
                        int64_t max_chunks, int64_t row_base, const uint8_t* rpos, const uint8_t* rstart,
                        const float* kv, int l, cudaStream_t s) {
    const int n = mc.n;
    const size_t smem = ch_attention_smem<MODE, DH, H>(n);
    static int configured = -1;
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (configured != dev) {
        NQS_CK(cudaFuncSetAttribute(ch_attention_kernel<MODE, DH, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    220 * 1024));
        configured = dev;
    }
    if (smem > 220 * 1024) { set_error("prefix-sharing attention: staging exceeds shared memory"); return NQS_ERR_UNSUPPORTED; }
    const int per_sm = std::max(1, std::min(6, (int)((227 * 1024) / (smem + 1024))));
    constexpr int GROUPS = H < CH_ATT_HG ? 1 : H / CH_ATT_HG;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(max_chunks * GROUPS, (int64_t)num_sms() * per_sm));
    ch_attention_kernel<MODE, DH, H><<<grid, CH_ATT_THREADS, smem, s>>>(qkv, o, n, chunks, n_chunks, row_base, rpos,
                                                                       rstart, kv, mc.layers, l);
    NQS_LAUNCHED();
    return NQS_OK;
}

// Tensor-path attention over the split layout (bf16 forms, head size 16).
template <int MODE, int H>
int ch_attention_mma_launch(const ModelConst& mc, const void* qkv, void* o, const int64_t* chunks,
                            const int64_t* n_chunks, int64_t max_chunks, const int32_t* tiles, int64_t row_base,
                            const void* kv, int l, cudaStream_t s) {
    const int n = mc.n, cap = ch_chunk_cap(n);
    const size_t smem = 2 * (size_t)chm_buf_bytes(n, cap) + 128;
    static int configured = -1;
    int dev = 0;
    NQS_CK(cudaGetDevice(&dev));
    if (configured != dev) {
        NQS_CK(cudaFuncSetAttribute(ch_attention_mma_kernel<MODE, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    220 * 1024));
        configured = dev;
    }
    if (smem > 220 * 1024 || cap > CHM_MAX_TILES) {
        set_error("prefix-sharing attention: staging exceeds shared memory");
        return NQS_ERR_UNSUPPORTED;
    }
    const int per_sm = std::max(1, std::min(5, (int)((227 * 1024) / (smem + 1024))));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(max_chunks * H, (int64_t)num_sms() * per_sm));
    ch_attention_mma_kernel<MODE, H><<<grid, CHM_THREADS, smem, s>>>(
        reinterpret_cast<const uint16_t*>(qkv), o, n, cap, chunks, n_chunks, tiles, row_base,
        reinterpret_cast<const uint16_t*>(kv), mc.layers, l);
    NQS_LAUNCHED();
    return NQS_OK;
}

// The attention of a pass: the tensor path for the bf16 forms with head size 16 (q, k, v and the
// caches in the split layout), else the CUDA-core kernel (fp32 layout).
template <int MODE>
bool ch_split_qkv(const ModelConst& mc) {
    return (MODE == ACT_BF16 || MODE == ACT_BF16X2) && mc.hidden == 16 * mc.heads &&
           (mc.heads == 1 || mc.heads == 2 || mc.heads == 4 || mc.heads == 8);
}

template <int MODE>
int ch_attention(const ModelConst& mc, const float* qkv, void* o, const int64_t* chunks, const int64_t* n_chunks,
                 int64_t max_chunks, const int32_t* tiles, int64_t row_base, const uint8_t* rpos,
                 const uint8_t* rstart, const float* kv, int l, cudaStream_t s) {
    if (max_chunks <= 0) return NQS_OK;
    const int H = mc.heads, dh = mc.hidden / mc.heads;
    if constexpr (MODE == ACT_BF16 || MODE == ACT_BF16X2) {
        if (ch_split_qkv<MODE>(mc)) {
#define CH_MMA(H_)                                                                                                \
            if (H == H_) return ch_attention_mma_launch<MODE, H_>(mc, qkv, o, chunks, n_chunks, max_chunks, tiles,  \
                                                                  row_base, kv, l, s);
            CH_MMA(1) CH_MMA(2) CH_MMA(4) CH_MMA(8)
#undef CH_MMA
        }
    }
#define CH_ATT(DH_, H_)                                                                                           \
    if (dh == DH_ && H == H_)                                                                                     \
        return ch_attention_launch<MODE, DH_, H_>(mc, qkv, o, chunks, n_chunks, max_chunks, row_base, rpos,       \
                                                  rstart, kv, l, s);
    CH_ATT(16, 1) CH_ATT(16, 2) CH_ATT(16, 4) CH_ATT(16, 8) CH_ATT(32, 1) CH_ATT(32, 2) CH_ATT(32, 4) CH_ATT(32, 8)
#undef CH_ATT
    set_error("prefix-sharing attention: head size 16 or 32 with 1, 2, 4 or 8 heads");
    return NQS_ERR_UNSUPPORTED;
}

}  // namespace

// ---------------------------------------------------------------- host side
bool chain_supported(const ModelConst& mc) {
    const int H = mc.heads, dh = mc.hidden / std::max(1, mc.heads);
    const int HG = H < CH_ATT_HG ? H : CH_ATT_HG;
    const size_t smem = (size_t)(mc.n + ch_chunk_cap(mc.n)) * (HG * (2 * dh + 4) + 4) * sizeof(float);
    return mc.arch == NQS_ARCH_TRANSFORMER && (dh == 16 || dh == 32) && (H == 1 || H == 2 || H == 4 || H == 8) &&
           smem <= 220 * 1024;
}

int64_t chain_jobs_per_sample(const ModelConst& mc, int depth) {
    const int64_t n = mc.n;
    return 1 + (depth >= 2 ? n : 0) + (depth >= 3 ? n * (n - 1) / 2 : 0);
}

// Rows of the pass-A jobs of one sample at most: n for x, n - 1 - f for the level-1 job of f,
// n - 1 - f2 for the level-2 job (f1, f2).
static int64_t chain_rows_per_sample(const ModelConst& mc, int depth) {
    const int64_t n = mc.n;
    int64_t r = n;
    if (depth >= 2) r += n * (n - 1) / 2;
    if (depth >= 3)
        for (int64_t f2 = 1; f2 < n; ++f2) r += f2 * (n - 1 - f2);
    return r;
}

int64_t chain_chunk(const ModelConst& mc, int depth) {
    const int64_t per = chain_jobs_per_sample(mc, depth) * mc.layers * mc.n * 2 * mc.hidden * 4;
    return std::max<int64_t>(1, std::min<int64_t>(CHAIN_MAX_CHUNK, CHAIN_CACHE_BYTES / per));
}

// Rows of one pass: all of pass A, and pass-B sub-passes of about pass_bytes of activations
// (about 40 d bytes a row; 0: CHAIN_PASS_BYTES), never more than the chunk's leaves can need.
int64_t chain_pass_rows(const ModelConst& mc, int depth, int64_t chunk, int64_t rows_cap, int64_t pass_bytes) {
    const int64_t rows_a = chunk * chain_rows_per_sample(mc, depth);
    const int64_t pb = pass_bytes > 0 ? pass_bytes : CHAIN_PASS_BYTES;
    const int64_t rows_b = std::min<int64_t>(std::max<int64_t>(pb / ((int64_t)mc.hidden * 40), 4 * (int64_t)mc.n),
                                             rows_cap * mc.n + mc.n);
    return std::max(rows_a, rows_b);
}

void chain_layout(Carver& c, const ModelConst& mc, int depth, int64_t chunk, int64_t rows_cap, int64_t pass_bytes,
                  ChainBufs& b) {
    const int64_t n = mc.n;
    b.chunk = chunk;
    b.rows_cap = rows_cap;
    b.jobs_cap = chunk * chain_jobs_per_sample(mc, depth);
    b.pass_rows = chain_pass_rows(mc, depth, chunk, rows_cap, pass_bytes);
    b.l1 = c.take<unsigned long long>(chunk);
    b.l2 = c.take<unsigned long long>(chunk * 64);
    b.cnt1 = c.take<int64_t>(chunk);
    b.cnt2 = c.take<int64_t>(chunk);
    b.base1 = c.take<int64_t>(chunk + 1);
    b.base2 = c.take<int64_t>(chunk + 1);
    b.cum2 = c.take<int32_t>(chunk * 64);
    b.jbits = c.take<uint64_t>(b.jobs_cap);
    b.jstart = c.take<int32_t>(b.jobs_cap);
    b.jpar = c.take<int32_t>(b.jobs_cap);
    b.jrows = c.take<int64_t>(b.jobs_cap);
    b.joff = c.take<int64_t>(b.jobs_cap + 1);
    b.jseg = c.take<int64_t>(b.jobs_cap);
    b.lpar = c.take<int32_t>(rows_cap);
    b.lstart = c.take<int32_t>(rows_cap);
    b.lrows = c.take<int64_t>(rows_cap);
    b.lorder = c.take<int32_t>(rows_cap);
    b.srows = c.take<int64_t>(rows_cap);
    b.soff = c.take<int64_t>(rows_cap + 1);
    b.sseg = c.take<int64_t>(rows_cap);
    b.hist = c.take<unsigned long long>(b.jobs_cap + 1);
    b.hoff = c.take<int64_t>(b.jobs_cap + 2);
    b.kv = c.take<float>(b.jobs_cap * mc.layers * n * 2 * mc.hidden);
    b.cum = c.take<float2>(b.jobs_cap * (n + 1));
    b.logit = c.take<float>(b.jobs_cap * n);
    b.ph4 = c.take<float>(b.jobs_cap * 4);
    b.rjob = c.take<int32_t>(b.pass_rows);
    b.rpos = c.take<uint8_t>(b.pass_rows);
    b.rstart = c.take<uint8_t>(b.pass_rows);
    const int64_t max_slots = std::max(b.jobs_cap, rows_cap);
    b.ccnt = c.take<int64_t>(max_slots);
    b.coff = c.take<int64_t>(max_slots + 1);
    b.tcnt = c.take<int64_t>(max_slots);
    b.toff = c.take<int64_t>(max_slots + 1);
    b.chunks = c.take<int64_t>(4 * max_slots);
    // 16-row tiles of one pass: at most one per 16 rows plus one per job
    b.tiles = c.take<int32_t>(4 * (b.pass_rows / 16 + max_slots + 1));
    b.split = c.take<int64_t>(CHAIN_MAX_SPLIT + 1);
    b.split_off = c.take<int64_t>(CHAIN_MAX_SPLIT + 1);
    tf_layout(c, mc, (b.pass_rows + n - 1) / n, b.tf);
}

// One layer-by-layer forward over the pass's M rows (table rjob / rpos, job strings jbits);
// pass A (jobs of levels 0..2, level boundaries lev[]) also fills the caches.
template <int MODE>
static int ch_forward(const ModelConst& mc, const float* P, const TfWeights& w, ChainBufs& b, const uint64_t* jbits,
                      int64_t M, bool pass_a, const int64_t* lev, int64_t j0, int64_t j1, const int32_t* order,
                      const int32_t* jstart, const int32_t* jpar, const int64_t* joff, const int64_t* segend,
                      int64_t row_base, cudaStream_t s) {
    const int d = mc.hidden, n = mc.n;
    TfBufs& t = b.tf;
    return with_dpl_c(d, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        const double act_b = MODE == ACT_BF16 ? 2.0 : 4.0;
        const double ln_bytes = (double)M * d * (4.0 + act_b);
        // attention FLOPs for the profile (query . key and weight . value, 2d each per row and key
        // 0..t): from the pass's position table, read back only while profiling
        double att_flops = 0.0;
        if (prof_enabled() && M > 0) {
            std::vector<uint8_t> pos((size_t)M);
            NQS_CK(cudaMemcpyAsync(pos.data(), b.rpos, (size_t)M, cudaMemcpyDeviceToHost, s));
            NQS_CK(cudaStreamSynchronize(s));
            double keys = 0.0;
            for (uint8_t t : pos) keys += (double)t + 1.0;
            att_flops = 4.0 * d * keys;
        }
        if (M > 0) {
            ProfScope ps("tf_layernorm", s, 0.0, ln_bytes);
            ch_embed_ln_kernel<MODE, DPL><<<ln_grid(M), 256, 0, s>>>(mc, P, jbits, b.rjob, b.rpos, M, t.h, t.a);
            NQS_LAUNCHED();
        }
        // the attention's chunk list (shared by every layer)
        const int64_t nsl = j1 - j0;
        if (M > 0) {
            ProfScope ps("ch_build", s);
            const int cap = ch_chunk_cap(n);
            ch_chunk_count_kernel<<<grid_for(nsl, 256), 256, 0, s>>>(joff, segend, nullptr, j0, j1, cap, b.ccnt, b.tcnt);
            NQS_LAUNCHED();
            NQS_TRY(launch_scan_i64(b.ccnt, nsl, nullptr, b.coff, s));
            NQS_TRY(launch_scan_i64(b.tcnt, nsl, nullptr, b.toff, s));
            ch_chunk_write_kernel<<<grid_for(nsl, 256), 256, 0, s>>>(joff, segend, nullptr, j0, j1, cap, b.coff, b.toff,
                                                                     order, jstart, jpar, b.chunks, b.tiles);
            NQS_LAUNCHED();
        }
        // q, k, v (and so the caches) in the split layout where the tensor-path attention runs
        const int qkv_epi = ch_split_qkv<MODE>(mc) ? TF_EPI_SPLIT : TF_EPI_STORE;
        for (int l = 0; l < mc.layers; ++l) {
            if (M > 0) NQS_TRY(tf_gemm(mc, w, TF_WQKV, l, t.a, t.qkv, M, 3 * d, d, qkv_epi, P + mc.bqkv[l], s));
            if (pass_a) {
                ProfScope ps("ch_cache", s, 0.0, (double)(lev[3]) * n * 2 * d * 4 * 2);
                for (int v = 0; v < 3; ++v) {
                    if (lev[v + 1] <= lev[v]) continue;
                    ch_cache_fill_kernel<<<grid_for(lev[v + 1] - lev[v], 1, 8), 256, 0, s>>>(
                        b.kv, mc.layers, l, n, d, lev[v], lev[v + 1], jstart, jpar, joff, t.qkv);
                    NQS_LAUNCHED();
                }
            }
            if (M > 0) {
                {
                    ProfScope ps("ch_attention", s, att_flops, (double)M * 3 * d * 4 + (double)M * d * act_b);
                    NQS_TRY(ch_attention<MODE>(mc, t.qkv, t.o, b.chunks, b.coff + nsl, nsl, b.tiles, row_base, b.rpos,
                                               b.rstart, b.kv, l, s));
                }
                if (MODE == ACT_BF16X2 && (d == 64 || d == 128)) {
                    // attention output + residual + LayerNorm 2 in one tensor-core kernel
                    NQS_TRY(tf_resid_ln(mc, P, w, l, t.o, t.h, t.a, M, s));
                } else {
                    NQS_TRY(tf_gemm(mc, w, TF_WO, l, t.o, t.h, M, d, d, TF_EPI_RESID, P + mc.bo[l], s));
                    ProfScope ps2("tf_layernorm", s, 0.0, ln_bytes);
                    layernorm_kernel<MODE, DPL><<<ln_grid(M), 256, 0, s>>>(t.h, M, d, P + mc.ln2_g[l], P + mc.ln2_b[l], t.a);
                    NQS_LAUNCHED();
                }
                NQS_TRY(tf_mlp(mc, P, w, l, t.a, t.mid, t.h, M, s));
                if (l + 1 < mc.layers) {
                    ProfScope ps3("tf_layernorm", s, 0.0, ln_bytes);
                    layernorm_kernel<MODE, DPL><<<ln_grid(M), 256, 0, s>>>(t.h, M, d, P + mc.ln1_g[l + 1], P + mc.ln1_b[l + 1], t.a);
                    NQS_LAUNCHED();
                }
            }
        }
        return NQS_OK;
    });
}

template <int MODE>
static int ch_local_energy_mode(const ModelConst& mc, const float* P, const TfWeights& w, ChainBufs& b, int depth,
                                const uint64_t* xs, int64_t nb, const int64_t* seg, int64_t seg_stride,
                                const uint64_t* xprime, const float4* S, const int64_t* rows_dev, int64_t rows_max,
                                float* la_x, float* ph_x, float2* contrib, cudaStream_t s) {
    const int n = mc.n, d = mc.hidden;
    {
        ProfScope ps("ch_build", s);
        NQS_CK(cudaMemsetAsync(b.l1, 0, (size_t)nb * 8, s));
        NQS_CK(cudaMemsetAsync(b.l2, 0, (size_t)nb * 64 * 8, s));
        ch_mark_kernel<<<grid_for(rows_max, 256), 256, 0, s>>>(mc, xs, nb, seg, seg_stride, xprime, rows_dev, rows_max,
                                                               depth, b.l1, b.l2);
        NQS_LAUNCHED();
        ch_count_kernel<<<(unsigned)((nb + 7) / 8), 256, 0, s>>>(b.l1, b.l2, nb, b.cnt1, b.cnt2, b.cum2);
        NQS_LAUNCHED();
        NQS_TRY(launch_scan_i64(b.cnt1, nb, nullptr, b.base1, s));
        NQS_TRY(launch_scan_i64(b.cnt2, nb, nullptr, b.base2, s));
        ch_jobs_kernel<<<(unsigned)((nb * n + 255) / 256), 256, 0, s>>>(mc, xs, nb, b.l1, b.l2, b.base1, b.base2, b.cum2, b.jbits,
                                                                 b.jstart, b.jpar, b.jrows, b.jseg);
        NQS_LAUNCHED();
        ch_leaf_kernel<<<grid_for(rows_max, 256), 256, 0, s>>>(mc, xs, nb, seg, seg_stride, xprime, rows_dev, rows_max,
                                                               depth, b.l1, b.l2, b.base1, b.base2, b.cum2, b.lpar,
                                                               b.lstart, b.lrows);
        NQS_LAUNCHED();
    }
    // host: level sizes (jobs = nb + base1[nb] + base2[nb]), then the row offsets of the jobs
    // and of the leaves
    int64_t h2[2] = {0, 0};
    NQS_CK(cudaMemcpyAsync(h2, b.base1 + nb, 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaMemcpyAsync(h2 + 1, b.base2 + nb, 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    const int64_t lev[4] = {0, nb, nb + h2[0], nb + h2[0] + h2[1]};
    const int64_t jobs = lev[3];
    if (jobs > b.jobs_cap) { set_error("prefix-sharing jobs exceed the workspace"); return NQS_ERR_CAPACITY; }
    NQS_TRY(launch_scan_i64(b.jrows, jobs, nullptr, b.joff, s));
    int64_t hrows[2] = {0, 0};
    NQS_CK(cudaMemcpyAsync(hrows, b.joff + jobs, 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaMemcpyAsync(hrows + 1, rows_dev, 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    const int64_t rows_a = hrows[0];
    const int64_t rows = std::min(hrows[1], rows_max);
    if (rows_a > b.pass_rows) { set_error("prefix-sharing pass A exceeds the workspace"); return NQS_ERR_CAPACITY; }

    ChainView V{b.cum, b.logit, b.ph4};
    // pass A
    ch_rows_kernel<<<grid_for(jobs, 256), 256, 0, s>>>(b.joff, nullptr, b.jstart, 0, jobs, 0, n, b.rjob, b.rpos, b.rstart);
    NQS_LAUNCHED();
    NQS_TRY(ch_forward<MODE>(mc, P, w, b, b.jbits, rows_a, true, lev, 0, jobs, nullptr, b.jstart, b.jpar, b.joff,
                             b.jseg, 0, s));
    NQS_TRY(with_dpl_c(d, [&](auto dpl) -> int {
        constexpr int DPL = decltype(dpl)::value;
        ProfScope ps("ch_heads", s);
        for (int v = 0; v < 3; ++v) {
            if (lev[v + 1] <= lev[v]) continue;
            ch_chain_heads_kernel<DPL><<<(unsigned)((lev[v + 1] - lev[v] + 7) / 8), 256, 0, s>>>(
                mc, P, b.tf.h, lev[v], lev[v + 1], b.jbits, b.jstart, b.jpar, b.joff, V, nb, la_x, ph_x);
            NQS_LAUNCHED();
        }
        return NQS_OK;
    }));
    // pass B: leaves with own rows grouped by parent (slots), in sub-passes of at most pass_rows
    // rows: slots [split[k], split[k+1])
    {
        ProfScope ps("ch_build", s);
        NQS_CK(cudaMemsetAsync(b.hist, 0, (size_t)(jobs + 1) * 8, s));
        ch_hist_kernel<<<grid_for(rows_max, 256), 256, 0, s>>>(b.lpar, b.lrows, rows_dev, rows_max, jobs, b.hist);
        NQS_LAUNCHED();
        NQS_TRY(launch_scan_i64(reinterpret_cast<const int64_t*>(b.hist), jobs + 1, nullptr, b.hoff, s));
        NQS_CK(cudaMemsetAsync(b.hist, 0, (size_t)(jobs + 1) * 8, s));
        ch_scatter_kernel<<<grid_for(rows_max, 256), 256, 0, s>>>(b.lpar, b.lrows, rows_dev, rows_max, jobs, b.hoff,
                                                                  b.hist, b.lorder, b.srows, b.sseg);
        NQS_LAUNCHED();
        NQS_TRY(launch_scan_i64(b.srows, rows_max, b.hoff + jobs + 1, b.soff, s));
    }
    int64_t nslots = 0, rows_b = 0;
    NQS_CK(cudaMemcpyAsync(&nslots, b.hoff + jobs + 1, 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    NQS_CK(cudaMemcpyAsync(&rows_b, b.soff + nslots, 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    const int64_t cap = b.pass_rows - n;
    const int nsplit = (int)std::max<int64_t>(1, (rows_b + cap - 1) / cap);
    if (nsplit > CHAIN_MAX_SPLIT) { set_error("prefix-sharing pass B needs too many sub-passes"); return NQS_ERR_CAPACITY; }
    ch_split_kernel<<<(nsplit + 1 + 127) / 128, 128, 0, s>>>(b.soff, b.hoff + jobs + 1, rows_max, cap, nsplit, b.split,
                                                             b.split_off);
    NQS_LAUNCHED();
    std::vector<int64_t> sp(nsplit + 1), so(nsplit + 1);
    NQS_CK(cudaMemcpyAsync(sp.data(), b.split, (nsplit + 1) * 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaMemcpyAsync(so.data(), b.split_off, (nsplit + 1) * 8, cudaMemcpyDeviceToHost, s));
    NQS_CK(cudaStreamSynchronize(s));
    for (int k = 0; k < nsplit; ++k) {
        const int64_t i0 = sp[k], i1 = sp[k + 1];
        if (i1 <= i0) continue;
        const int64_t M = so[k + 1] - so[k];
        if (M > b.pass_rows) { set_error("prefix-sharing sub-pass exceeds the workspace"); return NQS_ERR_CAPACITY; }
        ch_rows_kernel<<<grid_for(i1 - i0, 256), 256, 0, s>>>(b.soff, b.lorder, b.lstart, i0, i1, so[k], n, b.rjob,
                                                             b.rpos, b.rstart);
        NQS_LAUNCHED();
        NQS_TRY(ch_forward<MODE>(mc, P, w, b, xprime, M, false, lev, i0, i1, b.lorder, b.lstart, b.lpar, b.soff,
                                 b.sseg, so[k], s));
        NQS_TRY(with_dpl_c(d, [&](auto dpl) -> int {
            constexpr int DPL = decltype(dpl)::value;
            ProfScope ps("ch_heads", s);
            ch_leaf_heads_kernel<DPL><<<(unsigned)((i1 - i0 + 7) / 8), 256, 0, s>>>(
                mc, P, b.tf.h, i0, i1, b.lorder, b.soff, so[k], xprime, b.lstart, b.lpar, b.lrows, V, xs, nb, seg,
                seg_stride, la_x, ph_x, S, contrib, rows_dev);
            NQS_LAUNCHED();
            return NQS_OK;
        }));
    }
    // leaves without own rows: the diagonal rows and branches at the last position
    if (rows > 0) {
        NQS_TRY(with_dpl_c(d, [&](auto dpl) -> int {
            constexpr int DPL = decltype(dpl)::value;
            ProfScope ps("ch_heads", s);
            ch_leaf_heads_kernel<DPL><<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(
                mc, P, b.tf.h, 0, rows, nullptr, nullptr, 0, xprime, b.lstart, b.lpar, b.lrows, V, xs, nb, seg,
                seg_stride, la_x, ph_x, S, contrib, rows_dev);
            NQS_LAUNCHED();
            return NQS_OK;
        }));
    }
    return NQS_OK;
}

int chain_local_energy(const ModelConst& mc, const float* P, const TfWeights& w, ChainBufs& b, int depth,
                       const uint64_t* xs, int64_t nb, const int64_t* seg, int64_t seg_stride, const uint64_t* xprime,
                       const float4* S, const int64_t* rows_dev, int64_t rows_max, float* la_x, float* ph_x,
                       float2* contrib, cudaStream_t s) {
    if (nb <= 0) return NQS_OK;
    if (mc.precision != NQS_PREC_BF16)
        return ch_local_energy_mode<ACT_F32>(mc, P, w, b, depth, xs, nb, seg, seg_stride, xprime, S, rows_dev, rows_max,
                                             la_x, ph_x, contrib, s);
    if (mc.compensated)
        return ch_local_energy_mode<ACT_BF16X2>(mc, P, w, b, depth, xs, nb, seg, seg_stride, xprime, S, rows_dev,
                                                rows_max, la_x, ph_x, contrib, s);
    return ch_local_energy_mode<ACT_BF16>(mc, P, w, b, depth, xs, nb, seg, seg_stride, xprime, S, rows_dev, rows_max,
                                          la_x, ph_x, contrib, s);
}

}  // namespace nqs
