"""Unique-sample autoregressive sampling with occurrence counts (paper Section 4, Sampling).

The paper keeps a buffer of distinct partial samples with counts: it starts from one entry,
doubles the buffer on one qubit per step, updates the counts by Bernoulli sampling with the
model's conditional, and evicts the entries with the lowest counts.  Readings used here (the
paper fixes no random number generator, no total count and no tie-break):
  * N_s nominal samples; the first buffer entry is the empty prefix with count N_s;
  * step k draws one Bernoulli per nominal sample: nominal index j runs over the exclusive
    prefix sum of the counts in canonical (bits ascending) buffer order, u = word 0 of
    Philox4x32-10(counter = (j, k, 0, 0), key = (seed lo 32 bits, seed hi 32 bits)), and the
    draw is 1 iff u < floor(p * 2^32) with p the fp32 probability (compared in 64 bits, so
    p = 1 always gives 1 and p = 0 always 0);
  * children with count 0 are dropped; if more than max_unique entries remain, the top
    max_unique by (count descending, bits ascending) are kept.

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11):
ten rounds of two 32x32->64 multiplies with a Weyl-sequence key schedule.
"""
import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; inputs are integer arrays holding 32-bit values."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def threshold(p32: np.ndarray) -> np.ndarray:
    """floor(p * 2^32) of fp32 probabilities, exactly (values 0 .. 2^32)."""
    p = np.asarray(p32, dtype=np.float32).astype(np.float64)
    return np.floor(p * 4294967296.0).astype(np.uint64)


def bernoulli_ones(counts, thr, k: int, seed: int) -> np.ndarray:
    """Number of ones among the draws of each parent's nominal samples at step k; parent s
    owns the nominal indices [sum_{s'<s} counts, sum_{s'<=s} counts)."""
    total = int(np.sum(counts))
    if total == 0:
        return np.zeros(len(counts), dtype=np.int64)
    parent = np.repeat(np.arange(len(counts)), counts)
    j = np.arange(total, dtype=np.uint64)
    u, _, _, _ = philox4x32_10(j, np.uint64(k), 0, 0, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    one = (u < thr[parent]).astype(np.int64)
    return np.bincount(parent, weights=one, minlength=len(counts)).astype(np.int64)


def sample(p_fn, n: int, order, n_samples: int, max_unique: int, seed: int, trace=None):
    """Run the buffer sampler.  p_fn(parent_bits, k) -> fp32 pihat(x_{order[k]}=1 | prefix) per
    parent, in the current canonical order.  If trace is a list, (bits, counts, p32) of every
    step's parents is appended to it.  Returns (bits uint64[U], counts int64[U]) bits-ascending."""
    bits = np.zeros(1, dtype=np.uint64)
    counts = np.array([n_samples], dtype=np.int64)
    for k in range(n):
        q = np.uint64(order[k])
        p32 = np.asarray(p_fn(bits, k), dtype=np.float32)
        if trace is not None:
            trace.append((bits.copy(), counts.copy(), p32.copy()))
        n1 = bernoulli_ones(counts, threshold(p32), k, seed)
        cb = np.concatenate([bits, bits | (np.uint64(1) << q)])
        cc = np.concatenate([counts - n1, n1])
        keep = cc > 0
        cb, cc = cb[keep], cc[keep]
        idx = np.argsort(cb, kind="stable")
        bits, counts = evict(cb[idx], cc[idx], max_unique)
    return bits, counts


def evict(bits, counts, max_unique: int):
    """Eviction of the buffer (Section 4, Sampling: the entries with the lowest numbers of
    occurrences are dropped): if more than max_unique entries remain, keep the max_unique with
    the highest counts, ties broken by bits ascending (a reading: the paper names no
    tie-break).  Input and output are in bits-ascending order."""
    bits = np.asarray(bits, dtype=np.uint64)
    counts = np.asarray(counts, dtype=np.int64)
    if len(bits) <= max_unique:
        return bits, counts
    top = np.lexsort((bits, -counts))[:max_unique]
    top = top[np.argsort(bits[top], kind="stable")]
    return bits[top], counts[top]


def model_p_fn(model):
    """p_fn backed by an oracle Model: FP64 conditional with the constraint, cast to fp32."""
    def fn(parent_bits, k):
        return model.sampling_p(parent_bits, k).astype(np.float32)
    return fn
