"""The oracle's definitions for registers of more than 64 qubits (paper Table 1 reaches 76
qubits; Section 3 and Eq. hamiltonpauli put no bound on n).  Test infrastructure only: the
tests, the entry point's smoke check and the benchmark's CPU baseline use it; the library does
not.

A configuration or Pauli mask of n qubits is a row of W = ceil(n / 64) uint64 words, qubit j in
bit j % 64 of word j // 64.  Every function expands the words into per-qubit bits first and then
applies the same plain definitions as the one-word oracle:

  * <x|P|x ^ xm> is the product of the per-qubit sigma entries (Section 3; not the popcount
    formula of Eq. mtx_element, which the tests check against this);
  * the Hamming-weight constraint counts the spin-up (even) and spin-down (odd) qubits
    (Eq. hamming_weight_constraint);
  * the local energy is the per-term sum of Eq. local_energy_auto with f(x') = 0 outside the
    sector;
  * grouping follows the steps of oracle.grouping with multi-word keys.

The models of oracle.models are generic in n; only their input (the positions matrix) is built
here from the words.
"""
import numpy as np
import torch

from .pauli import SIGMA

_MINUS_I_POW = np.array([1.0, -1.0j, -1.0, 1.0j])


def words_of(n: int) -> int:
    return (n + 63) // 64


def bits_of_words(x, n: int) -> np.ndarray:
    """[..., W] uint64 words -> [..., n] int64 bits (bit j = qubit j)."""
    x = np.asarray(x, dtype=np.uint64)
    j = np.arange(n)
    w = j // 64
    b = (j % 64).astype(np.uint64)
    return ((x[..., w] >> b) & np.uint64(1)).astype(np.int64)


def words_of_bits(bits) -> np.ndarray:
    """[..., n] 0/1 -> [..., W] uint64 words."""
    bits = np.asarray(bits, dtype=np.uint64)
    n = bits.shape[-1]
    out = np.zeros(bits.shape[:-1] + (words_of(n),), dtype=np.uint64)
    for j in range(n):
        out[..., j // 64] |= bits[..., j] << np.uint64(j % 64)
    return out


def codes_words(xm, zm, n: int) -> np.ndarray:
    """Per-qubit sigma index in {0,1,2,3} of symplectic masks: (x,z) = (0,0)->0, (1,0)->1,
    (1,1)->2, (0,1)->3.  Shape [..., n]."""
    table = np.array([[0, 3], [1, 2]])
    return table[bits_of_words(xm, n), bits_of_words(zm, n)]


def matrix_element_words(x, xm, zm, n: int) -> np.ndarray:
    """<x| P |x ^ xm> = prod_j sigma_{p_j}[x_j, (x ^ xm)_j] for one configuration x [W] and
    masks xm, zm [K, W]."""
    x = np.asarray(x, dtype=np.uint64)
    xm = np.asarray(xm, dtype=np.uint64)
    p = codes_words(xm, zm, n)
    row = np.broadcast_to(bits_of_words(x, n), p.shape)
    col = bits_of_words(x[None, :] ^ xm, n)
    return np.prod(SIGMA[p, row, col], axis=-1)


def in_sector_words(bits, n: int, n_up: int, n_dn: int) -> np.ndarray:
    """Hamming-weight constraint of [..., W] configurations (up = even qubits, down = odd)."""
    X = bits_of_words(bits, n)
    return (X[..., 0::2].sum(axis=-1) == n_up) & (X[..., 1::2].sum(axis=-1) == n_dn)


def log_psi_words(model, bits, chunk: int = 4096):
    """(log|psi|, phi) in FP64 of the oracle model for [B, W] configurations."""
    bits = np.asarray(bits, dtype=np.uint64)
    la = np.empty(len(bits))
    ph = np.empty(len(bits))
    with torch.no_grad():
        for lo in range(0, len(bits), chunk):
            X = bits_of_words(bits[lo: lo + chunk], model.n)[:, model.order]
            a, p = model.log_psi_t(torch.tensor(X.astype(np.float64)))
            la[lo: lo + chunk] = a.numpy()
            ph[lo: lo + chunk] = p.numpy()
    return la, ph


def local_energy_words(model, xm, zm, c, bits, term_chunk: int = 1 << 15, return_abs: bool = False):
    """Complex E_loc (Eq. local_energy_auto, per term, no grouping) of [B, W] configurations;
    with return_abs also the sums of the magnitudes of each sample's terms."""
    xm = np.asarray(xm, dtype=np.uint64)
    zm = np.asarray(zm, dtype=np.uint64)
    c = np.asarray(c, dtype=np.float64)
    bits = np.asarray(bits, dtype=np.uint64)
    n = model.n
    la_x, ph_x = log_psi_words(model, bits)
    out = np.zeros(len(bits), dtype=np.complex128)
    mag = np.zeros(len(bits))
    for i, x in enumerate(bits):
        xp = x[None, :] ^ xm
        ok = in_sector_words(xp, n, model.n_up, model.n_dn)
        uniq, inv = np.unique(xp[ok], axis=0, return_inverse=True)
        la, ph = log_psi_words(model, uniq)
        ratio = np.zeros(len(xm), dtype=np.complex128)
        ratio[ok] = np.exp((la[inv.ravel()] - la_x[i]) + 1j * (ph[inv.ravel()] - ph_x[i]))
        total, absum = 0.0 + 0.0j, 0.0
        for lo in range(0, len(xm), term_chunk):
            sl = slice(lo, lo + term_chunk)
            terms = c[sl] * matrix_element_words(x, xm[sl], zm[sl], n) * ratio[sl]
            total += np.sum(terms)
            absum += np.sum(np.abs(terms))
        out[i] = total
        mag[i] = absum
    return (out, mag) if return_abs else out


def group_terms_words(xm, zm, c, n: int) -> dict:
    """oracle.grouping.group_terms for [K, W] masks: merge equal (x, z) by FP64 summation in
    input order, drop exact zeros, order by (x, z) as integers, group by x, fold (-i)^r with
    r = the number of sigma_2 factors.  Masks come back as [G, W] and [K', W] words (W from the
    input masks' shape)."""
    W = np.asarray(xm).shape[-1]
    acc = {}
    for a, b, v in zip(np.asarray(xm, np.uint64).tolist(), np.asarray(zm, np.uint64).tolist(),
                       np.asarray(c, np.float64).tolist()):
        ka = sum(int(w) << (64 * i) for i, w in enumerate(a))
        kb = sum(int(w) << (64 * i) for i, w in enumerate(b))
        acc[(ka, kb)] = acc.get((ka, kb), 0.0) + v
    keys = sorted(k for k, v in acc.items() if v != 0.0)
    alpha = sum(1 << j for j in range(0, n, 2))
    beta = sum(1 << j for j in range(1, n, 2))
    g_m, g_off, g_na, g_nb, t_z, t_c = [], [], [], [], [], []
    for a, b in keys:
        if not g_m or g_m[-1] != a:
            g_m.append(a)
            g_off.append(len(t_z))
            g_na.append(bin(a & alpha).count("1"))
            g_nb.append(bin(a & beta).count("1"))
        t_z.append(b)
        t_c.append(acc[(a, b)] * _MINUS_I_POW[bin(a & b).count("1") % 4])
    g_off.append(len(t_z))
    mask64 = (1 << 64) - 1

    def words(vals):
        return np.array([[(v >> (64 * i)) & mask64 for i in range(W)] for v in vals], dtype=np.uint64)
    tc = np.array(t_c, dtype=np.complex128)
    return dict(group_mask=words(g_m), group_offset=np.array(g_off, dtype=np.int64),
                group_n_alpha=np.array(g_na, dtype=np.int64), group_n_beta=np.array(g_nb, dtype=np.int64),
                term_z=words(t_z), term_c_re=tc.real.copy(), term_c_im=tc.imag.copy())


# ----------------------------------------------------------------------------- sampling
def _order_words(bits):
    """Indices that sort [U, W] configurations ascending as W-word integers (word W-1 most
    significant)."""
    bits = np.asarray(bits, dtype=np.uint64)
    return np.lexsort([bits[:, w] for w in range(bits.shape[1])])


def evict_words(bits, counts, max_unique: int):
    """oracle.sampler.evict for [U, W] configurations: keep the max_unique highest counts, ties
    broken by the configuration ascending; input and output in ascending order."""
    bits = np.asarray(bits, dtype=np.uint64)
    counts = np.asarray(counts, dtype=np.int64)
    if len(bits) <= max_unique:
        return bits, counts
    keys = [bits[:, w] for w in range(bits.shape[1])] + [-counts]   # last key is primary
    top = np.lexsort(keys)[:max_unique]
    top = top[_order_words(bits[top])]
    return bits[top], counts[top]


def sample_words(p_fn, n: int, order, n_samples: int, max_unique: int, seed: int, trace=None):
    """oracle.sampler.sample for registers of W = ceil(n / 64) words: the same buffer sampler
    (Section 4, Sampling) with the same Philox draws over the nominal indices in ascending
    configuration order; p_fn(parent_bits [U, W], k) -> fp32 probabilities.  Returns
    (bits uint64 [U, W], counts int64 [U]) ascending."""
    from .sampler import bernoulli_ones, threshold
    W = words_of(n)
    bits = np.zeros((1, W), dtype=np.uint64)
    counts = np.array([n_samples], dtype=np.int64)
    for k in range(n):
        q = int(order[k])
        p32 = np.asarray(p_fn(bits, k), dtype=np.float32)
        if trace is not None:
            trace.append((bits.copy(), counts.copy(), p32.copy()))
        n1 = bernoulli_ones(counts, threshold(p32), k, seed)
        ones = bits.copy()
        ones[:, q // 64] |= np.uint64(1) << np.uint64(q % 64)
        cb = np.concatenate([bits, ones])
        cc = np.concatenate([counts - n1, n1])
        keep = cc > 0
        cb, cc = cb[keep], cc[keep]
        idx = _order_words(cb)
        bits, counts = evict_words(cb[idx], cc[idx], max_unique)
    return bits, counts


def model_p_fn_words(model):
    """p_fn of sample_words backed by an oracle Model: FP64 conditional with the constraint,
    cast to fp32."""
    def fn(parent_bits, k):
        X = bits_of_words(parent_bits, model.n)[:, model.order]
        return model.sampling_p_positions(torch.tensor(X.astype(np.float64)), k).astype(np.float32)
    return fn
