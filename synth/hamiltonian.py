"""Seeded molecular-like integrals and their Jordan-Wigner qubit Hamiltonian as Pauli strings.

Stand-in for the paper's chemistry front end (Section 5.1: PubChem geometry, Psi4 integrals,
OpenFermion Jordan-Wigner), whose data is not available here.

Integrals (real orbitals, chemists' notation):
  h_pq        upper triangle ~ N(0, 1), mirrored;
  (pq|rs)     = sum_l L^l_pq L^l_rs over four symmetric Cholesky vectors with upper entries
                ~ N(0, 1/4), which gives the 8-fold symmetry and a positive semidefinite ERI.
Optional symmetry: every spatial orbital carries a label in Z2 (irreps=2) or Z2 x Z2 (irreps=4);
h_pq is zero unless the labels agree and L^l_pq is zero unless label_p ^ label_q equals the
vector's own label (l mod irreps), so (pq|rs) vanishes unless the XOR of all four labels is 0.
Optional decay: h_pq and L^l_pq are multiplied by exp(-|p-q|/3).

Hamiltonian (spin orbital j = 2p + s, s = 0 for spin up, 1 for spin down):
  H = sum_{pq,s} h_pq a+_{ps} a_{qs} + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
Jordan-Wigner: a+_j = Z_0..Z_{j-1} (X_j - i Y_j)/2 with |1> the occupied state.

Pauli strings use the symplectic form: qubit j of (x, z) is I for (0,0), X for (1,0),
Z for (0,1) and Y for (1,1); the string is the tensor product of those Hermitian matrices.
"""
import numpy as np

from .rng import SplitMix64

_PHASE = np.array([1.0, 1.0j, -1.0, -1.0j])


def _labels(n_orb: int, irreps: int, rng: SplitMix64) -> np.ndarray:
    if irreps == 0:
        return np.zeros(n_orb, dtype=np.int64)
    if irreps == 2 and n_orb == 2:
        return np.array([0, 1], dtype=np.int64)          # bonding / antibonding pair
    return rng.integers(n_orb, irreps)


def integrals(n_orb: int, irreps: int, decay: bool, seed: int, n_chol: int = 4):
    """Return (h [N,N], eri [N,N,N,N], labels [N]) as float64 / int64 arrays."""
    rng = SplitMix64(seed)
    lab = _labels(n_orb, irreps, rng)
    p, q = np.triu_indices(n_orb)
    dist = np.abs(np.subtract.outer(np.arange(n_orb), np.arange(n_orb)))
    damp = np.exp(-dist / 3.0) if decay else np.ones((n_orb, n_orb))

    h = np.zeros((n_orb, n_orb))
    h[p, q] = rng.normal(len(p))
    h = np.triu(h) + np.triu(h, 1).T
    if irreps:
        h = h * (lab[:, None] == lab[None, :])
    h = h * damp

    chol = np.zeros((n_chol, n_orb, n_orb))
    for l in range(n_chol):
        m = np.zeros((n_orb, n_orb))
        m[p, q] = 0.5 * rng.normal(len(p))
        m = np.triu(m) + np.triu(m, 1).T
        if irreps:
            m = m * ((lab[:, None] ^ lab[None, :]) == (l % irreps))
        chol[l] = m * damp
    eri = np.einsum("lpq,lrs->pqrs", chol, chol)
    return h, eri, lab


def _pauli_mul_phase(x1, z1, x2, z2):
    """Power of i in P(x1,z1) P(x2,z2) = i^g P(x1^x2, z1^z2), bitwise over all qubits (mod 4)."""
    y1 = x1 & z1
    xo = x1 & ~z1
    zo = ~x1 & z1
    bc = np.bitwise_count
    g = (bc(y1 & z2).astype(np.int64) - bc(y1 & x2)
         + bc(xo & z2 & x2) - bc(xo & z2 & ~x2)
         + bc(zo & x2 & ~z2) - bc(zo & x2 & z2))
    return g & 3


def _ladder(j: np.ndarray, dagger: bool):
    """JW images of a+_j (dagger) or a_j for an index array j: arrays of shape [T, 2]."""
    j = j.astype(np.uint64)
    e = np.uint64(1) << j
    low = e - np.uint64(1)
    x = np.stack([e, e], axis=1)
    z = np.stack([low, low | e], axis=1)
    c = np.empty((len(j), 2), dtype=np.complex128)
    c[:, 0] = 0.5
    c[:, 1] = -0.5j if dagger else 0.5j
    return x, z, c


def _product(a, b):
    xa, za, ca = a
    xb, zb, cb = b
    x1, x2 = xa[:, :, None], xb[:, None, :]
    z1, z2 = za[:, :, None], zb[:, None, :]
    g = _pauli_mul_phase(x1, z1, x2, z2)
    c = ca[:, :, None] * cb[:, None, :] * _PHASE[g]
    t = xa.shape[0]
    return (x1 ^ x2).reshape(t, -1), (z1 ^ z2).reshape(t, -1), c.reshape(t, -1)


def _accumulate(xs, zs, cs):
    """Sum coefficients of equal (x, z) keys; returns keys sorted by (x, z)."""
    x = np.concatenate([a.ravel() for a in xs])
    z = np.concatenate([a.ravel() for a in zs])
    c = np.concatenate([a.ravel() for a in cs])
    if len(x) == 0:
        return x, z, c
    order = np.lexsort((z, x))
    x, z, c = x[order], z[order], c[order]
    new = np.ones(len(x), dtype=bool)
    new[1:] = (x[1:] != x[:-1]) | (z[1:] != z[:-1])
    starts = np.flatnonzero(new)
    return x[starts], z[starts], np.add.reduceat(c, starts)


def jordan_wigner(h: np.ndarray, eri: np.ndarray, rel_cutoff: float = 1e-14, chunk: int = 1 << 16):
    """Pauli strings (x_mask, z_mask, coeff) of the JW image of (h, eri), merged and sorted.

    Coefficients whose magnitude is below rel_cutoff * max|c| are dropped (rounding residue of
    terms that cancel exactly); the imaginary parts must vanish to 1e-12 * max|c|.
    """
    n_orb = h.shape[0]
    parts_x, parts_z, parts_c = [], [], []

    # one-body
    p, q = np.nonzero(h)
    for s in (0, 1):
        P, Q = 2 * p + s, 2 * q + s
        x, z, c = _product(_ladder(P, True), _ladder(Q, False))
        c = c * h[p, q][:, None]
        xx, zz, cc = _accumulate([x], [z], [c])
        parts_x.append(xx); parts_z.append(zz); parts_c.append(cc)

    # two-body
    p, q, r, s_ = np.nonzero(eri)
    val = eri[p, q, r, s_]
    for sa in (0, 1):
        for sb in (0, 1):
            P, Q, R, S = 2 * p + sa, 2 * q + sa, 2 * r + sb, 2 * s_ + sb
            keep = (P != R) & (Q != S)
            P, Q, R, S, v = P[keep], Q[keep], R[keep], S[keep], val[keep]
            for lo in range(0, len(P), chunk):
                sl = slice(lo, lo + chunk)
                op = _product(_ladder(P[sl], True), _ladder(R[sl], True))
                op = _product(op, _ladder(S[sl], False))
                x, z, c = _product(op, _ladder(Q[sl], False))
                c = c * (0.5 * v[sl])[:, None]
                xx, zz, cc = _accumulate([x], [z], [c])
                parts_x.append(xx); parts_z.append(zz); parts_c.append(cc)

    x, z, c = _accumulate(parts_x, parts_z, parts_c)
    cmax = np.max(np.abs(c))
    assert np.max(np.abs(c.imag)) <= 1e-12 * cmax, "JW image of a real Hamiltonian must be real"
    keep = np.abs(c.real) >= rel_cutoff * cmax
    return x[keep].astype(np.uint64), z[keep].astype(np.uint64), c.real[keep].astype(np.float64)


_CACHE = {}


def hamiltonian_for(cfg):
    """(x_mask, z_mask, coeff) for a WorkloadConfig, memoised per process."""
    key = (cfg.n_orb, cfg.irreps, cfg.decay, cfg.seed_integrals)
    if key not in _CACHE:
        h, eri, _ = integrals(cfg.n_orb, cfg.irreps, cfg.decay, cfg.seed_integrals)
        _CACHE[key] = jordan_wigner(h, eri)
    return _CACHE[key]


# ----------------------------------------------------------------------------- two-word masks
# The same Jordan-Wigner construction for registers of up to 128 qubits: a mask is W uint64
# words (qubit j in bit j % 64 of word j // 64), stored along a trailing axis of length W.

def _pauli_mul_phase_w(x1, z1, x2, z2):
    """Power of i in P(x1,z1) P(x2,z2), the popcounts summed over the trailing word axis."""
    y1 = x1 & z1
    xo = x1 & ~z1
    zo = ~x1 & z1

    def bc(v):
        return np.bitwise_count(v).astype(np.int64).sum(axis=-1)
    g = (bc(y1 & z2) - bc(y1 & x2)
         + bc(xo & z2 & x2) - bc(xo & z2 & ~x2)
         + bc(zo & x2 & ~z2) - bc(zo & x2 & z2))
    return g & 3


def _ladder_w(j: np.ndarray, dagger: bool, words: int):
    """JW images of a+_j or a_j: masks of shape [T, 2, W]."""
    j = j.astype(np.int64)
    T = len(j)
    e = np.zeros((T, words), dtype=np.uint64)
    low = np.zeros((T, words), dtype=np.uint64)
    w_of, b_of = j // 64, (j % 64).astype(np.uint64)
    rows = np.arange(T)
    e[rows, w_of] = np.uint64(1) << b_of
    for w in range(words):
        low[:, w] = np.where(w < w_of, ~np.uint64(0), np.uint64(0))
    low[rows, w_of] = e[rows, w_of] - np.uint64(1)
    x = np.stack([e, e], axis=1)
    z = np.stack([low, low | e], axis=1)
    c = np.empty((T, 2), dtype=np.complex128)
    c[:, 0] = 0.5
    c[:, 1] = -0.5j if dagger else 0.5j
    return x, z, c


def _product_w(a, b):
    xa, za, ca = a
    xb, zb, cb = b
    x1, x2 = xa[:, :, None, :], xb[:, None, :, :]
    z1, z2 = za[:, :, None, :], zb[:, None, :, :]
    g = _pauli_mul_phase_w(x1, z1, x2, z2)
    c = ca[:, :, None] * cb[:, None, :] * _PHASE[g]
    t, W = xa.shape[0], xa.shape[-1]
    return (x1 ^ x2).reshape(t, -1, W), (z1 ^ z2).reshape(t, -1, W), c.reshape(t, -1)


def _accumulate_w(xs, zs, cs):
    """Sum coefficients of equal (x, z) keys; keys sorted by (x, z) as multi-word integers."""
    W = xs[0].shape[-1]
    x = np.concatenate([a.reshape(-1, W) for a in xs])
    z = np.concatenate([a.reshape(-1, W) for a in zs])
    c = np.concatenate([a.ravel() for a in cs])
    if len(x) == 0:
        return x, z, c
    keys = [z[:, w] for w in range(W)] + [x[:, w] for w in range(W)]   # last key is primary
    order = np.lexsort(keys)
    x, z, c = x[order], z[order], c[order]
    new = np.ones(len(x), dtype=bool)
    new[1:] = np.any(x[1:] != x[:-1], axis=1) | np.any(z[1:] != z[:-1], axis=1)
    starts = np.flatnonzero(new)
    return x[starts], z[starts], np.add.reduceat(c, starts)


def jordan_wigner_words(h: np.ndarray, eri: np.ndarray, words: int, rel_cutoff: float = 1e-14,
                        chunk: int = 1 << 15):
    """jordan_wigner with W-word masks: (x_mask [K, W], z_mask [K, W], coeff [K]), merged and
    sorted by (x, z) as multi-word integers; the same strings and coefficients as jordan_wigner
    where both apply (n <= 64)."""
    n_orb = h.shape[0]
    assert 2 * n_orb <= 64 * words
    parts_x, parts_z, parts_c = [], [], []
    p, q = np.nonzero(h)
    for s in (0, 1):
        P, Q = 2 * p + s, 2 * q + s
        x, z, c = _product_w(_ladder_w(P, True, words), _ladder_w(Q, False, words))
        c = c * h[p, q][:, None]
        xx, zz, cc = _accumulate_w([x], [z], [c])
        parts_x.append(xx); parts_z.append(zz); parts_c.append(cc)
    p, q, r, s_ = np.nonzero(eri)
    val = eri[p, q, r, s_]
    for sa in (0, 1):
        for sb in (0, 1):
            P, Q, R, S = 2 * p + sa, 2 * q + sa, 2 * r + sb, 2 * s_ + sb
            keep = (P != R) & (Q != S)
            P, Q, R, S, v = P[keep], Q[keep], R[keep], S[keep], val[keep]
            for lo in range(0, len(P), chunk):
                sl = slice(lo, lo + chunk)
                op = _product_w(_ladder_w(P[sl], True, words), _ladder_w(R[sl], True, words))
                op = _product_w(op, _ladder_w(S[sl], False, words))
                x, z, c = _product_w(op, _ladder_w(Q[sl], False, words))
                c = c * (0.5 * v[sl])[:, None]
                xx, zz, cc = _accumulate_w([x], [z], [c])
                parts_x.append(xx); parts_z.append(zz); parts_c.append(cc)
    x, z, c = _accumulate_w(parts_x, parts_z, parts_c)
    cmax = np.max(np.abs(c))
    assert np.max(np.abs(c.imag)) <= 1e-12 * cmax, "JW image of a real Hamiltonian must be real"
    keep = np.abs(c.real) >= rel_cutoff * cmax
    return x[keep].astype(np.uint64), z[keep].astype(np.uint64), c.real[keep].astype(np.float64)


def hamiltonian_words_for(cfg):
    """(x_mask [K, W], z_mask [K, W], coeff) of a workload whose register needs W = 2 words,
    memoised per process."""
    words = (cfg.n_qubits + 63) // 64
    key = ("w", words, cfg.n_orb, cfg.irreps, cfg.decay, cfg.seed_integrals)
    if key not in _CACHE:
        h, eri, _ = integrals(cfg.n_orb, cfg.irreps, cfg.decay, cfg.seed_integrals)
        _CACHE[key] = jordan_wigner_words(h, eri, words)
    return _CACHE[key]
