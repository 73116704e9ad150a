"""Sector-restricted Hamiltonian and a textbook Lanczos eigensolver (for the Rayleigh-Ritz bound
of paper Section 3: every variational energy upper-bounds lambda_min)."""
from itertools import combinations

import numpy as np
import scipy.sparse as sp

from .pauli import matrix_element


def sector_states(n_orb: int, n_up: int, n_dn: int) -> np.ndarray:
    ups = [sum(1 << (2 * p) for p in c) for c in combinations(range(n_orb), n_up)]
    dns = [sum(1 << (2 * p + 1) for p in c) for c in combinations(range(n_orb), n_dn)]
    return np.sort(np.array([u | d for u in ups for d in dns], dtype=np.uint64))


def sector_hamiltonian(xm, zm, c, n: int, states: np.ndarray) -> sp.csr_matrix:
    """H restricted to the given (sorted) basis states, built term by term."""
    dim = len(states)
    rows, cols, vals = [], [], []
    idx = np.arange(dim)
    for xk, zk, ck in zip(np.asarray(xm, np.uint64), np.asarray(zm, np.uint64), c):
        tgt = states ^ xk
        pos = np.searchsorted(states, tgt)
        pos_c = np.minimum(pos, dim - 1)
        ok = states[pos_c] == tgt
        rows.append(idx[ok]); cols.append(pos_c[ok])
        vals.append(ck * matrix_element(states[ok], xk, zk, n))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(dim, dim))


def lanczos_min(matvec, dim: int, iters: int = 200, seed: int = 0) -> float:
    """Smallest eigenvalue by Lanczos with full reorthogonalisation (Golub & Van Loan 10.1)."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(dim) + 0j
    q /= np.linalg.norm(q)
    Q = [q]
    alpha, beta = [], []
    b_prev = 0.0
    q_prev = np.zeros(dim, dtype=np.complex128)
    for _ in range(min(iters, dim)):
        w = matvec(Q[-1])
        a = np.vdot(Q[-1], w).real
        w = w - a * Q[-1] - b_prev * q_prev
        for v in Q:                       # full reorthogonalisation
            w = w - np.vdot(v, w) * v
        alpha.append(a)
        b = np.linalg.norm(w)
        if b < 1e-12:
            break
        beta.append(b)
        q_prev, b_prev = Q[-1], b
        Q.append(w / b)
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    return float(np.linalg.eigvalsh(T)[0])
