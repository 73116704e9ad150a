"""Second-quantised Hamiltonian acting directly on occupation bitstrings (independent of Pauli
algebra).  Used to check that a Pauli list is the Jordan-Wigner image of given integrals
(paper Section 3: JW encoding; Section 5.1: molecular Hamiltonians).

Spin orbital j = 2p + s.  Ordering convention: a+_j |x> = (-1)^{#occupied orbitals below j}
|x + e_j> when orbital j is empty, which is what the JW string Z_0..Z_{j-1} produces.
"""
import numpy as np


def _apply(states, amp, j, create):
    occ = (states >> j) & 1
    ok = (occ == 0) if create else (occ == 1)
    below = states & ((1 << j) - 1)
    sign = 1 - 2 * (np.bitwise_count(below.astype(np.uint64)).astype(np.int64) & 1)
    new = states ^ (1 << j)
    return new, amp * sign * ok


def dense_from_integrals(h: np.ndarray, eri: np.ndarray) -> np.ndarray:
    """H = sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs on all 2^(2N) states."""
    n_orb = h.shape[0]
    n = 2 * n_orb
    dim = 1 << n
    H = np.zeros((dim, dim))
    cols = np.arange(dim, dtype=np.int64)

    def add(ops, coef):
        # ops applied right to left to every column state |x>
        st = cols.copy()
        amp = np.ones(dim, dtype=np.int64)
        for j, create in reversed(ops):
            st, amp = _apply(st, amp, j, create)
        nz = amp != 0
        np.add.at(H, (st[nz], cols[nz]), coef * amp[nz])

    for p in range(n_orb):
        for q in range(n_orb):
            if h[p, q] == 0.0:
                continue
            for s in (0, 1):
                add([(2 * p + s, True), (2 * q + s, False)], h[p, q])
    for p in range(n_orb):
        for q in range(n_orb):
            for r in range(n_orb):
                for s_ in range(n_orb):
                    v = eri[p, q, r, s_]
                    if v == 0.0:
                        continue
                    for sa in (0, 1):
                        for sb in (0, 1):
                            P, Q, R, S = 2 * p + sa, 2 * q + sa, 2 * r + sb, 2 * s_ + sb
                            add([(P, True), (R, True), (S, False), (Q, False)], 0.5 * v)
    return H


def hf_energy(h: np.ndarray, eri: np.ndarray, n_up: int, n_dn: int) -> float:
    """Slater-Condon closed form <HF|H|HF> = sum_i h_ii + 1/2 sum_ij [(ii|jj) - d_st (ij|ji)]
    over occupied spin orbitals i=(a,s), j=(b,t) (lowest n_up up, n_dn down spatial orbitals)."""
    occ = [(a, 0) for a in range(n_up)] + [(a, 1) for a in range(n_dn)]
    e = sum(h[a, a] for a, _ in occ)
    for a, s in occ:
        for b, t in occ:
            e += 0.5 * eri[a, a, b, b]
            if s == t:
                e -= 0.5 * eri[a, b, b, a]
    return float(e)
