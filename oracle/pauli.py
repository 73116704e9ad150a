"""Pauli strings as tensor products of the 2x2 sigma matrices (paper Section 3, Eq. hamiltonpauli).

Matrix elements are products of per-qubit sigma entries -- deliberately NOT the popcount
formula of Eq. mtx_element, so that the tests can check that formula against this definition.
Dense index convention: basis state x has index sum_j x_j 2^j (qubit n-1 is the leftmost
Kronecker factor).
"""
import numpy as np

# sigma_0..sigma_3 exactly as printed in Section 3.
SIGMA = np.array([
    [[1, 0], [0, 1]],
    [[0, 1], [1, 0]],
    [[0, -1j], [1j, 0]],
    [[1, 0], [0, -1]],
], dtype=np.complex128)


def codes(xm, zm, n: int) -> np.ndarray:
    """Per-qubit sigma index p_j in {0,1,2,3} of symplectic masks: (x,z) = (0,0)->0, (1,0)->1
    (sigma_1), (1,1)->2 (sigma_2), (0,1)->3 (sigma_3).  Shape [..., n]."""
    xm = np.asarray(xm, dtype=np.uint64)[..., None]
    zm = np.asarray(zm, dtype=np.uint64)[..., None]
    j = np.arange(n, dtype=np.uint64)
    xb = ((xm >> j) & np.uint64(1)).astype(np.int64)
    zb = ((zm >> j) & np.uint64(1)).astype(np.int64)
    table = np.array([[0, 3], [1, 2]])
    return table[xb, zb]


def bits_of(x, n: int) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)[..., None]
    return ((x >> np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)


def matrix_element(x, xm, zm, n: int) -> np.ndarray:
    """<x| P |x ^ xm> = prod_j sigma_{p_j}[x_j, (x ^ xm)_j]  (broadcast over x and the masks)."""
    x = np.asarray(x, dtype=np.uint64)
    xm = np.asarray(xm, dtype=np.uint64)
    p = codes(xm, zm, n)
    row = bits_of(x, n)
    col = bits_of(x ^ xm, n)
    row, col, p = np.broadcast_arrays(row, col, p)
    return np.prod(SIGMA[p, row, col], axis=-1)


def pauli_matrix(xm: int, zm: int, n: int) -> np.ndarray:
    """Full 2^n x 2^n matrix of one Pauli string by Kronecker products (qubit n-1 leftmost)."""
    p = codes(np.uint64(xm), np.uint64(zm), n)
    out = np.array([[1.0 + 0j]])
    for j in range(n - 1, -1, -1):
        out = np.kron(out, SIGMA[p[j]])
    return out


def dense_hamiltonian(xm, zm, c, n: int) -> np.ndarray:
    """H = sum_k c_k P_k as a dense 2^n x 2^n complex matrix (each P_k has one entry per row)."""
    dim = 1 << n
    rows = np.arange(dim, dtype=np.uint64)
    H = np.zeros((dim, dim), dtype=np.complex128)
    for xk, zk, ck in zip(np.asarray(xm, np.uint64), np.asarray(zm, np.uint64), c):
        cols = rows ^ xk
        H[rows.astype(np.int64), cols.astype(np.int64)] += ck * matrix_element(rows, xk, zk, n)
    return H


def pauli_coefficients(H: np.ndarray, n: int):
    """alpha_p = tr(H P_p) / 2^n for all 4^n strings (Section 3); returns (xm, zm, alpha)."""
    out_x, out_z, out_a = [], [], []
    for xm in range(1 << n):
        for zm in range(1 << n):
            P = pauli_matrix(xm, zm, n)
            out_x.append(xm); out_z.append(zm)
            out_a.append(np.trace(H @ P) / (1 << n))
    return (np.array(out_x, dtype=np.uint64), np.array(out_z, dtype=np.uint64),
            np.array(out_a))
