"""Local energy by its plain per-term definition (paper Eq. local_energy_auto, Algorithm 1).

    l(x) = sum_k c_k <x|P_k|x^k> f(x^k) / f(x),   x^k = x XOR xmask_k

No grouping: every Pauli string is visited, its matrix element is the product of per-qubit
sigma entries (oracle.pauli), and f(x^k) = 0 whenever x^k violates the Hamming-weight
constraint (the constrained model assigns it probability 0, Section 4 Constraints).
"""
import numpy as np

from .pauli import matrix_element
from .models import in_sector


def local_energy(model, xm, zm, c, bits, term_chunk: int = 1 << 16, return_abs: bool = False):
    """Complex E_loc for each sample in bits (uint64[B]) in FP64.

    With return_abs, also returns A[B] = sum_k |c_k <x|P_k|x^k> f(x^k)/f(x)|, the sum of the
    magnitudes of the terms (the conditioning of the sum: an FP32 evaluation of the same terms
    carries rounding errors of order A times the unit roundoff)."""
    xm = np.asarray(xm, dtype=np.uint64)
    zm = np.asarray(zm, dtype=np.uint64)
    c = np.asarray(c, dtype=np.float64)
    bits = np.asarray(bits, dtype=np.uint64)
    n = model.n
    la_x, ph_x = model.log_psi(bits)
    out = np.zeros(len(bits), dtype=np.complex128)
    mag = np.zeros(len(bits), dtype=np.float64)
    for i, x in enumerate(bits):
        xp = x ^ xm
        ok = in_sector(xp, n, model.n_up, model.n_dn)
        uniq, inv = np.unique(xp[ok], return_inverse=True)
        la, ph = model.log_psi(uniq)
        ratio = np.zeros(len(xm), dtype=np.complex128)
        ratio[ok] = np.exp((la[inv] - la_x[i]) + 1j * (ph[inv] - ph_x[i]))
        total = 0.0 + 0.0j
        absum = 0.0
        for lo in range(0, len(xm), term_chunk):
            sl = slice(lo, lo + term_chunk)
            elem = matrix_element(x, xm[sl], zm[sl], n)
            terms = c[sl] * elem * ratio[sl]
            total += np.sum(terms)
            absum += np.sum(np.abs(terms))
        out[i] = total
        mag[i] = absum
    return (out, mag) if return_abs else out


def connected_count(model, xm, bits) -> np.ndarray:
    """Number of distinct in-sector x^k per sample (the rows the network must evaluate)."""
    xm = np.asarray(xm, dtype=np.uint64)
    out = np.zeros(len(bits), dtype=np.int64)
    for i, x in enumerate(np.asarray(bits, dtype=np.uint64)):
        xp = np.unique(x ^ xm)
        out[i] = int(np.sum(in_sector(xp, model.n, model.n_up, model.n_dn)))
    return out
