"""Grouping of Pauli strings by their X flip mask (paper Section 5.1: "a buffer of unique
flippings"; Eq. mtx_element for the phase).

Steps, in order:
  1. merge strings with equal (x_mask, z_mask) by FP64 summation in input order;
  2. drop merged coefficients that are exactly 0.0;
  3. order by (x_mask, z_mask) and group equal x_mask (the flip pattern m);
  4. fold the constant phase of Eq. mtx_element into each coefficient:
       c'_k = c_k * (-i)^{r_k},  r_k = number of sigma_2 factors = popcount(x_mask & z_mask),
     so that <x|P_k|x^m> = c'_k/c_k * (-1)^{popcount(x & z_k)}.
  5. per group record n_alpha = popcount(m & 0x55..) and n_beta = popcount(m & 0xAA..).
"""
import numpy as np

_MINUS_I_POW = np.array([1.0, -1.0j, -1.0, 1.0j])


def group_terms(xm, zm, c, n: int) -> dict:
    acc = {}
    for a, b, v in zip(np.asarray(xm, np.uint64).tolist(), np.asarray(zm, np.uint64).tolist(),
                       np.asarray(c, np.float64).tolist()):
        acc[(a, b)] = acc.get((a, b), 0.0) + v
    keys = sorted(k for k, v in acc.items() if v != 0.0)
    alpha = sum(1 << j for j in range(0, n, 2))
    beta = sum(1 << j for j in range(1, n, 2))

    g_m, g_off, g_na, g_nb = [], [], [], []
    t_z, t_c = [], []
    for a, b in keys:
        if not g_m or g_m[-1] != a:
            g_m.append(a)
            g_off.append(len(t_z))
            g_na.append(bin(a & alpha).count("1"))
            g_nb.append(bin(a & beta).count("1"))
        r = bin(a & b).count("1")
        t_z.append(b)
        t_c.append(acc[(a, b)] * _MINUS_I_POW[r % 4])
    g_off.append(len(t_z))
    tc = np.array(t_c, dtype=np.complex128)
    return dict(
        group_mask=np.array(g_m, dtype=np.uint64),
        group_offset=np.array(g_off, dtype=np.int64),
        group_n_alpha=np.array(g_na, dtype=np.int64),
        group_n_beta=np.array(g_nb, dtype=np.int64),
        term_z=np.array(t_z, dtype=np.uint64),
        term_c_re=tc.real.copy(),
        term_c_im=tc.imag.copy(),
    )
