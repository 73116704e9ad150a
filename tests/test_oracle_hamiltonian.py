"""Pins for the Pauli algebra, the JW generator and the oracle's dense Hamiltonians (Section 3)."""
import os

import numpy as np
import pytest

import synth
from oracle import pauli, fermion
from oracle.grouping import group_terms

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_strings(n, k, seed):
    rng = np.random.default_rng(seed)
    xm = rng.integers(0, 1 << n, size=k, dtype=np.uint64)
    zm = rng.integers(0, 1 << n, size=k, dtype=np.uint64)
    c = rng.standard_normal(k)
    return xm, zm, c


def test_matrix_element_matches_paper_popcount_formula():
    # Eq. mtx_element: <x|P|x^p> = (-i)^r prod_{k: p_k in {2,3}} (-1)^{x_k}, r = #sigma_2.
    n = 10
    xm, zm, _ = _random_strings(n, 300, 1)
    rng = np.random.default_rng(2)
    xs = rng.integers(0, 1 << n, size=300, dtype=np.uint64)
    got = pauli.matrix_element(xs, xm, zm, n)
    r = np.bitwise_count(xm & zm).astype(np.int64)
    sign = 1 - 2 * (np.bitwise_count(xs & zm).astype(np.int64) & 1)
    want = ((-1j) ** r) * sign
    assert np.any(r % 2 == 1), "odd sigma_2 counts must be exercised"
    np.testing.assert_allclose(got, want, atol=0, rtol=0)


def test_pauli_matrix_one_nonzero_per_row_and_dense_sum():
    n = 4
    xm, zm, c = _random_strings(n, 12, 3)
    H = np.zeros((16, 16), dtype=complex)
    for a, b, v in zip(xm, zm, c):
        P = pauli.pauli_matrix(int(a), int(b), n)
        assert np.all(np.count_nonzero(P, axis=1) == 1)      # Section 3: one entry per row
        assert np.allclose(P @ P.conj().T, np.eye(16))
        H += v * P
    np.testing.assert_allclose(pauli.dense_hamiltonian(xm, zm, c, n), H, atol=1e-14)


def test_pauli_decomposition_round_trip_config1():
    # alpha_p = tr(H P_p) / 2^n recovers exactly the generator's coefficients (Section 3).
    cfg = synth.get_config(1)
    xm, zm, c = synth.hamiltonian_for(cfg)
    H = pauli.dense_hamiltonian(xm, zm, c, 4)
    ax, az, al = pauli.pauli_coefficients(H, 4)
    found = {(int(a), int(b)): v for a, b, v in zip(ax, az, al) if abs(v) > 1e-12}
    want = {(int(a), int(b)): v for a, b, v in zip(xm, zm, c)}
    assert set(found) == set(want)
    for key, v in want.items():
        assert abs(found[key] - v) < 1e-12


def test_config1_term_count_matches_table1():
    vals = {}
    for line in open(os.path.join(GOLDEN, "table1_h2_term_count.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    cfg = synth.get_config(1)
    assert (cfg.n_qubits, cfg.n_up, cfg.n_dn) == (vals["n_qubits"], vals["n_up"], vals["n_dn"])
    xm, zm, c = synth.hamiltonian_for(cfg)
    assert len(c) == vals["K"]


@pytest.mark.parametrize("n_orb,irreps,decay,seed", [(2, 2, False, 1001), (3, 0, True, 77),
                                                     (4, 4, True, 78), (6, 4, True, 1002)])
def test_jw_pauli_list_equals_fermionic_hamiltonian(n_orb, irreps, decay, seed):
    h, eri, _ = synth.integrals(n_orb, irreps, decay, seed)
    xm, zm, c = synth.jordan_wigner(h, eri)
    n = 2 * n_orb
    Hp = pauli.dense_hamiltonian(xm, zm, c, n)
    Hf = fermion.dense_from_integrals(h, eri)
    assert np.max(np.abs(Hp.imag)) < 1e-12
    np.testing.assert_allclose(Hp.real, Hf, atol=1e-11)


def test_dense_h_hermitian_and_particle_number_conserving():
    cfg = synth.get_config(2)
    xm, zm, c = synth.hamiltonian_for(cfg)
    n = cfg.n_qubits
    H = pauli.dense_hamiltonian(xm, zm, c, n)
    np.testing.assert_allclose(H, H.conj().T, atol=1e-12)
    idx = np.arange(1 << n, dtype=np.uint64)
    a = np.uint64(sum(1 << j for j in range(0, n, 2)))
    na = np.bitwise_count(idx & a).astype(float)
    nb = np.bitwise_count(idx & ~a & np.uint64((1 << n) - 1)).astype(float)
    for N in (na, nb):
        comm = H * N[None, :] - N[:, None] * H          # [H, N] for diagonal N
        assert np.max(np.abs(comm)) < 1e-12


@pytest.mark.parametrize("cid", [1, 2])
def test_hartree_fock_energy_closed_form(cid):
    cfg = synth.get_config(cid)
    h, eri, _ = synth.integrals(cfg.n_orb, cfg.irreps, cfg.decay, cfg.seed_integrals)
    xm, zm, c = synth.hamiltonian_for(cfg)
    hf = synth.hf_occupied(cfg.n_orb, cfg.n_up, cfg.n_dn)
    # <HF|H|HF> = sum over diagonal (xm = 0) strings of c_k <x|P_k|x>
    diag = xm == 0
    e = np.sum(c[diag] * pauli.matrix_element(np.uint64(hf), xm[diag], zm[diag], cfg.n_qubits))
    assert abs(e.imag) < 1e-14
    assert abs(e.real - fermion.hf_energy(h, eri, cfg.n_up, cfg.n_dn)) < 1e-11


def _grouped_dense(g, n):
    dim = 1 << n
    x = np.arange(dim, dtype=np.uint64)
    H = np.zeros((dim, dim), dtype=complex)
    for gi, m in enumerate(g["group_mask"]):
        lo, hi = g["group_offset"][gi], g["group_offset"][gi + 1]
        for k in range(lo, hi):
            cp = g["term_c_re"][k] + 1j * g["term_c_im"][k]
            sign = 1 - 2 * (np.bitwise_count(x & g["term_z"][k]).astype(np.int64) & 1)
            H[x.astype(np.int64), (x ^ m).astype(np.int64)] += cp * sign
    return H


def test_grouping_reconstructs_h_with_duplicates_and_odd_y():
    n = 6
    xm, zm, c = _random_strings(n, 60, 11)
    # duplicates that merge, and a pair that cancels exactly
    xm = np.concatenate([xm, xm[:10], [np.uint64(5), np.uint64(5)]])
    zm = np.concatenate([zm, zm[:10], [np.uint64(3), np.uint64(3)]])
    c = np.concatenate([c, 0.5 * c[:10], [0.25, -0.25]])
    perm = np.random.default_rng(12).permutation(len(c))
    xm, zm, c = xm[perm], zm[perm], c[perm]
    g = group_terms(xm, zm, c, n)
    np.testing.assert_allclose(_grouped_dense(g, n), pauli.dense_hamiltonian(xm, zm, c, n),
                               atol=1e-13)
    assert np.all(np.diff(g["group_mask"].astype(np.float64)) > 0)
    for gi in range(len(g["group_mask"])):
        z = g["term_z"][g["group_offset"][gi]: g["group_offset"][gi + 1]]
        assert np.all(np.diff(z.astype(np.float64)) > 0)
    assert len(g["term_z"]) == len({(int(a), int(b)) for a, b in zip(xm, zm)}) - 1
