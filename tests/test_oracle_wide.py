"""Pins of the oracle's two-word (64 < n <= 128 qubits) definitions (oracle/wide.py).

The word-generic code is checked (1) against the pinned one-word oracle where both apply,
(2) against Eq. mtx_element's popcount formula and the Slater-Condon closed form on qubits on
both sides of the word boundary, and (3) by the exact invariance of the local energy under a
relabelling of the qubits that moves them across the boundary (the Hamiltonian's strings, the
configuration and the sampling order permuted together)."""
import numpy as np
import pytest

import synth
from oracle import fermion, pauli
from oracle.eloc import local_energy
from oracle.grouping import group_terms
from oracle.models import Model
from oracle.wide import (bits_of_words, group_terms_words, in_sector_words, local_energy_words,
                         matrix_element_words, words_of_bits)
from tests.common import oracle_model


def _two_words(a):
    a = np.asarray(a, dtype=np.uint64)
    return np.stack([a, np.zeros_like(a)], axis=-1)


def test_matrix_element_words_matches_one_word_oracle():
    rng = np.random.default_rng(1)
    n = 20
    xm = rng.integers(0, 1 << n, 300, dtype=np.uint64)
    zm = rng.integers(0, 1 << n, 300, dtype=np.uint64)
    for x in rng.integers(0, 1 << n, 5, dtype=np.uint64):
        want = pauli.matrix_element(x, xm, zm, n)
        got = matrix_element_words(_two_words(x), _two_words(xm), _two_words(zm), n)
        assert np.array_equal(got, want)


def test_matrix_element_words_is_the_popcount_formula_across_the_boundary():
    # Eq. mtx_element: <x|P|x ^ xm> = (-i)^r (-1)^{popcount(x & z)}, r = popcount(xm & zm)
    rng = np.random.default_rng(2)
    n = 76
    X = rng.integers(0, 2, (200, n))
    Z = rng.integers(0, 2, (200, n))
    Xs = rng.integers(0, 2, (4, n))
    xm, zm = words_of_bits(X), words_of_bits(Z)
    for xb in Xs:
        x = words_of_bits(xb)
        got = matrix_element_words(x, xm, zm, n)
        r = (X & Z).sum(axis=1)
        par = (Z & xb[None, :]).sum(axis=1)
        want = (-1j) ** r * (-1.0) ** par
        assert np.allclose(got, want, atol=0, rtol=0)
    assert np.array_equal(bits_of_words(xm, n), X)


def test_in_sector_words_counts_both_words():
    n = 76
    b = np.zeros((3, n), dtype=np.int64)
    b[0, [0, 2, 64, 66, 1, 75]] = 1     # 4 up, 2 down
    b[1, [70, 72, 74, 68, 3, 65]] = 1   # 4 up, 2 down
    b[2, [0, 2, 4, 64, 1, 75]] = 1      # 4 up, 2 down
    b[2, 6] = 1                         # 5 up
    assert in_sector_words(words_of_bits(b), n, 4, 2).tolist() == [True, True, False]


def test_grouping_words_matches_one_word_grouping():
    cfg = synth.get_config(3)
    xm, zm, c = synth.hamiltonian_for(cfg)
    perm = np.random.default_rng(3).permutation(len(c))
    xm, zm, c = xm[perm], zm[perm], c[perm]
    want = group_terms(xm, zm, c, cfg.n_qubits)
    got = group_terms_words(_two_words(xm), _two_words(zm), c, cfg.n_qubits)
    for k in ("group_offset", "group_n_alpha", "group_n_beta", "term_c_re", "term_c_im"):
        assert np.array_equal(got[k], want[k]), k
    for k in ("group_mask", "term_z"):
        assert np.array_equal(got[k][:, 0], want[k]) and not got[k][:, 1].any(), k


def test_local_energy_words_matches_one_word_oracle():
    cfg = synth.get_config(2)
    xm, zm, c = synth.hamiltonian_for(cfg)
    om, _ = oracle_model(cfg)
    bits = synth.random_sector_bits(cfg.n_orb, cfg.n_up, cfg.n_dn, 6, seed=5)
    want, wa = local_energy(om, xm, zm, c, bits, return_abs=True)
    got, ga = local_energy_words(om, _two_words(xm), _two_words(zm), c, _two_words(bits), return_abs=True)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.max(np.abs(want)))
    assert np.allclose(ga, wa, rtol=1e-13)


def test_local_energy_invariant_under_relabelling_across_the_word_boundary():
    # a 76-qubit register: random Pauli strings (sector-preserving flips, odd sigma_2 counts
    # included) and a MADE model; relabel every qubit by a spin-parity-preserving permutation
    # that moves the low qubits above bit 64 and back, applied to the strings, the configuration
    # and the sampling order at once: the local energy is the same number
    n, n_up, n_dn = 76, 5, 4
    rng = np.random.default_rng(7)
    K = 160
    X = np.zeros((K, n), dtype=np.int64)
    for k in range(K):
        kind = k % 3
        if kind:                       # a same-spin pair flip (2 or 4 flipped qubits)
            for _ in range(kind):
                s = rng.integers(0, 2)
                a, b = rng.choice(np.arange(s, n, 2), 2, replace=False)
                X[k, a] ^= 1; X[k, b] ^= 1
    Z = rng.integers(0, 2, (K, n)) * (rng.random((K, n)) < 0.2)
    c = rng.standard_normal(K)
    order = np.arange(n - 1, -1, -1)
    params = synth.init_params("made", n, n_up, n_dn, 16, 2, 0, 11, beta=0.5, order=order)
    samples = synth.random_sector_bits_words(n // 2, n_up, n_dn, 3, seed=9, words=2)
    Xs = bits_of_words(samples, n)

    half = n // 2
    perm = np.empty(n, dtype=np.int64)              # qubit j -> perm[j]; keeps j's parity
    perm[0::2] = (np.arange(half) * 2 + 2 * 31) % n
    perm[1::2] = (np.arange(half) * 2 + 1 + 2 * 17) % n
    assert sorted(perm.tolist()) == list(range(n))
    assert np.all(perm % 2 == np.arange(n) % 2)

    def relabel(B):
        out = np.zeros_like(B)
        out[..., perm] = B
        return out

    m1 = Model("made", params, n, n_up, n_dn, order, 16, 2, 0)
    m2 = Model("made", params, n, n_up, n_dn, perm[order], 16, 2, 0)
    e1 = local_energy_words(m1, words_of_bits(X), words_of_bits(Z), c, samples)
    e2 = local_energy_words(m2, words_of_bits(relabel(X)), words_of_bits(relabel(Z)), c,
                            words_of_bits(relabel(Xs)))
    assert np.max(np.abs(e1.imag)) > 1e-3            # complex: odd sigma_2 counts contribute
    assert np.allclose(e1, e2, rtol=1e-12, atol=1e-12 * np.max(np.abs(e1)))


def test_words_jordan_wigner_matches_one_word_generator():
    for cid in (2, 3):
        cfg = synth.get_config(cid)
        h, eri, _ = synth.integrals(cfg.n_orb, cfg.irreps, cfg.decay, cfg.seed_integrals)
        x, z, c = synth.jordan_wigner(h, eri)
        xw, zw, cw = synth.jordan_wigner_words(h, eri, 2)
        assert np.array_equal(xw[:, 0], x) and np.array_equal(zw[:, 0], z) and np.array_equal(cw, c)
        assert not xw[:, 1].any() and not zw[:, 1].any()


def _determinant_energy(h, eri, occ):
    """Slater-Condon energy of the determinant with occupied spin orbitals occ = [(p, s)]."""
    e = sum(h[a, a] for a, _ in occ)
    for a, s in occ:
        for b, t in occ:
            e += 0.5 * eri[a, a, b, b]
            if s == t:
                e -= 0.5 * eri[a, b, b, a]
    return e


@pytest.mark.slow
def test_words_hamiltonian_diagonal_is_slater_condon_across_the_boundary():
    # 66 qubits: determinants with electrons on both sides of qubit 64
    n_orb = 33
    h, eri, _ = synth.integrals(n_orb, 4, True, 1234)
    xm, zm, c = synth.jordan_wigner_words(h, eri, 2)
    n = 2 * n_orb
    diag = ~xm.any(axis=1)
    rng = np.random.default_rng(4)
    for _ in range(3):
        # qubits 64 (orbital 32 up) and 63 (orbital 31 down) occupied, the rest random
        up = np.concatenate([[32], rng.choice(32, 3, replace=False)])
        dn = np.concatenate([[31], rng.choice(31, 2, replace=False)])
        occ = [(int(p), 0) for p in up] + [(int(p), 1) for p in dn]
        b = np.zeros(n, dtype=np.int64)
        for p, s in occ:
            b[2 * p + s] = 1
        e = np.sum(c[diag] * matrix_element_words(words_of_bits(b), xm[diag], zm[diag], n))
        assert abs(e.imag) < 1e-12
        assert abs(e.real - _determinant_energy(h, eri, occ)) < 1e-10 * max(1.0, abs(e.real))


def test_hf_energy_helper_agrees_with_determinant_energy():
    cfg = synth.get_config(2)
    h, eri, _ = synth.integrals(cfg.n_orb, cfg.irreps, cfg.decay, cfg.seed_integrals)
    occ = [(a, 0) for a in range(cfg.n_up)] + [(a, 1) for a in range(cfg.n_dn)]
    assert abs(_determinant_energy(h, eri, occ) - fermion.hf_energy(h, eri, cfg.n_up, cfg.n_dn)) < 1e-12


def test_words_sampler_matches_one_word_sampler():
    # the same draws and buffers: the two-word sampler on a 12-qubit register (high word zero)
    # gives the one-word sampler's samples and counts, with and without eviction
    from oracle.sampler import model_p_fn, sample
    from oracle.wide import model_p_fn_words, sample_words
    cfg = synth.get_config(2)
    om, _ = oracle_model(cfg, beta=1.0)
    for max_unique in (10 ** 6, 40):
        b1, c1 = sample(model_p_fn(om), om.n, om.order, 5000, max_unique, 77)
        b2, c2 = sample_words(model_p_fn_words(om), om.n, om.order, 5000, max_unique, 77)
        assert np.array_equal(b2[:, 0], b1) and np.array_equal(c2, c1)


def test_words_ordering_and_eviction_are_integer_order():
    # ascending order and the eviction tie-break follow the configurations as 128-bit integers
    from oracle.wide import evict_words
    rng = np.random.default_rng(8)
    b = rng.integers(0, 2 ** 63, (300, 2), dtype=np.uint64) >> rng.integers(0, 62, (300, 2)).astype(np.uint64)
    b[:50, 1] = 5                               # many equal high words: order decided by the low word
    ints = [int(x[0]) + (int(x[1]) << 64) for x in b]
    srt = np.argsort(np.array(ints, dtype=object), kind="stable")
    b = b[srt]
    counts = rng.integers(1, 4, 300)
    kb, kc = evict_words(b, counts, 100)
    ki = [int(x[0]) + (int(x[1]) << 64) for x in kb]
    assert ki == sorted(ki)
    # survivors by hand: every count above the cut, then the smallest integers at the cut
    pairs = sorted(zip((-counts).tolist(), [int(x[0]) + (int(x[1]) << 64) for x in b]))[:100]
    assert sorted(v for _, v in pairs) == ki


def test_words_sampler_on_76_qubits_stays_in_the_sector():
    from oracle.wide import model_p_fn_words, sample_words
    n, n_up, n_dn = 76, 8, 8
    order = synth.default_order(n)
    params = synth.init_params("made", n, n_up, n_dn, 16, 1, 0, 5, beta=1.0, order=order)
    om = Model("made", params, n, n_up, n_dn, order, 16, 1, 0)
    bits, counts = sample_words(model_p_fn_words(om), n, order, 400, 10 ** 6, 3)
    assert counts.sum() == 400 and np.all(counts > 0)
    assert np.all(in_sector_words(bits, n, n_up, n_dn))
    assert bits[:, 1].any()                   # electrons above qubit 64 are drawn


def test_model_positions_of_words_match_the_word_expansion():
    # oracle.models.Model accepts [B, W] configurations directly (log psi, VJP, gradient)
    from oracle.wide import log_psi_words
    n, n_up, n_dn = 76, 8, 8
    order = np.random.default_rng(3).permutation(n)
    params = synth.init_params("made", n, n_up, n_dn, 16, 2, 0, 5, beta=1.0, order=order)
    om = Model("made", params, n, n_up, n_dn, order, 16, 2, 0)
    bits = synth.random_sector_bits_words(n // 2, n_up, n_dn, 20, seed=2, words=2)
    la, ph = om.log_psi(bits)
    wl, wp = log_psi_words(om, bits)
    assert np.array_equal(la, wl) and np.array_equal(ph, wp)
    one = synth.random_sector_bits(10, 3, 3, 20, seed=2)
    m12 = Model("made", synth.init_params("made", 20, 3, 3, 16, 1, 0, 5, order=np.arange(20)), 20, 3, 3,
                np.arange(20), 16, 1, 0)
    assert np.array_equal(m12.positions(one).numpy(), m12.positions(_two_words(one)).numpy())
