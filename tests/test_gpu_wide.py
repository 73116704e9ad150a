"""GPU parity for registers of more than 64 qubits (two-word masks and configurations): the
76-qubit workload (38 orbitals, 8+8 electrons, 1,551,511 Pauli strings from the two-word
Jordan-Wigner generator; the paper's largest system in Table 1 has 76 qubits and ~1.6M strings)
and random two-word strings with odd sigma_2 counts.  Grouping bit-exact, term-sweep rows
bit-exact with S within fp32 tolerance, MADE / product log psi and local energies against the
oracle's two-word definitions (oracle/wide.py)."""
import numpy as np
import pytest

import synth
from oracle.models import Model
from oracle.wide import (group_terms_words, in_sector_words, local_energy_words, log_psi_words,
                         matrix_element_words, words_of_bits, bits_of_words)
from tests.common import check_eloc
from tests.gpu_common import lib

pytestmark = pytest.mark.gpu

WIDE = 6


def _dev(bits):
    import torch
    return torch.tensor(np.ascontiguousarray(bits, dtype=np.uint64).view(np.int64), device="cuda")


def _host(t):
    return t.cpu().numpy().view(np.uint64)


def _random_wide(n, K, seed, odd_y=True):
    """Random two-word strings whose flips are same-spin pairs (sector-preserving), with
    duplicates, an exact cancellation and (optionally) odd sigma_2 counts."""
    rng = np.random.default_rng(seed)
    X = np.zeros((K, n), dtype=np.int64)
    for k in range(K):
        for _ in range(k % 3):
            s = rng.integers(0, 2)
            a, b = rng.choice(np.arange(s, n, 2), 2, replace=False)
            X[k, a] ^= 1; X[k, b] ^= 1
    Z = rng.integers(0, 2, (K, n)) * (rng.random((K, n)) < 0.25)
    if not odd_y:
        # an even number of Y factors: clear Z on one flipped qubit where the count is odd
        for k in range(K):
            if (X[k] & Z[k]).sum() % 2:
                j = np.flatnonzero(X[k] & Z[k])[0]
                Z[k, j] = 0
    c = rng.standard_normal(K)
    xm, zm = words_of_bits(X), words_of_bits(Z)
    xm = np.concatenate([xm, xm[:20], xm[:1], xm[:1]])
    zm = np.concatenate([zm, zm[:20], zm[:1] ^ np.uint64(1), zm[:1] ^ np.uint64(1)])
    c = np.concatenate([c, -0.25 * c[:20], [0.75], [-0.75]])
    return xm, zm, c


def test_wide_grouping_bit_exact():
    P = lib()
    n = 76
    xm, zm, c = _random_wide(n, 400, 1)
    for xs, zs, cs in ((xm, zm, c), synth.hamiltonian_words_for(synth.get_config(WIDE))):
        if len(cs) > 10000:
            perm = np.random.default_rng(2).permutation(len(cs))[:200000]   # a large shuffled subset
            xs, zs, cs = xs[perm], zs[perm], cs[perm]
        h = P.Hamiltonian(n, xs, zs, cs)
        got = h.export()
        want = group_terms_words(xs, zs, cs, n)
        for k in ("group_mask", "group_offset", "term_z", "term_c_re", "term_c_im"):
            assert np.array_equal(got[k], want[k]), k


def _oracle_rows(x, xm, zm, c, n, n_up, n_dn):
    """{x' (as a tuple of words): (S, sum |c|)} of one sample: per-term matrix elements
    (products of sigma entries) summed over the strings of each flip mask, in-sector x' only."""
    order = np.lexsort([xm[:, w] for w in range(xm.shape[1])][::-1])
    xs, zs, cs = xm[order], zm[order], c[order]
    elem = np.concatenate([matrix_element_words(x, xs[lo: lo + (1 << 15)], zs[lo: lo + (1 << 15)], n)
                           for lo in range(0, len(cs), 1 << 15)])
    new = np.ones(len(cs), dtype=bool)
    new[1:] = np.any(xs[1:] != xs[:-1], axis=1)
    st = np.flatnonzero(new)
    S = np.add.reduceat(cs * elem, st)
    mass = np.add.reduceat(np.abs(cs), st)
    xp = x[None, :] ^ xs[st]
    ok = in_sector_words(xp, n, n_up, n_dn)
    return {tuple(int(w) for w in xp[i]): (S[i], mass[i]) for i in np.flatnonzero(ok)}


@pytest.mark.parametrize("which", ["random", "workload"])
@pytest.mark.parametrize("compensated", [True, False])
def test_wide_term_sweep_matches_definition(which, compensated):
    P = lib()
    n, n_up, n_dn = 76, 8, 8
    if which == "random":
        xm, zm, c = _random_wide(n, 600, 3)
        B = 37
    else:
        xm, zm, c = synth.hamiltonian_words_for(synth.get_config(WIDE))
        B = 3
    h = P.Hamiltonian(n, xm, zm, c)
    bits = synth.random_sector_bits_words(n // 2, n_up, n_dn, B, seed=13, words=2)
    ro, xp, sre, sim = P.nqs_term_sweep(h, n_up, n_dn, _dev(bits), compensated=compensated)
    ro = ro.cpu().numpy()
    xp = _host(xp).reshape(-1, 2)
    s = sre.cpu().numpy() + 1j * sim.cpu().numpy()
    rel = 3e-7 if compensated else 2e-5
    for i, x in enumerate(bits):
        want = _oracle_rows(x, xm, zm, c, n, n_up, n_dn)
        got = [tuple(int(w) for w in r) for r in xp[ro[i]: ro[i + 1]]]
        assert len(got) == len(set(got))
        assert sorted(got) == sorted(want), f"sample {i}: x' sets differ"
        for k, v in zip(got, s[ro[i]: ro[i + 1]]):
            S, mass = want[k]
            assert abs(v - S) <= rel * mass, (i, k, v, S)


def _models(arch):
    cfg = synth.get_config(WIDE)
    n = cfg.n_qubits
    order = synth.default_order(n)
    hidden, layers = (cfg.hidden, cfg.layers) if arch == "made" else (0, 0)
    named = synth.init_params(arch, n, cfg.n_up, cfg.n_dn, hidden, layers, 0, cfg.seed_params, beta=1.0,
                              order=order)
    P = lib()
    m = P.Model(arch, n, cfg.n_up, cfg.n_dn, hidden, layers, 0, order=order)
    m.bind(m.pack(named))
    om = Model(arch, named, n, cfg.n_up, cfg.n_dn, order, hidden, layers, 0)
    return cfg, m, om


@pytest.mark.parametrize("arch", ["made", "product"])
def test_wide_logpsi_matches_oracle(arch):
    P = lib()
    cfg, m, om = _models(arch)
    n = cfg.n_qubits
    bits = synth.random_sector_bits_words(cfg.n_orb, cfg.n_up, cfg.n_dn, 300, seed=21, words=2)
    bad = bits[:5].copy()
    bad[:, 1] ^= np.uint64(1) << np.uint64(70 - 64)           # one extra spin-up electron above bit 64
    allb = np.concatenate([bits, bad])
    la, ph = P.nqs_logpsi(m, _dev(allb))
    la = la.cpu().numpy().astype(np.float64); ph = ph.cpu().numpy().astype(np.float64)
    wl, wp = log_psi_words(om, allb)
    assert not np.any(in_sector_words(bad, n, cfg.n_up, cfg.n_dn))
    assert np.all(np.isneginf(la[-5:])) and np.all(np.isneginf(wl[-5:]))
    assert np.max(np.abs(la[:-5] - wl[:-5])) <= 2e-5 * max(1.0, np.max(np.abs(wl[:-5])))
    assert np.max(np.abs(ph[:-5] - wp[:-5])) <= 2e-5 * max(1.0, np.max(np.abs(wp[:-5])))


@pytest.mark.parametrize("arch,which", [("made", "workload"), ("product", "workload"), ("made", "random")])
def test_wide_local_energy_matches_oracle(arch, which):
    P = lib()
    cfg, m, om = _models(arch)
    n = cfg.n_qubits
    if which == "random":
        xm, zm, c = _random_wide(n, 800, 5)
        B = 24
    else:
        xm, zm, c = synth.hamiltonian_words_for(cfg)
        B = 3
    h = P.Hamiltonian(n, xm, zm, c)
    bits = synth.random_sector_bits_words(cfg.n_orb, cfg.n_up, cfg.n_dn, B, seed=31, words=2)
    e = P.nqs_local_energy(h, m, _dev(bits)).cpu().numpy().astype(np.float64)
    got = e[:, 0] + 1j * e[:, 1]
    want, absum = local_energy_words(om, xm, zm, c, bits, return_abs=True)
    check_eloc(got, want, absum, "fp32", label=f"76-qubit {arch} {which}")


@pytest.mark.parametrize("arch,n_samples,max_unique", [("made", 20000, 10 ** 6), ("made", 20000, 300),
                                                      ("product", 5000, 10 ** 6)])
def test_wide_sampler_trace_replay_bit_exact(arch, n_samples, max_unique):
    # the GPU's per-step probabilities replayed through the oracle's two-word buffer sampler give
    # the same samples and counts, bit for bit, with and without eviction
    from oracle.wide import model_p_fn_words, sample_words
    P = lib()
    cfg, m, om = _models(arch)
    seed = cfg.seed_sampler
    bits, counts, trace = P.nqs_sample(m, n_samples, max_unique, seed, trace=True)
    trace = trace.cpu().numpy()
    orc = model_p_fn_words(om)
    diffs = []

    def replay(parent_bits, k):
        p_gpu = trace[k, : len(parent_bits)]
        diffs.append(float(np.max(np.abs(p_gpu.astype(np.float64) - orc(parent_bits, k)))))
        return p_gpu

    wb, wc = sample_words(replay, cfg.n_qubits, om.order, n_samples, max_unique, seed)
    got = _host(bits).reshape(-1, 2)
    assert np.array_equal(got, wb)
    assert np.array_equal(counts.cpu().numpy(), wc)
    assert max(diffs) <= 2e-6
    assert np.all(in_sector_words(got, cfg.n_qubits, cfg.n_up, cfg.n_dn))
    assert got[:, 1].any()
    if max_unique >= n_samples:
        assert counts.sum().item() == n_samples


@pytest.mark.parametrize("arch", ["made", "product"])
def test_wide_backward_matches_oracle_vjp(arch):
    import torch
    from oracle.vmc import logpsi_vjp
    P = lib()
    cfg, m, _ = _models(arch)
    n = cfg.n_qubits
    hidden, layers = (cfg.hidden, cfg.layers) if arch == "made" else (0, 0)
    named = synth.init_params(arch, n, cfg.n_up, cfg.n_dn, hidden, layers, 0, cfg.seed_params, beta=1.0,
                              order=synth.default_order(n))
    om = Model(arch, named, n, cfg.n_up, cfg.n_dn, synth.default_order(n), hidden, layers, 0, requires_grad=True)
    bits = synth.random_sector_bits_words(cfg.n_orb, cfg.n_up, cfg.n_dn, 96, seed=41, words=2)
    rng = np.random.default_rng(41)
    ga = rng.standard_normal(96).astype(np.float32)
    gp = rng.standard_normal(96).astype(np.float32)
    grad = torch.zeros(m.param_count, dtype=torch.float32, device="cuda")
    P.nqs_logpsi_backward(m, _dev(bits).reshape(-1, 2), torch.tensor(ga, device="cuda"),
                          torch.tensor(gp, device="cuda"), grad)
    want = logpsi_vjp(om, bits, ga.astype(np.float64), gp.astype(np.float64))
    flat = np.concatenate([np.asarray(want[nm]).ravel() for nm, _, _ in m.param_layout()])
    from tests.common import rel_norm
    assert rel_norm(grad.cpu().numpy().astype(np.float64), flat) <= 1e-4


def test_wide_vmc_steps_on_the_76_qubit_workload():
    # full VMC steps (sample -> local energy over 1.55M strings -> FP64 statistics -> backward ->
    # Adam) on 76 qubits; the first step's gradient against the oracle's Eq. grad on its samples
    import torch
    from oracle.vmc import vmc_gradient
    from tests.common import rel_norm
    P = lib()
    cfg, m, _ = _models("made")
    n = cfg.n_qubits
    xm, zm, c = synth.hamiltonian_words_for(cfg)
    ham = P.Hamiltonian(n, xm, zm, c)
    named = synth.init_params("made", n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, 0, cfg.seed_params, beta=1.0,
                              order=synth.default_order(n))
    om = Model("made", named, n, cfg.n_up, cfg.n_dn, synth.default_order(n), cfg.hidden, cfg.layers, 0,
               requires_grad=True)
    vmc = P.VMC(ham, m, m.params.detach().clone(), cfg.n_samples, max_unique=6)
    bits, counts, _ = P.nqs_sample(m, cfg.n_samples, 6, cfg.seed_sampler)
    out = vmc.gradient(bits, counts)
    hb = _host(bits).reshape(-1, 2)
    hc = counts.cpu().numpy()
    e_or = local_energy_words(om, xm, zm, c, hb)
    want = vmc_gradient(om, hb, hc, e_or)
    flat = np.concatenate([np.asarray(want[nm]).ravel() for nm, _, _ in m.param_layout()])
    assert rel_norm(vmc.params.grad.cpu().numpy().astype(np.float64), flat) <= 1e-4
    e = [vmc.step(seed=cfg.seed_sampler + i)["stats"][0].item() for i in range(3)]
    assert np.all(np.isfinite(e))
    assert out["unique"] == len(hb) <= 6


def test_wide_registers_rejected_where_not_built():
    P = lib()
    cfg, m, _ = _models("made")
    bits = synth.random_sector_bits_words(cfg.n_orb, cfg.n_up, cfg.n_dn, 4, seed=1, words=2)
    with pytest.raises(P.NQSError) as e:
        P.Model("transformer", 76, 8, 8, 128, 4, 8)
    assert e.value.status == P.NQS_ERR_NQUBITS
    with pytest.raises(ValueError):
        P.Hamiltonian(76, np.zeros(3, np.uint64), np.zeros(3, np.uint64), np.ones(3))
    assert bits_of_words(bits, cfg.n_qubits).sum(axis=1).tolist() == [16] * 4
