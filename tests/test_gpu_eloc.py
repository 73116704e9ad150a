"""GPU parity: log psi and the local energy (MADE, product) against the FP64 oracle.

Tolerance (fp32 path): rel_norm = sqrt(sum w|dE|^2) / sqrt(sum w|E|^2) <= 1e-5 with the sample
counts (here 1) as weights, and element by element max |dE_i| / (|E_i| + A_i 2^-24) <= 1e-4 (A_i:
sum of the magnitudes of sample i's terms); log|psi| to 2e-6 (1 + |log|psi||) and the phase to
2e-6 (1 + |phi|).
"""
import numpy as np
import pytest

import synth
from oracle.eloc import local_energy
from oracle.lanczos import sector_states
from tests.common import check_eloc, oracle_model, rel_norm
from tests.gpu_common import gpu_model, lib, to_dev_bits

pytestmark = pytest.mark.gpu

PROD = dict(arch="product", n=12, n_up=2, n_dn=3, hidden=0, layers=0, seed=31)
MADE_WIDE = dict(arch="made", n=16, n_up=3, n_dn=2, hidden=40, layers=3, seed=32)


def _cfg(c):
    return synth.get_config(c) if isinstance(c, int) else c


def _bits(cfg, B, seed):
    d = cfg if isinstance(cfg, dict) else dict(n=cfg.n_qubits, n_up=cfg.n_up, n_dn=cfg.n_dn)
    return synth.random_sector_bits(d["n"] // 2, d["n_up"], d["n_dn"], B, seed)


@pytest.mark.parametrize("c", [1, 2, PROD, MADE_WIDE])
@pytest.mark.parametrize("beta", [0.0, 2.0])
def test_logpsi_matches_oracle(c, beta):
    P = lib()
    cfg = _cfg(c)
    m, _ = gpu_model(cfg, beta=beta)
    om, _ = oracle_model(cfg, beta=beta)
    n = om.n
    bits = _bits(cfg, 300, 5)
    # add a few out-of-sector inputs
    bad = np.array([0, (1 << n) - 1], dtype=np.uint64)
    allb = np.concatenate([bits, bad])
    la, ph = P.nqs_logpsi(m, to_dev_bits(allb))
    la = la.cpu().numpy().astype(np.float64); ph = ph.cpu().numpy().astype(np.float64)
    wla, wph = om.log_psi(allb)
    ok = np.isfinite(wla)
    assert np.array_equal(np.isfinite(la), ok)
    assert np.all(np.abs(la[ok] - wla[ok]) <= 2e-6 * (1 + np.abs(wla[ok])))
    assert np.all(np.abs(ph - wph) <= 2e-6 * (1 + np.abs(wph)))


@pytest.mark.parametrize("c", [1, 2, PROD, MADE_WIDE])
@pytest.mark.parametrize("beta", [0.0, 2.0])
@pytest.mark.parametrize("compensated", [True, False])
def test_local_energy_matches_oracle(c, beta, compensated):
    P = lib()
    cfg = _cfg(c)
    if isinstance(c, int):
        xm, zm, coef = synth.hamiltonian_for(cfg)
        bits = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    else:
        h, eri, _ = synth.integrals(cfg["n"] // 2, 0, True, 77)
        xm, zm, coef = synth.jordan_wigner(h, eri)
        bits = _bits(cfg, 200, 9)
    n = cfg.n_qubits if not isinstance(cfg, dict) else cfg["n"]
    ham = P.Hamiltonian(n, xm, zm, coef)
    m, _ = gpu_model(cfg, beta=beta, compensated=compensated)
    om, _ = oracle_model(cfg, beta=beta)
    got = P.nqs_local_energy(ham, m, to_dev_bits(bits)).cpu().numpy().astype(np.float64)
    got = got[:, 0] + 1j * got[:, 1]
    want, absum = local_energy(om, xm, zm, coef, bits, return_abs=True)
    check_eloc(got, want, absum, "fp32", label=f"{c} beta={beta} comp={compensated}")


def test_local_energy_spans_chunks_with_repeats():
    # 2600 samples (3 internal chunks of 1024, ragged tail) drawn with repetition
    P = lib()
    cfg = synth.get_config(2)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    st = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    bits = st[np.random.default_rng(3).integers(0, len(st), 2600)]
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    m, _ = gpu_model(cfg, beta=1.0)
    om, _ = oracle_model(cfg, beta=1.0)
    got = P.nqs_local_energy(ham, m, to_dev_bits(bits)).cpu().numpy().astype(np.float64)
    got = got[:, 0] + 1j * got[:, 1]
    uniq, inv = np.unique(bits, return_inverse=True)
    want, absum = local_energy(om, xm, zm, coef, uniq, return_abs=True)
    check_eloc(got, want[inv], absum[inv], "fp32", label="chunks")
    # identical inputs give identical outputs (deterministic reduction)
    for u in range(len(uniq)):
        sel = got[inv == u]
        assert np.all(sel == sel[0])


def test_local_energy_enumeration_identity_on_gpu():
    # sum_x |psi|^2 E_loc(x) over the sector = <psi|H|psi> (exact for config 2)
    P = lib()
    cfg = synth.get_config(2)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    st = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    m, _ = gpu_model(cfg, beta=0.5)
    om, _ = oracle_model(cfg, beta=0.5)
    from oracle.lanczos import sector_hamiltonian
    Hs = sector_hamiltonian(xm, zm, coef, cfg.n_qubits, st)
    la, ph = om.log_psi(st)
    psi = np.exp(la + 1j * ph)
    quad = np.vdot(psi, Hs @ psi).real
    e = P.nqs_local_energy(ham, m, to_dev_bits(st)).cpu().numpy().astype(np.float64)
    ident = np.sum(np.abs(psi) ** 2 * e[:, 0])
    assert abs(ident - quad) <= 1e-5 * abs(quad)
