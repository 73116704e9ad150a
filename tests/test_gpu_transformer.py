"""GPU parity for the transformer wavefunction (FP32 path): log psi, local energy and the
sampler, against the FP64 oracle.  Tolerances: log|psi| and phi to 1e-5 (1 + |value|); local
energy rel_norm <= 1e-5; sampler bit-exact under trace replay."""
import numpy as np
import pytest

import synth
from oracle.eloc import local_energy
from oracle.lanczos import sector_states
from oracle.models import in_sector
from oracle.sampler import sample
from tests.common import check_eloc, oracle_model, rel_norm
from tests.gpu_common import from_dev_bits, gpu_model, lib, to_dev_bits

pytestmark = pytest.mark.gpu

TF_SMALL = dict(arch="transformer", n=8, n_up=2, n_dn=1, hidden=32, layers=2, heads=2, seed=61)
TF_D64 = dict(arch="transformer", n=12, n_up=2, n_dn=3, hidden=64, layers=1, heads=4, seed=62)
TF_D128 = dict(arch="transformer", n=16, n_up=3, n_dn=3, hidden=128, layers=2, heads=8, seed=63)


def _cfg(c):
    return synth.get_config(c) if isinstance(c, int) else c


def _n(cfg):
    return cfg["n"] if isinstance(cfg, dict) else cfg.n_qubits


def _sector(cfg):
    return (cfg["n_up"], cfg["n_dn"]) if isinstance(cfg, dict) else (cfg.n_up, cfg.n_dn)


@pytest.mark.parametrize("c", [TF_SMALL, TF_D64, TF_D128, 3])
@pytest.mark.parametrize("beta", [0.0, 2.0])
def test_transformer_logpsi(c, beta):
    P = lib()
    cfg = _cfg(c)
    n = _n(cfg); nu, nd = _sector(cfg)
    m, _ = gpu_model(cfg, beta=beta)
    om, _ = oracle_model(cfg, beta=beta)
    bits = synth.random_sector_bits(n // 2, nu, nd, 257, seed=4)
    allb = np.concatenate([bits, np.array([0, (1 << n) - 1], dtype=np.uint64)])
    la, ph = P.nqs_logpsi(m, to_dev_bits(allb))
    la = la.cpu().numpy().astype(np.float64); ph = ph.cpu().numpy().astype(np.float64)
    wla, wph = om.log_psi(allb)
    ok = np.isfinite(wla)
    assert np.array_equal(np.isfinite(la), ok)
    assert np.max(np.abs(la[ok] - wla[ok]) / (1 + np.abs(wla[ok]))) <= 1e-5
    assert np.max(np.abs(ph - wph) / (1 + np.abs(wph))) <= 1e-5


@pytest.mark.parametrize("c,B", [(TF_SMALL, None), (TF_D64, 150), (TF_D128, 60), (3, 40)])
@pytest.mark.parametrize("beta", [0.0, 2.0])
def test_transformer_local_energy(c, B, beta):
    P = lib()
    cfg = _cfg(c)
    n = _n(cfg); nu, nd = _sector(cfg)
    if isinstance(c, int):
        xm, zm, coef = synth.hamiltonian_for(cfg)
    else:
        h, eri, _ = synth.integrals(n // 2, 0, True, 88)
        xm, zm, coef = synth.jordan_wigner(h, eri)
    bits = sector_states(n // 2, nu, nd) if B is None else synth.random_sector_bits(n // 2, nu, nd, B, seed=5)
    ham = P.Hamiltonian(n, xm, zm, coef)
    m, _ = gpu_model(cfg, beta=beta)
    om, _ = oracle_model(cfg, beta=beta)
    got = P.nqs_local_energy(ham, m, to_dev_bits(bits)).cpu().numpy().astype(np.float64)
    got = got[:, 0] + 1j * got[:, 1]
    want, absum = local_energy(om, xm, zm, coef, bits, return_abs=True)
    check_eloc(got, want, absum, "fp32", label=f"{c if isinstance(c, int) else n} beta={beta}")


@pytest.mark.parametrize("c,n_samples,max_unique", [(TF_SMALL, 5000, 10**6), (3, 100_000, 10**6),
                                                    (TF_D64, 20_000, 64)])
def test_transformer_sampler_trace_replay(c, n_samples, max_unique):
    P = lib()
    cfg = _cfg(c)
    m, _ = gpu_model(cfg, beta=1.0)
    om, _ = oracle_model(cfg, beta=1.0)
    seed = 77
    bits, counts, trace = P.nqs_sample(m, n_samples, max_unique, seed, trace=True)
    trace = trace.cpu().numpy()
    diffs = []

    def replay(parent_bits, k):
        p_gpu = trace[k, : len(parent_bits)]
        diffs.append(np.max(np.abs(p_gpu.astype(np.float64) - om.sampling_p(parent_bits, k))))
        return p_gpu

    wb, wc = sample(replay, om.n, om.order, n_samples, max_unique, seed)
    assert np.array_equal(from_dev_bits(bits), wb)
    assert np.array_equal(counts.cpu().numpy(), wc)
    assert max(diffs) <= 1e-5
    assert np.all(in_sector(wb, om.n, om.n_up, om.n_dn))


@pytest.mark.parametrize("c", [TF_SMALL, TF_D64, TF_D128, 3])
def test_transformer_backward_matches_oracle_vjp(c):
    import torch
    from oracle.vmc import logpsi_vjp
    P = lib()
    cfg = _cfg(c)
    n = _n(cfg); nu, nd = _sector(cfg)
    m, _ = gpu_model(cfg, beta=1.0)
    om, _ = oracle_model(cfg, beta=1.0, requires_grad=True)
    bits = synth.random_sector_bits(n // 2, nu, nd, 150, seed=8)
    rng = np.random.default_rng(9)
    ga = rng.standard_normal(len(bits)).astype(np.float32)
    gp = rng.standard_normal(len(bits)).astype(np.float32)
    grad = torch.zeros(m.param_count, dtype=torch.float32, device="cuda")
    P.nqs_logpsi_backward(m, to_dev_bits(bits), torch.tensor(ga, device="cuda"),
                          torch.tensor(gp, device="cuda"), grad)
    want = logpsi_vjp(om, bits, ga.astype(np.float64), gp.astype(np.float64))
    flat = np.concatenate([np.asarray(want[nm]).ravel() for nm, _, _ in m.param_layout()])
    got = grad.cpu().numpy().astype(np.float64)
    assert rel_norm(got, flat) <= 1e-4, rel_norm(got, flat)
    # every named tensor individually (catches a wrong layer or swapped gradient)
    for name, off, numel in m.param_layout():
        w = np.asarray(want[name]).ravel()
        if np.linalg.norm(w) > 1e-8:
            assert rel_norm(got[off: off + numel], w) <= 1e-3, name
