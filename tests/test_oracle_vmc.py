"""Pins for the energy statistics, the log psi gradient, the VMC gradient and Adam."""
import numpy as np
import pytest
import torch

import synth
from oracle.eloc import local_energy
from oracle.lanczos import sector_states, sector_hamiltonian
from oracle.vmc import energy_stats, logpsi_vjp, vmc_gradient, adam_step
from tests.common import oracle_model

SMALL_TF = dict(arch="transformer", n=8, n_up=2, n_dn=1, hidden=16, layers=2, heads=2, seed=5)


def test_energy_stats_reduce_to_numpy_on_replicated_samples():
    rng = np.random.default_rng(0)
    e = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    counts = rng.integers(1, 6, 50)
    mean, var = energy_stats(e, counts)
    rep = np.repeat(e, counts)
    assert abs(mean - rep.mean()) < 1e-13
    assert abs(var - np.var(rep)) < 1e-12


@pytest.mark.parametrize("dims", [1, 2, SMALL_TF,
                                  dict(arch="product", n=8, n_up=2, n_dn=1, hidden=0, layers=0, seed=3)])
def test_logpsi_vjp_matches_central_differences(dims):
    cfg = synth.get_config(dims) if isinstance(dims, int) else dims
    model, params = oracle_model(cfg, beta=1.0, requires_grad=True)
    n = model.n
    st = sector_states(n // 2, model.n_up, model.n_dn)[:64]
    rng = np.random.default_rng(1)
    ga, gp = rng.standard_normal(len(st)), rng.standard_normal(len(st))
    grads = vjp = logpsi_vjp(model, st, ga, gp)

    def f(p):
        m2, _ = oracle_model(cfg, beta=1.0)
        m2.p = {k: torch.tensor(v, dtype=torch.float64) for k, v in p.items()}
        la, ph = m2.log_psi(st)
        return np.sum(ga * la) + np.sum(gp * ph)

    base = {k: v.astype(np.float64) for k, v in params.items()}
    names = list(base)
    checked = 0
    for trial in range(40):
        k = names[rng.integers(len(names))]
        idx = tuple(rng.integers(s) for s in base[k].shape)
        hstep = 1e-6
        up = {a: b.copy() for a, b in base.items()}; up[k][idx] += hstep
        dn = {a: b.copy() for a, b in base.items()}; dn[k][idx] -= hstep
        fd = (f(up) - f(dn)) / (2 * hstep)
        assert abs(fd - grads[k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, grads[k][idx])
        checked += 1
    assert checked == 40


@pytest.mark.parametrize("dims", [1, 2, dict(arch="transformer", n=8, n_up=2, n_dn=2, hidden=16,
                                                 layers=1, heads=2, seed=8)])
def test_vmc_gradient_equals_derivative_of_exact_energy(dims):
    # Eq. grad with exact weights |f|^2 over the whole sector is the exact gradient of <H>.
    cfg = synth.get_config(dims) if isinstance(dims, int) else dims
    if isinstance(dims, int):
        xm, zm, c = synth.hamiltonian_for(cfg)
    else:
        h, eri, _ = synth.integrals(4, 0, True, 99)
        xm, zm, c = synth.jordan_wigner(h, eri)
    model, params = oracle_model(cfg, beta=0.7, requires_grad=True)
    n = model.n
    st = sector_states(n // 2, model.n_up, model.n_dn)
    Hs = sector_hamiltonian(xm, zm, c, n, st)

    def energy(p):
        m2, _ = oracle_model(cfg, beta=0.7)
        m2.p = {k: torch.tensor(v, dtype=torch.float64) for k, v in p.items()}
        la, ph = m2.log_psi(st)
        psi = np.exp(la + 1j * ph)
        return np.vdot(psi, Hs @ psi).real

    la, _ = model.log_psi(st)
    w = np.exp(2 * la)
    el = local_energy(model, xm, zm, c, st)
    g = vmc_gradient(model, st, w, el)
    base = {k: v.astype(np.float64) for k, v in params.items()}
    rng = np.random.default_rng(2)
    names = list(base)
    for trial in range(25):
        k = names[rng.integers(len(names))]
        idx = tuple(rng.integers(s) for s in base[k].shape)
        hstep = 1e-6
        up = {a: b.copy() for a, b in base.items()}; up[k][idx] += hstep
        dn = {a: b.copy() for a, b in base.items()}; dn[k][idx] -= hstep
        fd = (energy(up) - energy(dn)) / (2 * hstep)
        assert abs(fd - g[k][idx]) <= 2e-6 * max(1.0, abs(fd)), (k, idx, fd, g[k][idx])


def test_adam_matches_torch_optimizer():
    rng = np.random.default_rng(3)
    p0 = {"a": rng.standard_normal((4, 5)), "b": rng.standard_normal(7)}
    tp = [torch.tensor(v.copy(), requires_grad=True) for v in p0.values()]
    opt = torch.optim.Adam(tp, lr=1e-3, betas=(0.9, 0.99), eps=1e-8)
    p = dict(p0)
    m = {k: np.zeros_like(v) for k, v in p0.items()}
    v = {k: np.zeros_like(v) for k, v in p0.items()}
    for t in range(1, 6):
        g = {k: rng.standard_normal(val.shape) for k, val in p0.items()}
        for tens, k in zip(tp, p0):
            tens.grad = torch.tensor(g[k])
        opt.step()
        p, m, v = adam_step(p, g, m, v, t)
    for tens, k in zip(tp, p0):
        np.testing.assert_allclose(p[k], tens.detach().numpy(), rtol=1e-12, atol=1e-14)
