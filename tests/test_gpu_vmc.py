"""GPU parity: log psi backward, energy statistics, Adam and the VMC step.

Gradient tolerance (fp32 path): rel_norm <= 1e-4 against the oracle's FP64 autograd."""
import numpy as np
import pytest
import torch

import synth
from oracle.eloc import local_energy
from oracle.lanczos import sector_states
from oracle.vmc import adam_step, energy_stats, logpsi_vjp, surrogate_weights, vmc_gradient
from tests.common import oracle_model, rel_norm
from tests.gpu_common import gpu_model, lib, to_dev_bits

pytestmark = pytest.mark.gpu

PROD = dict(arch="product", n=12, n_up=2, n_dn=3, hidden=0, layers=0, seed=51)
MADE_WIDE = dict(arch="made", n=16, n_up=3, n_dn=2, hidden=40, layers=3, seed=52)


def _flat(m, named):
    return np.concatenate([np.asarray(named[name]).ravel() for name, _, _ in m.param_layout()])


@pytest.mark.parametrize("c", [1, 2, PROD, MADE_WIDE])
def test_backward_matches_oracle_vjp(c):
    P = lib()
    cfg = synth.get_config(c) if isinstance(c, int) else c
    m, _ = gpu_model(cfg, beta=1.0)
    om, _ = oracle_model(cfg, beta=1.0, requires_grad=True)
    n = om.n
    bits = synth.random_sector_bits(n // 2, om.n_up, om.n_dn, 333, seed=3)
    rng = np.random.default_rng(4)
    ga = rng.standard_normal(len(bits)).astype(np.float32)
    gp = rng.standard_normal(len(bits)).astype(np.float32)
    grad = torch.zeros(m.param_count, dtype=torch.float32, device="cuda")
    P.nqs_logpsi_backward(m, to_dev_bits(bits), torch.tensor(ga, device="cuda"),
                          torch.tensor(gp, device="cuda"), grad)
    want = logpsi_vjp(om, bits, ga.astype(np.float64), gp.astype(np.float64))
    got = grad.cpu().numpy().astype(np.float64)
    assert rel_norm(got, _flat(m, want)) <= 1e-4
    # accumulation: a second call adds the same amount
    P.nqs_logpsi_backward(m, to_dev_bits(bits), torch.tensor(ga, device="cuda"),
                          torch.tensor(gp, device="cuda"), grad)
    assert rel_norm(grad.cpu().numpy().astype(np.float64), 2 * _flat(m, want)) <= 1e-4


def test_energy_stats_and_surrogate_weights():
    P = lib()
    rng = np.random.default_rng(6)
    e = (rng.standard_normal((1000, 2)) * [3.0, 0.1]).astype(np.float32)
    counts = rng.integers(1, 50, 1000)
    stats, ga, gp = P.nqs_energy_stats(torch.tensor(e, device="cuda"), torch.tensor(counts, device="cuda"))
    ec = e[:, 0].astype(np.float64) + 1j * e[:, 1]
    mean, var = energy_stats(ec, counts)
    s = stats.cpu().numpy()
    assert abs(s[0] - mean.real) <= 1e-12 * max(1, abs(mean)) and abs(s[1] - mean.imag) <= 1e-12
    assert abs(s[2] - var) <= 1e-11 * var and s[3] == counts.sum()
    wa, wp = surrogate_weights(ec, counts)
    assert np.allclose(ga.cpu().numpy(), wa, rtol=1e-6, atol=1e-9)
    assert np.allclose(gp.cpu().numpy(), wp, rtol=1e-6, atol=1e-9)


def test_adam_matches_oracle():
    P = lib()
    rng = np.random.default_rng(7)
    p0 = rng.standard_normal(5000).astype(np.float32)
    p = torch.tensor(p0, device="cuda")
    m = torch.zeros_like(p); v = torch.zeros_like(p)
    op, om_, ov = {"a": p0.astype(np.float64)}, {"a": np.zeros(5000)}, {"a": np.zeros(5000)}
    for t in range(1, 4):
        g = rng.standard_normal(5000).astype(np.float32)
        P.nqs_adam_step(p, torch.tensor(g, device="cuda"), m, v, t)
        op, om_, ov = adam_step(op, {"a": g.astype(np.float64)}, om_, ov, t)
    assert np.allclose(p.cpu().numpy(), op["a"], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("cid", [1, 2])
def test_vmc_gradient_pipeline_matches_oracle(cid):
    # E_loc -> FP64 stats -> surrogate weights -> LogPsi.backward, against the oracle's
    # vmc_gradient on the same samples and counts
    P = lib()
    cfg = synth.get_config(cid)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    m, named = gpu_model(cfg, beta=1.0)
    om, _ = oracle_model(cfg, beta=1.0, requires_grad=True)
    bits, counts, _ = P.nqs_sample(m, cfg.n_samples, cfg.n_samples, cfg.seed_sampler)
    eloc = P.nqs_local_energy(ham, m, bits)
    stats, ga, gp = P.nqs_energy_stats(eloc, counts)
    params = m.params.detach().clone().requires_grad_(True)
    m.bind(params)
    la, ph = P.LogPsi.apply(params, m, bits)
    ((la * ga).sum() + (ph * gp).sum()).backward()
    hb = bits.cpu().numpy().view(np.uint64)
    hc = counts.cpu().numpy()
    want_e = local_energy(om, xm, zm, coef, hb)
    want = vmc_gradient(om, hb, hc, want_e)
    assert rel_norm(params.grad.cpu().numpy().astype(np.float64), _flat(m, want)) <= 1e-4
    mean, _ = energy_stats(want_e, hc)
    assert abs(stats[0].item() - mean.real) <= 1e-5 * abs(mean)


@pytest.mark.parametrize("cid", [1, 2])
def test_vmc_steps_run_and_respect_variational_bound(cid):
    P = lib()
    cfg = synth.get_config(cid)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    m, named = gpu_model(cfg, beta=2.0)
    from oracle.lanczos import sector_hamiltonian
    st = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    lam = np.linalg.eigvalsh(sector_hamiltonian(xm, zm, coef, cfg.n_qubits, st).toarray())[0]
    vmc = P.VMC(ham, m, m.params, cfg.n_samples, mini_batches=2)
    energies = []
    for it in range(30):
        out = vmc.step(seed=cfg.seed_sampler + it)
        energies.append(out["stats"][0].item())
    assert np.all(np.isfinite(energies))
    # exact variational energy of the final parameters is above the ground energy
    la, ph = P.nqs_logpsi(m, to_dev_bits(st))
    psi = np.exp(la.cpu().numpy().astype(np.float64) + 1j * ph.cpu().numpy())
    e_var = np.real(np.vdot(psi, sector_hamiltonian(xm, zm, coef, cfg.n_qubits, st) @ psi))
    assert e_var >= lam - 1e-5 * abs(lam)


@pytest.mark.parametrize("cid", [2, 3])
def test_vmc_direct_backward_equals_autograd(cid):
    # the step's default (backward entry called with the surrogate's upstream gradients) and the
    # torch-autograd route through LogPsi produce the same gradient and the same update, bitwise
    import torch
    P = lib()
    cfg = synth.get_config(cid)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    m, _ = gpu_model(cfg, beta=1.0)
    p0 = m.params.detach().clone()
    res = []
    for autograd in (True, False):
        vmc = P.VMC(ham, m, p0.clone(), cfg.n_samples, mini_batches=2, max_unique=512, autograd=autograd)
        out = vmc.step(seed=cfg.seed_sampler + 5)
        torch.cuda.synchronize()
        res.append((out["stats"].cpu(), vmc.params.grad.detach().cpu().clone(), vmc.params.detach().cpu().clone()))
    (sa, ga, pa), (sb, gb, pb) = res
    assert torch.equal(sa, sb)
    assert torch.equal(ga, gb)
    assert torch.equal(pa, pb)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_two_phase_backward_equals_one_call(precision):
    # nqs_logpsi_backward_phase 1 (recompute) then 2 (backward) == nqs_logpsi_backward, bitwise;
    # and the VMC step that runs phase 1 on a second stream gives the same step as the one-call path
    import torch
    P = lib()
    cfg = synth.get_config(3)
    m, _ = gpu_model(cfg, beta=1.0, precision=precision)
    bits = to_dev_bits(synth.random_sector_bits(cfg.n_qubits // 2, cfg.n_up, cfg.n_dn, 700, seed=8))
    g = torch.Generator(device="cpu").manual_seed(9)
    ga = torch.randn(bits.numel(), generator=g).cuda()
    gp = torch.randn(bits.numel(), generator=g).cuda()
    one = torch.zeros(m.param_count, dtype=torch.float32, device="cuda")
    P.nqs_logpsi_backward(m, bits, ga, gp, one)
    two = torch.zeros_like(one)
    ws = m.workspace(P.OP_BACKWARD, bits.numel())
    P.nqs_logpsi_backward_phase(m, 1, bits, ws=ws)
    P.nqs_logpsi_backward_phase(m, 2, bits, ga, gp, two, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(one, two)

    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    p0 = m.params.detach().clone()
    res = []
    for overlap in (True, False):
        vmc = P.VMC(ham, m, p0.clone(), cfg.n_samples, mini_batches=1, max_unique=1024)
        vmc.overlap_backward = overlap
        out = vmc.step(seed=cfg.seed_sampler + 6)
        torch.cuda.synchronize()
        res.append((out["stats"].cpu(), vmc.params.grad.detach().cpu().clone(), vmc.params.detach().cpu().clone()))
    (sa, ga_, pa), (sb, gb, pb) = res
    assert torch.equal(sa, sb)
    assert torch.equal(ga_, gb)
    assert torch.equal(pa, pb)


@pytest.mark.parametrize("cid", [2, 3])
def test_data_parallel_gradient_form_on_one_rank(cid):
    # the data-parallel form of the gradient (nqs_energy_sums, the two backward sums, the
    # combination of paper_2208_05637_b300.parallel with no process group: one rank) equals the
    # single-process gradient of the same samples and the oracle's Eq. grad
    P = lib()
    cfg = synth.get_config(cid)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    prec = "bf16" if cfg.arch == "transformer" else "fp32"
    m, _ = gpu_model(cfg, beta=1.0, precision=prec)
    p0 = m.params.detach().clone()
    cap = {2: 512, 3: 64}[cid]
    vmc = P.VMC(ham, m, p0.clone(), cfg.n_samples, max_unique=cap)
    bits, counts, _ = P.nqs_sample(m, cfg.n_samples, cap, cfg.seed_sampler)
    out = vmc.gradient(bits, counts)
    g_single = vmc.params.grad.detach().clone()
    U = bits.numel()
    outp = vmc._gradient_parallel(bits, counts, out["eloc"], U, False)
    g_par = vmc.params.grad.detach().clone()
    # the two forms round differently (the data-parallel one subtracts 2 Re(E_bar) second from first,
    # two fp32 backward sums that partly cancel): the FP32 gradient tolerance, 1e-4
    assert rel_norm(g_par.cpu().numpy().astype(np.float64), g_single.cpu().numpy().astype(np.float64)) <= 1e-4
    st1 = out["stats"].cpu().numpy(); st2 = outp["stats"].cpu().numpy()
    assert abs(st1[0] - st2[0]) <= 1e-9 * abs(st1[0]) and abs(st1[1] - st2[1]) <= 1e-9 * max(1.0, abs(st1[0]))
    assert abs(st1[2] - st2[2]) <= 1e-6 * abs(st1[2])
    om, _ = oracle_model(cfg, beta=1.0, quant="bf16x2" if prec == "bf16" else None, requires_grad=True)
    hb = bits.cpu().numpy().view(np.uint64)
    hc = counts.cpu().numpy()
    want = vmc_gradient(om, hb, hc, local_energy(om, xm, zm, coef, hb))
    assert rel_norm(g_par.cpu().numpy().astype(np.float64), _flat(m, want)) <= (1e-3 if prec == "bf16" else 1e-4)
