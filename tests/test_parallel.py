"""The data-parallel VMC gradient exchange on two CPU ranks (gloo): every rank holds its own
samples, computes its FP64 sums and its two backward sums with the oracle, and one all-reduce in
paper_2208_05637_b300.parallel.combine must give, on every rank, the gradient of Eq. grad (and the
energy statistics) of the union of the samples as the single-process oracle computes them."""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle.eloc import local_energy
from oracle.lanczos import sector_states
from oracle.vmc import energy_stats, logpsi_vjp, vmc_gradient
from tests.common import oracle_model


def _parallel_module():
    # the module imports torch only; load it by path so the test needs no built library
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("nqs_parallel", os.path.join(root, "paper_2208_05637_b300", "parallel.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _problem(cid):
    cfg = synth.get_config(cid)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    st = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    rng = np.random.default_rng(5)
    bits = st[rng.choice(len(st), min(len(st), 60), replace=False)]
    counts = rng.integers(1, 40, len(bits)).astype(np.int64)
    return cfg, xm, zm, coef, bits, counts


def _flat(model, grads):
    return np.concatenate([np.asarray(grads[k]).ravel() for k in model.p])


def _rank(rank, world, port, cid, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg, xm, zm, coef, bits, counts = _problem(cid)
        mine = np.arange(len(bits)) % world == rank          # disjoint shares
        b, w = bits[mine], counts[mine].astype(np.float64)
        om, _ = oracle_model(cfg, beta=1.0, requires_grad=True)
        e = local_energy(om, xm, zm, coef, b)
        sums = torch.tensor([np.sum(w * e.real), np.sum(w * e.imag), np.sum(w * np.abs(e) ** 2), np.sum(w)])
        first = _flat(om, logpsi_vjp(om, b, 2 * w * e.real, 2 * w * e.imag))
        second = _flat(om, logpsi_vjp(om, b, w, np.zeros_like(w)))
        par = _parallel_module()
        grad, stats = par.combine(sums, torch.tensor(first), torch.tensor(second))
        np.save(os.path.join(out_dir, f"grad{rank}.npy"), grad.numpy())
        np.save(os.path.join(out_dir, f"stats{rank}.npy"), stats.numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("cid", [1, 2])
def test_two_rank_gradient_equals_single_process_gradient(cid):
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(2, _free_port(), cid, d), nprocs=2, start_method="spawn")
        g0, g1 = (np.load(os.path.join(d, f"grad{r}.npy")) for r in range(2))
        s0, s1 = (np.load(os.path.join(d, f"stats{r}.npy")) for r in range(2))
    assert np.array_equal(g0, g1) and np.array_equal(s0, s1)     # identical on every rank
    cfg, xm, zm, coef, bits, counts = _problem(cid)
    om, _ = oracle_model(cfg, beta=1.0, requires_grad=True)
    e = local_energy(om, xm, zm, coef, bits)
    want = _flat(om, vmc_gradient(om, bits, counts, e))
    # fp32 result of an FP64 combination
    assert np.linalg.norm(g0 - want) <= 1e-6 * np.linalg.norm(want)
    mean, var = energy_stats(e, counts)
    assert abs(s0[0] - mean.real) <= 1e-12 * abs(mean) and abs(s0[1] - mean.imag) <= 1e-12 * abs(mean)
    assert abs(s0[2] - var) <= 1e-9 * max(var, 1.0) and s0[3] == counts.sum()


def test_single_process_combine_is_the_plain_formula():
    # without a process group the combination is the one-rank case of the same formula
    par = _parallel_module()
    rng = np.random.default_rng(3)
    first, second = rng.standard_normal(7), rng.standard_normal(7)
    sums = np.array([3.0, -1.0, 10.0, 4.0])
    g, st = par.combine(torch.tensor(sums), torch.tensor(first), torch.tensor(second))
    np.testing.assert_allclose(g.numpy(), (first - 2 * (3.0 / 4.0) * second) / 4.0, rtol=1e-6)
    np.testing.assert_allclose(st.numpy(), [0.75, -0.25, 10.0 / 4 - (0.75 ** 2 + 0.25 ** 2), 4.0])
