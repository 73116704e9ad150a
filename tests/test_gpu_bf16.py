"""GPU parity for the BF16 tensor-core transformer path.

Two forms: the compensated one (default; every GEMM input activation is hi + lo bf16, weights
bf16) is gated against the matching quantisation-aware FP64 oracle (quant="bf16x2"): local
energy rel_norm <= 1e-4, gradient rel_norm <= 1e-3, sampler bit-exact under trace replay.  The
plain form (single bf16 activations) is checked against quant="bf16" with looser bounds: its
rounding-boundary flips of activations move log|psi| by up to ~1e-3.  The error against the
unquantised FP64 oracle (the cost of bf16 weights) is printed, not gated."""
import numpy as np
import pytest

import synth
from oracle.eloc import local_energy
from oracle.models import in_sector
from oracle.sampler import sample
from tests.common import check_eloc, oracle_model, rel_norm
from tests.gpu_common import from_dev_bits, gpu_model, lib, to_dev_bits

pytestmark = pytest.mark.gpu

TF_D64 = dict(arch="transformer", n=12, n_up=2, n_dn=3, hidden=64, layers=2, heads=4, seed=71)
TF_D128 = dict(arch="transformer", n=16, n_up=3, n_dn=3, hidden=128, layers=2, heads=8, seed=72)


def _cfg(c):
    return synth.get_config(c) if isinstance(c, int) else c


def _dims(cfg):
    if isinstance(cfg, dict):
        return cfg["n"], cfg["n_up"], cfg["n_dn"]
    return cfg.n_qubits, cfg.n_up, cfg.n_dn


@pytest.mark.parametrize("c", [TF_D64, TF_D128, 3])
@pytest.mark.parametrize("comp", [True, False])
def test_bf16_logpsi_against_quantised_oracle(c, comp):
    P = lib()
    cfg = _cfg(c)
    n, nu, nd = _dims(cfg)
    m, _ = gpu_model(cfg, beta=1.0, precision="bf16", compensated=comp)
    oq, _ = oracle_model(cfg, beta=1.0, quant="bf16x2" if comp else "bf16")
    o64, _ = oracle_model(cfg, beta=1.0)
    bits = synth.random_sector_bits(n // 2, nu, nd, 400, seed=3)
    la, ph = P.nqs_logpsi(m, to_dev_bits(bits))
    la = la.cpu().numpy().astype(np.float64); ph = ph.cpu().numpy().astype(np.float64)
    qla, qph = oq.log_psi(bits)
    fla, fph = o64.log_psi(bits)
    dq = np.max(np.abs(la - qla)); dp = np.max(np.abs(ph - qph))
    d64 = np.max(np.abs(la - fla))
    print(f"bf16 (comp={comp}) log|psi| vs quantised oracle {dq:.2e}, phase {dp:.2e}; vs fp64 oracle {d64:.2e}")
    if comp:
        assert dq <= 2e-5 * (1 + np.max(np.abs(qla))) and dp <= 2e-5 * (1 + np.max(np.abs(qph)))
    else:
        assert dq <= 3e-3 and dp <= 3e-3
        assert np.median(np.abs(la - qla)) <= 2e-4
    assert d64 <= 0.1


@pytest.mark.parametrize("c,B", [(TF_D64, 120), (TF_D128, 60), (3, 40)])
def test_bf16_local_energy_against_quantised_oracle(c, B):
    P = lib()
    cfg = _cfg(c)
    n, nu, nd = _dims(cfg)
    if isinstance(c, int):
        xm, zm, coef = synth.hamiltonian_for(cfg)
    else:
        h, eri, _ = synth.integrals(n // 2, 0, True, 89)
        xm, zm, coef = synth.jordan_wigner(h, eri)
    bits = synth.random_sector_bits(n // 2, nu, nd, B, seed=6)
    ham = P.Hamiltonian(n, xm, zm, coef)
    m, _ = gpu_model(cfg, beta=1.0, precision="bf16")
    oq, _ = oracle_model(cfg, beta=1.0, quant="bf16x2")
    o64, _ = oracle_model(cfg, beta=1.0)
    got = P.nqs_local_energy(ham, m, to_dev_bits(bits)).cpu().numpy().astype(np.float64)
    got = got[:, 0] + 1j * got[:, 1]
    wq, absum = local_energy(oq, xm, zm, coef, bits, return_abs=True)
    w64 = local_energy(o64, xm, zm, coef, bits)
    e64 = rel_norm(got, w64)
    print(f"bf16 E_loc rel_norm vs fp64 oracle {e64:.2e} (reported, not gated)")
    check_eloc(got, wq, absum, "bf16", label="bf16 vs quantised oracle")


# d_model 64 / four heads runs the one-kernel sampler step: compensated and plain bf16 forms,
# with and without eviction (max_unique below the unique count), and the 20-qubit workload with
# its 1024-sample buffer; called twice, so the second call replays the captured graph.
@pytest.mark.parametrize("c,comp,n_samples,max_unique", [(TF_D64, True, 20_000, 10**6), (TF_D64, False, 20_000, 10**6),
                                                         (TF_D64, True, 20_000, 40), (3, True, 100_000, 1024)])
def test_bf16_sampler_trace_replay(c, comp, n_samples, max_unique):
    P = lib()
    cfg = _cfg(c)
    m, _ = gpu_model(cfg, beta=1.0, precision="bf16", compensated=comp)
    oq, _ = oracle_model(cfg, beta=1.0, quant="bf16x2" if comp else "bf16")
    seed = 99
    for call in range(2):
        bits, counts, trace = P.nqs_sample(m, n_samples, max_unique, seed + call, trace=True)
        trace = trace.cpu().numpy()
        diffs = []

        def replay(parent_bits, k):
            p = trace[k, : len(parent_bits)]
            diffs.append(np.max(np.abs(p.astype(np.float64) - oq.sampling_p(parent_bits, k))))
            return p

        wb, wc = sample(replay, oq.n, oq.order, n_samples, max_unique, seed + call)
        assert np.array_equal(from_dev_bits(bits), wb)
        assert np.array_equal(counts.cpu().numpy(), wc)
        # the plain form's activation rounding flips move p by up to ~1e-4 (log|psi| bounds above)
        assert max(diffs) <= (1e-5 if comp else 1e-3)
        assert np.all(in_sector(wb, oq.n, oq.n_up, oq.n_dn))


@pytest.mark.parametrize("c,comp", [(TF_D64, True), (3, True), (TF_D64, False)])
def test_bf16_backward_against_quantised_oracle(c, comp):
    import torch
    from oracle.vmc import logpsi_vjp
    P = lib()
    cfg = _cfg(c)
    n, nu, nd = _dims(cfg)
    m, _ = gpu_model(cfg, beta=1.0, precision="bf16", compensated=comp)
    oq, _ = oracle_model(cfg, beta=1.0, quant="bf16x2" if comp else "bf16", requires_grad=True)
    bits = synth.random_sector_bits(n // 2, nu, nd, 120, seed=7)
    rng = np.random.default_rng(8)
    ga = rng.standard_normal(len(bits)).astype(np.float32)
    gp = rng.standard_normal(len(bits)).astype(np.float32)
    grad = torch.zeros(m.param_count, dtype=torch.float32, device="cuda")
    P.nqs_logpsi_backward(m, to_dev_bits(bits), torch.tensor(ga, device="cuda"),
                          torch.tensor(gp, device="cuda"), grad)
    want = logpsi_vjp(oq, bits, ga.astype(np.float64), gp.astype(np.float64))
    flat = np.concatenate([np.asarray(want[nm]).ravel() for nm, _, _ in m.param_layout()])
    err = rel_norm(grad.cpu().numpy().astype(np.float64), flat)
    print(f"bf16 gradient rel_norm vs quantised oracle {err:.2e}")
    assert err <= 1e-3, err
