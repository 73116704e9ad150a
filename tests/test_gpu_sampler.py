"""GPU parity: unique-sample sampling with counts.

Integer results are compared bit-exactly.  With the product model both sides use the same fp32
probabilities, so the whole output must match; with MADE the GPU's per-step fp32 probabilities
(its trace) are replayed through the oracle's sampler, which must reproduce every step's buffer
exactly, and the traced probabilities must agree with the oracle's FP64 conditionals."""
import numpy as np
import pytest

import synth
from oracle.models import in_sector
from oracle.sampler import sample, model_p_fn
from tests.common import oracle_model
from tests.gpu_common import gpu_model, lib, from_dev_bits

pytestmark = pytest.mark.gpu

PROD = dict(arch="product", n=16, n_up=3, n_dn=2, hidden=0, layers=0, seed=41)


@pytest.mark.parametrize("n_samples,max_unique,seed", [(1, 1, 3), (1000, 10**6, 4), (100_000, 10**6, 5),
                                                       (20_000, 37, 6), (5000, 1, 7)])
def test_product_model_bit_exact(n_samples, max_unique, seed):
    P = lib()
    m, params = gpu_model(PROD, beta=0.5)
    om, _ = oracle_model(PROD, beta=0.5)
    bits, counts, _ = P.nqs_sample(m, n_samples, max_unique, seed)
    wb, wc = sample(model_p_fn(om), om.n, om.order, n_samples, max_unique, seed)
    assert np.array_equal(from_dev_bits(bits), wb)
    assert np.array_equal(counts.cpu().numpy(), wc)


@pytest.mark.parametrize("cid,n_samples,max_unique,beta", [(1, 1024, 10**6, 2.0), (2, 10_000, 10**6, 0.0),
                                                           (2, 10_000, 10**6, 2.0), (2, 10_000, 40, 0.0)])
def test_made_trace_replay_bit_exact(cid, n_samples, max_unique, beta):
    P = lib()
    cfg = synth.get_config(cid)
    m, _ = gpu_model(cfg, beta=beta)
    om, _ = oracle_model(cfg, beta=beta)
    seed = cfg.seed_sampler
    bits, counts, trace = P.nqs_sample(m, n_samples, max_unique, seed, trace=True)
    trace = trace.cpu().numpy()
    steps = []

    def replay(parent_bits, k):
        p_gpu = trace[k, : len(parent_bits)]
        p_orc = om.sampling_p(parent_bits, k)
        steps.append(np.max(np.abs(p_gpu.astype(np.float64) - p_orc)) if len(p_orc) else 0.0)
        return p_gpu

    wb, wc = sample(replay, om.n, om.order, n_samples, max_unique, seed)
    assert np.array_equal(from_dev_bits(bits), wb)
    assert np.array_equal(counts.cpu().numpy(), wc)
    assert max(steps) <= 2e-6
    assert counts.sum().item() <= n_samples
    assert np.all(in_sector(wb, om.n, om.n_up, om.n_dn))
    if max_unique >= n_samples:
        assert counts.sum().item() == n_samples


def test_capacity_error_reports_needed_size():
    P = lib()
    m, _ = gpu_model(PROD, beta=0.0)
    import ctypes
    import torch
    ws = m.workspace(P.OP_SAMPLE, 5000)
    out_b = torch.empty(2, dtype=torch.int64, device="cuda")
    out_c = torch.empty(2, dtype=torch.int64, device="cuda")
    nu = ctypes.c_int64()
    st = P._lib.nqs_sample(m.handle, 5000, 10**6, 1, P._ptr(out_b), P._ptr(out_c), 2, ctypes.byref(nu),
                           None, 0, P._ptr(ws), ws.numel(), P._stream())
    assert st == P.NQS_ERR_CAPACITY and nu.value > 2
