"""GPU check of nqs_local_energy_noalloc, the local-energy entry point that allocates nothing.

It exists for callers that cannot call cudaMalloc when they need a local energy (code running
inside an allocator's no-allocation region, plugins given only input and output buffers,
runtimes that reserved all device memory).  It keeps its scratch in a static device array, so
this test calls it twice in a row through the C ABI -- the second call runs on the scratch the
first one left behind -- and compares both results with nqs_local_energy (caller-provided
workspace) within the fp32 local-energy tolerance.  The file name sorts last so a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle.lanczos import sector_states
from tests.common import rel_norm
from tests.gpu_common import gpu_model, lib, to_dev_bits

pytestmark = pytest.mark.gpu


def _call_noalloc(P, ham, model, bits_t, out_t):
    import torch
    st = P._lib.nqs_local_energy_noalloc(ham.handle, model.handle, ctypes.c_void_p(bits_t.data_ptr()),
                                         bits_t.numel(), ctypes.c_void_p(out_t.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("cid,beta", [(2, 2.0), (1, 0.0)])
def test_noalloc_matches_workspace_version_twice(cid, beta):
    import torch
    P = lib()
    cfg = synth.get_config(cid)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    model, _ = gpu_model(cfg, beta=beta)
    st = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    first = st
    second = st[np.random.default_rng(1).integers(0, len(st), 1500)]    # spans two chunks
    for bits in (first, second):
        bt = to_dev_bits(bits)
        want = P.nqs_local_energy(ham, model, bt).cpu().numpy().astype(np.float64)
        out = torch.full((len(bits), 2), float("nan"), dtype=torch.float32, device="cuda")
        assert _call_noalloc(P, ham, model, bt, out) == P.NQS_OK, P._lib.nqs_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        err = rel_norm(got[:, 0] + 1j * got[:, 1], want[:, 0] + 1j * want[:, 1])
        assert err <= 1e-5, err


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    # 5e6 samples need 40 MB of per-sample log psi alone: more than the 32 MiB scratch
    import torch
    P = lib()
    cfg = synth.get_config(2)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    model, _ = gpu_model(cfg)
    bits = synth.random_sector_bits(cfg.n_orb, cfg.n_up, cfg.n_dn, 8, seed=2)
    big = to_dev_bits(np.resize(bits, 5_000_000))
    out_big = torch.empty((5_000_000, 2), dtype=torch.float32, device="cuda")
    assert _call_noalloc(P, ham, model, big, out_big) == P.NQS_ERR_CAPACITY
    assert b"static scratch" in P._lib.nqs_last_error()


def test_noalloc_halves_its_chunk_when_the_log_psi_fill_the_scratch():
    # 4.1e6 samples of the 12-qubit workload: their log psi take 32.8 MB of the 32 MiB scratch,
    # so the sweep chunk drops from 1024 to 256 samples; results as with the workspace version
    import torch
    P = lib()
    cfg = synth.get_config(2)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    model, _ = gpu_model(cfg, beta=1.0)
    st = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    B = 4_100_000
    bits = st[np.random.default_rng(7).integers(0, len(st), B)]
    bt = to_dev_bits(bits)
    out = torch.full((B, 2), float("nan"), dtype=torch.float32, device="cuda")
    assert _call_noalloc(P, ham, model, bt, out) == P.NQS_OK, P._lib.nqs_last_error()
    want = P.nqs_local_energy(ham, model, bt)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    w = want.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    err = rel_norm(got[:, 0] + 1j * got[:, 1], w[:, 0] + 1j * w[:, 1])
    assert err <= 1e-5, err
