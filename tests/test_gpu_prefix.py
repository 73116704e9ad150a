"""GPU parity of the transformer local energy with prefix reuse (Section 5.1's unique flippings
applied to prefixes: the row at sampling position t depends on the bits before t only).

Depth 0 evaluates every connected x' from position 0; depths 1-3 take the rows before an x''s
first, second or third flip from the sample or from shared one- and two-flip strings, with
their keys and values cached per layer.  Every row is computed by the same kernels and its keys
and values are the same numbers wherever they are read from, so all depths must give the same
local energies bit for bit; each is also checked against the FP64 oracle (norm 1e-5 FP32,
1e-4 compensated BF16 against the quantisation-aware oracle; element-wise ten times that), on
molecular and general (odd sigma_2) Hamiltonians and in the reverse, forward and a shuffled
sampling order.
"""
import numpy as np
import pytest

import synth
from oracle.eloc import local_energy
from tests.common import check_eloc, oracle_model
from tests.gpu_common import gpu_model, lib, to_dev_bits
from tests.test_gpu_pauli_general import general_hamiltonian

pytestmark = pytest.mark.gpu

TF32 = dict(arch="transformer", n=12, n_up=2, n_dn=3, hidden=32, layers=2, heads=2, seed=71)
TF64 = dict(arch="transformer", n=14, n_up=3, n_dn=2, hidden=64, layers=2, heads=4, seed=72)
TF128 = dict(arch="transformer", n=16, n_up=3, n_dn=3, hidden=128, layers=2, heads=8, seed=73)


def _order(n, kind):
    if kind == "reverse":
        return synth.default_order(n)
    if kind == "forward":
        return np.arange(n)
    return np.random.default_rng(n).permutation(n)


def _molecular(n):
    h, eri, _ = synth.integrals(n // 2, 0, True, 91)
    return synth.jordan_wigner(h, eri)


@pytest.mark.parametrize("dims", [TF32, TF64, TF128])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("order_kind", ["reverse", "forward", "shuffled"])
def test_prefix_reuse_depths_agree_and_match_oracle(dims, precision, order_kind):
    P = lib()
    n = dims["n"]
    order = _order(n, order_kind)
    xm, zm, coef = _molecular(n)
    ham = P.Hamiltonian(n, xm, zm, coef)
    m, _ = gpu_model(dims, beta=1.0, precision=precision, order=order)
    bits = synth.random_sector_bits(n // 2, dims["n_up"], dims["n_dn"], 70, seed=17)
    bt = to_dev_bits(bits)
    res = {}
    for depth in (0, 1, 2, 3):
        m.set_prefix_reuse(depth)
        res[depth] = P.nqs_local_energy(ham, m, bt).cpu().numpy()
    for depth in (1, 2, 3):
        assert np.array_equal(res[depth], res[0]), f"depth {depth} differs from depth 0"
    om, _ = oracle_model(dims, beta=1.0, quant="bf16x2" if precision == "bf16" else None, order=order)
    want, absum = local_energy(om, xm, zm, coef, bits, return_abs=True)
    got = res[3][:, 0].astype(np.float64) + 1j * res[3][:, 1]
    check_eloc(got, want, absum, precision, label=f"d={dims['hidden']} {precision} {order_kind} prefix reuse")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_prefix_reuse_general_strings_and_chunks(precision):
    # complex groups, 150 samples (several chunks at 64 samples each, ragged tail), repeats
    P = lib()
    from tests.test_gpu_pauli_general import MODELS, N, NU, ND
    dims = MODELS["transformer128"]
    xm, zm, c = general_hamiltonian(8)
    ham = P.Hamiltonian(N, xm, zm, c)
    m, _ = gpu_model(dims, beta=1.0, precision=precision)
    base = synth.random_sector_bits(N // 2, NU, ND, 120, seed=9)
    bits = np.concatenate([base, base[:30]])
    m.set_prefix_reuse(3)
    got3 = P.nqs_local_energy(ham, m, to_dev_bits(bits)).cpu().numpy()
    m.set_prefix_reuse(0)
    got0 = P.nqs_local_energy(ham, m, to_dev_bits(bits)).cpu().numpy()
    assert np.array_equal(got3, got0)
    assert np.array_equal(got3[120:], got3[:30])
    om, _ = oracle_model(dims, beta=1.0, quant="bf16x2" if precision == "bf16" else None)
    want, absum = local_energy(om, xm, zm, c, base, return_abs=True)
    g = got3[:120, 0].astype(np.float64) + 1j * got3[:120, 1]
    check_eloc(g, want, absum, precision, label=f"general strings {precision} prefix reuse")


@pytest.mark.parametrize("cid", [4, 5])
def test_prefix_reuse_depths_agree_on_the_large_workloads(cid):
    P = lib()
    cfg = synth.get_config(cid)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    m, _ = gpu_model(cfg, beta=2.0, precision="bf16")
    bits = synth.random_sector_bits(cfg.n_orb, cfg.n_up, cfg.n_dn, 6 if cid == 5 else 40, seed=23)
    bt = to_dev_bits(bits)
    m.set_prefix_reuse(3)
    e3 = P.nqs_local_energy(ham, m, bt).cpu().numpy()
    m.set_prefix_reuse(1)
    e1 = P.nqs_local_energy(ham, m, bt).cpu().numpy()
    assert np.all(np.isfinite(e3))
    assert np.array_equal(e3, e1)


def test_prefix_reuse_setter_validates():
    P = lib()
    m, _ = gpu_model(TF32)
    with pytest.raises(P.NQSError):
        m.set_prefix_reuse(4)
    made, _ = gpu_model(dict(arch="made", n=8, n_up=2, n_dn=2, hidden=8, layers=1, seed=3))
    with pytest.raises(P.NQSError) as e:
        made.set_prefix_reuse(2)
    assert e.value.status == P.NQS_ERR_UNSUPPORTED
