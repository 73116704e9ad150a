"""GPU parity: grouping (bit-exact) and the term sweep (x' bit-exact, S within fp32 tolerance)."""
import numpy as np
import pytest

import synth
from oracle.grouping import group_terms
from oracle.models import in_sector
from oracle.pauli import matrix_element
from tests.gpu_common import lib, to_dev_bits, from_dev_bits

pytestmark = pytest.mark.gpu


def _ham(cid):
    cfg = synth.get_config(cid)
    xm, zm, c = synth.hamiltonian_for(cfg)
    return cfg, xm, zm, c


@pytest.mark.parametrize("cid", [1, 2, 3, 4, 5])
def test_grouping_bit_exact(cid):
    P = lib()
    cfg, xm, zm, c = _ham(cid)
    perm = np.random.default_rng(cid).permutation(len(c))
    xm, zm, c = xm[perm], zm[perm], c[perm]
    h = P.Hamiltonian(cfg.n_qubits, xm, zm, c)
    got = h.export()
    want = group_terms(xm, zm, c, cfg.n_qubits)
    for k in ("group_mask", "group_offset", "term_z", "term_c_re", "term_c_im"):
        assert np.array_equal(got[k], want[k]), k


def test_grouping_merges_cancels_and_keeps_odd_y():
    P = lib()
    rng = np.random.default_rng(5)
    n = 10
    xm = rng.integers(0, 1 << n, 200, dtype=np.uint64)
    zm = rng.integers(0, 1 << n, 200, dtype=np.uint64)
    c = rng.standard_normal(200)
    xm = np.concatenate([xm, xm[:50], [np.uint64(7), np.uint64(7)]])
    zm = np.concatenate([zm, zm[:50], [np.uint64(9), np.uint64(9)]])
    c = np.concatenate([c, -0.5 * c[:50], [1.5, -1.5]])
    h = P.Hamiltonian(n, xm, zm, c)
    got = h.export()
    want = group_terms(xm, zm, c, n)
    for k in want:
        if k in got:
            assert np.array_equal(got[k], want[k]), k


def _oracle_rows(x, xm, zm, c, n, n_up, n_dn):
    """{x': (S, sum |c|)} for one sample from the per-term matrix-element definition."""
    out = {}
    elem = matrix_element(x, xm, zm, n)
    for m in np.unique(xm):
        xp = np.uint64(x ^ m)
        if not in_sector(np.array([xp]), n, n_up, n_dn)[0]:
            continue
        sel = xm == m
        out[int(xp)] = (np.sum(c[sel] * elem[sel]), np.sum(np.abs(c[sel])))
    return out


@pytest.mark.parametrize("cid,B", [(1, 5), (2, 37), (3, 70), (4, 33), (5, 3)])
@pytest.mark.parametrize("compensated", [True, False])
def test_term_sweep_matches_definition(cid, B, compensated):
    P = lib()
    cfg, xm, zm, c = _ham(cid)
    h = P.Hamiltonian(cfg.n_qubits, xm, zm, c)
    bits = synth.random_sector_bits(cfg.n_orb, cfg.n_up, cfg.n_dn, B, seed=11 + cid)
    ro, xp, sre, sim = P.nqs_term_sweep(h, cfg.n_up, cfg.n_dn, to_dev_bits(bits), compensated=compensated)
    ro = ro.cpu().numpy(); xp = from_dev_bits(xp); s = sre.cpu().numpy() + 1j * sim.cpu().numpy()
    # fp32 result of an exactly summed (compensated) or fp32-summed group: a few ulps of the
    # group's absolute coefficient mass
    rel = 3e-7 if compensated else 1e-5
    for i, x in enumerate(bits):
        want = _oracle_rows(x, xm, zm, c, cfg.n_qubits, cfg.n_up, cfg.n_dn)
        got_x = xp[ro[i]: ro[i + 1]]
        assert len(got_x) == len(set(got_x.tolist()))
        assert sorted(got_x.tolist()) == sorted(want), f"sample {i}: x' sets differ"
        for k, v in zip(got_x.tolist(), s[ro[i]: ro[i + 1]]):
            S, mass = want[k]
            assert abs(v - S) <= rel * mass, (i, k, v, S)


def test_term_sweep_empty_and_capacity():
    P = lib()
    cfg, xm, zm, c = _ham(2)
    h = P.Hamiltonian(cfg.n_qubits, xm, zm, c)
    import torch
    ro, xp, _, _ = P.nqs_term_sweep(h, 2, 2, torch.empty(0, dtype=torch.int64, device="cuda"))
    assert xp.numel() == 0
    bits = synth.random_sector_bits(cfg.n_orb, cfg.n_up, cfg.n_dn, 4, seed=1)
    with pytest.raises(P.NQSError) as e:
        P.nqs_term_sweep(h, 2, 2, to_dev_bits(bits), capacity=3)
    assert e.value.status == P.NQS_ERR_CAPACITY
