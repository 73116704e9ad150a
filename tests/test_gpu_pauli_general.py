"""GPU parity on general Pauli strings and on inputs outside the sector.

Jordan-Wigner Hamiltonians of real integrals only have strings with an even number of sigma_2
factors, so their grouped sums S_g are real.  Here random particle-conserving flip patterns get
random z masks, so about half of the strings carry an odd number of sigma_2 factors and the
phase (-i)^r of Eq. mtx_element makes S_g complex: the term sweep and the local energy are
checked against the per-term definition (sigma-matrix products, oracle.pauli) with the same
tolerances as the molecular workloads.  A sample outside the (n_up, n_dn) sector gets one NaN
row from the sweep and a NaN local energy, and leaves the other samples' results unchanged.
"""
import numpy as np
import pytest

import synth
from oracle.eloc import local_energy
from oracle.models import in_sector
from oracle.pauli import matrix_element
from tests.common import check_eloc, oracle_model
from tests.gpu_common import from_dev_bits, gpu_model, lib, to_dev_bits

pytestmark = pytest.mark.gpu

N, NU, ND = 12, 2, 3
MODELS = {
    "product": dict(arch="product", n=N, n_up=NU, n_dn=ND, hidden=0, layers=0, seed=41),
    "made": dict(arch="made", n=N, n_up=NU, n_dn=ND, hidden=24, layers=2, seed=42),
    "transformer": dict(arch="transformer", n=N, n_up=NU, n_dn=ND, hidden=32, layers=2, heads=2, seed=43),
    "transformer128": dict(arch="transformer", n=N, n_up=NU, n_dn=ND, hidden=128, layers=2, heads=8, seed=44),
}


def general_hamiltonian(seed, n_terms=600):
    """Random strings whose flip pattern keeps both spin counts (none, one same-spin pair or two
    pairs) and whose z mask is uniform, so sigma_2 counts of both parities occur."""
    rng = np.random.default_rng(seed)
    xm = np.zeros(n_terms, dtype=np.uint64)
    for k in range(n_terms):
        kind = rng.integers(0, 3)
        m = 0
        for _ in range(kind):
            s = rng.integers(0, 2)
            p, q = rng.choice(N // 2, 2, replace=False)
            m ^= (1 << int(2 * p + s)) | (1 << int(2 * q + s))
        xm[k] = m
    zm = rng.integers(0, 1 << N, n_terms, dtype=np.uint64)
    c = rng.standard_normal(n_terms)
    return xm, zm, c


def test_general_hamiltonian_has_odd_sigma2_strings():
    xm, zm, _ = general_hamiltonian(1)
    r = np.bitwise_count(xm & zm) & 1
    assert 0.3 < r.mean() < 0.7


@pytest.mark.parametrize("compensated", [True, False])
def test_term_sweep_complex_groups(compensated):
    P = lib()
    xm, zm, c = general_hamiltonian(2)
    h = P.Hamiltonian(N, xm, zm, c)
    bits = synth.random_sector_bits(N // 2, NU, ND, 90, seed=3)
    ro, xp, sre, sim = P.nqs_term_sweep(h, NU, ND, to_dev_bits(bits), compensated=compensated)
    ro = ro.cpu().numpy(); xp = from_dev_bits(xp); s = sre.cpu().numpy() + 1j * sim.cpu().numpy()
    rel = 3e-7 if compensated else 1e-5
    n_complex = 0
    for i, x in enumerate(bits):
        elem = matrix_element(x, xm, zm, N)
        want = {}
        for m in np.unique(xm):
            xq = np.uint64(x ^ m)
            if in_sector(np.array([xq]), N, NU, ND)[0]:
                sel = xm == m
                want[int(xq)] = (np.sum(c[sel] * elem[sel]), np.sum(np.abs(c[sel])))
        got_x = xp[ro[i]: ro[i + 1]].tolist()
        assert sorted(got_x) == sorted(want)
        for k, v in zip(got_x, s[ro[i]: ro[i + 1]]):
            S, mass = want[k]
            n_complex += abs(S.imag) > 1e-9 * mass
            assert abs(v - S) <= rel * mass, (i, k, v, S)
    assert n_complex > 100            # the imaginary branch really ran


@pytest.mark.parametrize("name,precision", [("product", "fp32"), ("made", "fp32"), ("transformer", "fp32"),
                                            ("transformer128", "fp32"), ("transformer", "bf16"),
                                            ("transformer128", "bf16")])
def test_local_energy_complex_groups(name, precision):
    P = lib()
    xm, zm, c = general_hamiltonian(4)
    ham = P.Hamiltonian(N, xm, zm, c)
    dims = MODELS[name]
    m, _ = gpu_model(dims, beta=1.0, precision=precision)
    om, _ = oracle_model(dims, beta=1.0, quant="bf16x2" if precision == "bf16" else None)
    bits = synth.random_sector_bits(N // 2, NU, ND, 150, seed=5)
    got = P.nqs_local_energy(ham, m, to_dev_bits(bits)).cpu().numpy().astype(np.float64)
    got = got[:, 0] + 1j * got[:, 1]
    want, absum = local_energy(om, xm, zm, c, bits, return_abs=True)
    assert np.mean(np.abs(want.imag) > 1e-6 * absum) > 0.5     # complex local energies
    check_eloc(got, want, absum, precision, label=f"{name} {precision} general strings")


@pytest.mark.parametrize("name", ["made", "transformer", "transformer128"])
def test_out_of_sector_sample_gives_nan_only_for_itself(name):
    P = lib()
    cfg = synth.get_config(2)
    xm, zm, c = general_hamiltonian(6)
    ham = P.Hamiltonian(N, xm, zm, c)
    m, _ = gpu_model(MODELS[name], beta=0.5)
    good = synth.random_sector_bits(N // 2, NU, ND, 40, seed=7)
    bad = np.uint64((1 << 0) | (1 << 2) | (1 << 4) | (1 << 1))        # 3 up, 1 down electrons
    assert not in_sector(np.array([bad]), N, NU, ND)[0]
    mixed = np.concatenate([good[:17], [bad], good[17:]])
    # the sweep: one NaN row x' = x for the bad sample, the others' rows as without it
    ro, xp, sre, _ = P.nqs_term_sweep(ham, NU, ND, to_dev_bits(mixed))
    ro = ro.cpu().numpy()
    assert ro[18] - ro[17] == 1
    assert from_dev_bits(xp)[ro[17]] == bad and np.isnan(sre.cpu().numpy()[ro[17]])
    ro0, xp0, sre0, _ = P.nqs_term_sweep(ham, NU, ND, to_dev_bits(good))
    keep = np.r_[0:ro[17], ro[18]:ro[-1]]
    assert np.array_equal(from_dev_bits(xp)[keep], from_dev_bits(xp0))
    # the local energy: NaN for the bad sample, the others as in the batch without it (bit for bit
    # for MADE; the transformer's grouped attention rescales its softmax per warp, so there the
    # batch composition may move the last bits)
    e_mix = P.nqs_local_energy(ham, m, to_dev_bits(mixed)).cpu().numpy()
    e_good = P.nqs_local_energy(ham, m, to_dev_bits(good)).cpu().numpy()
    assert np.all(np.isnan(e_mix[17]))
    rest = np.delete(e_mix, 17, axis=0)
    assert np.all(np.isfinite(rest))
    if name == "made":
        assert np.array_equal(rest, e_good)
    else:
        assert np.max(np.abs(rest - e_good)) <= 1e-6 * np.max(np.abs(e_good))
    del cfg
