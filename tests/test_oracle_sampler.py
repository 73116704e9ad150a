"""Pins for Philox4x32-10 and the unique-sample buffer sampler (paper Section 4, Sampling)."""
import os

import numpy as np
import pytest
from scipy import stats

import synth
from oracle.lanczos import sector_states
from oracle.models import in_sector
from oracle.sampler import bernoulli_ones, evict, philox4x32_10, sample, model_p_fn, threshold
from tests.common import oracle_model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [int(t, 16) for t in r]
        out = philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_threshold_is_exact_at_the_ends():
    assert int(threshold(np.float32(1.0))) == 1 << 32
    assert int(threshold(np.float32(0.0))) == 0
    assert int(threshold(np.float32(0.5))) == 1 << 31
    p = np.float32(0.3)
    assert int(threshold(p)) == int(np.floor(np.float64(p) * 2.0 ** 32))


def _chi2_vs_exact(model, n_samples, seed):
    bits, counts = sample(model_p_fn(model), model.n, model.order, n_samples, 1 << 30, seed)
    assert counts.sum() == n_samples
    assert np.all(counts > 0)
    assert np.all(np.diff(bits.astype(np.float64)) > 0)
    assert np.all(in_sector(bits, model.n, model.n_up, model.n_dn))
    st = sector_states(model.n // 2, model.n_up, model.n_dn)
    la, _ = model.log_psi(st)
    prob = np.exp(2 * la)
    obs = np.zeros(len(st))
    obs[np.searchsorted(st, bits)] = counts
    exp = prob * n_samples
    big = exp >= 5
    chi2 = np.sum((obs[big] - exp[big]) ** 2 / exp[big]) + \
        (obs[~big].sum() - exp[~big].sum()) ** 2 / max(exp[~big].sum(), 1e-9)
    dof = int(big.sum())
    return stats.chi2.sf(chi2, dof)


@pytest.mark.parametrize("dims,beta", [(1, 2.0), (2, 0.0), (2, 2.0),
                                       (dict(arch="product", n=8, n_up=2, n_dn=1, hidden=0,
                                             layers=0, seed=3), 0.5)])
def test_sampler_distribution_matches_born_probabilities(dims, beta):
    cfg = synth.get_config(dims) if isinstance(dims, int) else dims
    model, _ = oracle_model(cfg, beta=beta)
    pval = _chi2_vs_exact(model, 200_000, 42)
    assert pval > 1e-3


def test_sampler_eviction_keeps_top_counts():
    model, _ = oracle_model(synth.get_config(2), beta=0.0)
    trace = []
    bits, counts = sample(model_p_fn(model), model.n, model.order, 10_000, 50, 7, trace=trace)
    assert len(bits) <= 50
    assert np.all(np.diff(bits.astype(np.float64)) > 0)
    # replaying the trace step by step reproduces each step's eviction rule
    for k in range(len(trace) - 1):
        pb, pc, _ = trace[k]
        nb, nc, _ = trace[k + 1]
        assert len(nb) <= 50 and nc.sum() <= pc.sum()


def test_sampler_deterministic_and_seed_dependent():
    model, _ = oracle_model(synth.get_config(1), beta=0.0)
    a = sample(model_p_fn(model), 4, model.order, 1024, 1 << 30, 1)
    b = sample(model_p_fn(model), 4, model.order, 1024, 1 << 30, 1)
    c = sample(model_p_fn(model), 4, model.order, 1024, 1 << 30, 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))


def test_sampler_single_nominal_sample_follows_draws():
    # brute force for N_s = 1: each step the lone sample takes bit 1 iff its Philox word is
    # below the threshold of its conditional (nominal index 0, step k)
    model, _ = oracle_model(synth.get_config(2), beta=0.0)
    seed = 123
    bits, counts = sample(model_p_fn(model), model.n, model.order, 1, 1, seed)
    x = np.zeros(1, dtype=np.uint64)
    for k in range(model.n):
        p = model.sampling_p(x, k).astype(np.float32)
        u = philox4x32_10(0, k, 0, 0, seed & 0xFFFFFFFF, seed >> 32)[0]
        if int(u) < int(threshold(p)[0]):
            x |= np.uint64(1) << np.uint64(model.order[k])
    assert counts.tolist() == [1] and bits.tolist() == x.tolist()


def test_eviction_rule_on_a_hand_built_buffer():
    # Section 4, Sampling: the entries with the lowest numbers of occurrences are evicted; the
    # tie-break (bits ascending) is this build's reading.  The survivors below are written by
    # hand from that rule: counts 7 (bits 3) and 4 (bits 5) first, then the count-2 tie among
    # bits 1, 7, 9 in ascending bit order, then the count-1 tie among bits 2 and 12.
    bits = np.array([1, 2, 3, 5, 7, 9, 12], dtype=np.uint64)
    counts = np.array([2, 1, 7, 4, 2, 2, 1], dtype=np.int64)
    want = {
        1: ([3], [7]),
        2: ([3, 5], [7, 4]),
        3: ([1, 3, 5], [2, 7, 4]),
        4: ([1, 3, 5, 7], [2, 7, 4, 2]),
        5: ([1, 3, 5, 7, 9], [2, 7, 4, 2, 2]),
        6: ([1, 2, 3, 5, 7, 9], [2, 1, 7, 4, 2, 2]),
        7: ([1, 2, 3, 5, 7, 9, 12], [2, 1, 7, 4, 2, 2, 1]),
        9: ([1, 2, 3, 5, 7, 9, 12], [2, 1, 7, 4, 2, 2, 1]),
    }
    for mu, (wb, wc) in want.items():
        b, c = evict(bits, counts, mu)
        assert b.tolist() == wb and c.tolist() == wc, mu


def test_sampler_applies_the_eviction_rule_at_the_step_that_overflows():
    # A step-dependent p makes the buffer overflow only at the last step: p = 1/2 at steps 0
    # and n-1, p = 0 in between (no split).  The sampler with max_unique = 2 must then equal
    # the unevicted run cut by the hand-pinned rule above, and the seed is chosen so that the
    # cut falls inside a tie of counts (so the bits-ascending tie-break decides).
    n, N = 6, 40
    order = np.arange(n)[::-1]

    def p_fn(parent_bits, k):
        return np.full(len(parent_bits), 0.5 if k in (0, n - 1) else 0.0, dtype=np.float32)

    seed = None
    for s in range(1, 400):
        b_all, c_all = sample(p_fn, n, order, N, 1 << 30, s)
        srt = np.sort(c_all)[::-1]
        if len(c_all) == 4 and srt[1] == srt[2]:
            seed = s
            break
    assert seed is not None
    b_all, c_all = sample(p_fn, n, order, N, 1 << 30, seed)
    b2, c2 = sample(p_fn, n, order, N, 2, seed)
    wb, wc = evict(b_all, c_all, 2)
    assert b2.tolist() == wb.tolist() and c2.tolist() == wc.tolist()
    # the tie at the cut is broken toward the smaller bitstring
    tied = np.sort(c_all)[::-1][1]
    cand = b_all[c_all == tied]
    assert cand.min() in b2 and cand.max() not in b2


def test_nominal_indices_after_eviction_run_over_the_survivors():
    # after an eviction the surviving parents own consecutive nominal indices from 0 in
    # bits-ascending order (the dropped entries' draws are not consumed)
    counts = np.array([3, 5, 2], dtype=np.int64)
    thr = threshold(np.array([0.5, 0.25, 0.75], dtype=np.float32))
    seed, k = 99, 4
    u = philox4x32_10(np.arange(10), k, 0, 0, seed & 0xFFFFFFFF, seed >> 32)[0]
    want = [int(np.sum(u[0:3] < thr[0])), int(np.sum(u[3:8] < thr[1])), int(np.sum(u[8:10] < thr[2]))]
    assert bernoulli_ones(counts, thr, k, seed).tolist() == want
