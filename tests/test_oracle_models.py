"""Pins for the oracle's wavefunction models (paper Section 4)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle.lanczos import sector_states
from oracle.models import bf16_round, in_sector
from tests.common import oracle_model

SMALL_TF = dict(arch="transformer", n=8, n_up=2, n_dn=1, hidden=16, layers=2, heads=2, seed=5)
SMALL_MADE = dict(arch="made", n=8, n_up=2, n_dn=2, hidden=12, layers=2, seed=6)
SMALL_PROD = dict(arch="product", n=8, n_up=1, n_dn=3, hidden=0, layers=0, seed=9)


def _all_states(n):
    return np.arange(1 << n, dtype=np.uint64)


@pytest.mark.parametrize("dims", [SMALL_TF, SMALL_MADE, SMALL_PROD, 1, 2])
@pytest.mark.parametrize("beta", [0.0, 2.0])
def test_normalised_over_sector_and_zero_outside(dims, beta):
    # Section 4: the autoregressive product normalises; pihat "still normalize to one".
    cfg = synth.get_config(dims) if isinstance(dims, int) else dims
    model, _ = oracle_model(cfg, beta=beta)
    n = model.n
    x = _all_states(n)
    la, _ = model.log_psi(x)
    ok = in_sector(x, n, model.n_up, model.n_dn)
    assert np.all(np.isneginf(la[~ok]))
    assert abs(np.sum(np.exp(2 * la[ok])) - 1.0) < 1e-13


def test_normalised_config3_sector():
    cfg = synth.get_config(3)
    model, _ = oracle_model(cfg, beta=0.5)
    st = sector_states(cfg.n_orb, cfg.n_up, cfg.n_dn)
    la, _ = model.log_psi(st)
    assert abs(np.sum(np.exp(2 * la)) - 1.0) < 1e-12


@pytest.mark.parametrize("dims", [SMALL_TF, SMALL_MADE])
def test_autoregressive_dependence(dims):
    # conditional at position t must not depend on positions >= t
    model, _ = oracle_model(dims, beta=1.0)
    n = model.n
    rng = np.random.default_rng(0)
    X = torch.tensor(rng.integers(0, 2, size=(64, n)).astype(np.float64))
    base = model.cond_p1(X)
    for t in range(n):
        Y = X.clone()
        Y[:, t:] = 1.0 - Y[:, t:]
        p = model.cond_p1(Y)
        assert torch.allclose(p[:, : t + 1], base[:, : t + 1], atol=1e-14, rtol=0)


def test_transformer_matches_torch_library_modules():
    model, params = oracle_model(SMALL_TF, beta=1.0)
    P = {k: torch.tensor(v, dtype=torch.float64) for k, v in params.items()}
    n, d, H = model.n, model.hidden, model.heads
    rng = np.random.default_rng(1)
    X = torch.tensor(rng.integers(0, 2, size=(16, n)).astype(np.float64))
    logits, phase_out = model._transformer(X)

    F = torch.nn.functional
    tok = torch.cat([torch.full((16, 1), 2), X[:, : n - 1].long()], 1)
    h = F.embedding(tok, P["tok_emb"]) + P["pos_emb"]
    for l in range(model.layers):
        g = lambda s: P[f"blk{l}.{s}"]
        a = F.layer_norm(h, (d,), g("ln1_g"), g("ln1_b"), eps=1e-5)
        qkv = F.linear(a, g("wqkv"), g("bqkv"))
        q, k, v = (t.reshape(16, n, H, d // H).transpose(1, 2) for t in qkv.split(d, -1))
        o = F.scaled_dot_product_attention(q, k, v, is_causal=True).transpose(1, 2).reshape(16, n, d)
        h = h + F.linear(o, g("wo"), g("bo"))
        a2 = F.layer_norm(h, (d,), g("ln2_g"), g("ln2_b"), eps=1e-5)
        h = h + F.linear(F.gelu(F.linear(a2, g("w1"), g("b1")), approximate="tanh"), g("w2"), g("b2"))
    hf = F.layer_norm(h, (d,), P["lnf_g"], P["lnf_b"], eps=1e-5)
    want_logits = hf @ P["head_w"] + P["head_b"]
    want_phase = F.linear(hf[:, n - 2], P["phase_w"], P["phase_b"])
    torch.testing.assert_close(logits, want_logits, atol=1e-12, rtol=0)
    torch.testing.assert_close(phase_out, want_phase, atol=1e-12, rtol=0)


def test_bf16_round_matches_torch_rne_conversion():
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.standard_normal(20000) * 10 ** rng.uniform(-6, 6, 20000),
                        [0.0, 1.0, -1.0, 1.00390625, 1.005859375]]).astype(np.float32)
    want = torch.tensor(v).to(torch.bfloat16).to(torch.float64)
    got = bf16_round(torch.tensor(v.astype(np.float64)))
    assert torch.equal(got, want)


def test_phase_selected_by_last_two_positions():
    model, _ = oracle_model(SMALL_MADE, beta=0.0)
    X = torch.tensor(np.random.default_rng(4).integers(0, 2, size=(32, model.n)).astype(np.float64))
    _, _, po = model.cond_logp(X)
    _, ph = model.log_psi_t(X)
    sel = (2 * X[:, -2] + X[:, -1]).long()
    assert torch.equal(ph, po[torch.arange(32), sel])


def test_sampling_conditionals_respect_constraint():
    # sequentially drawing the most likely allowed bit must always end inside the sector
    for dims in (SMALL_TF, SMALL_MADE, SMALL_PROD):
        model, _ = oracle_model(dims, beta=0.0)
        rng = np.random.default_rng(5)
        for trial in range(20):
            bits = np.zeros(1, dtype=np.uint64)
            for k in range(model.n):
                p = model.sampling_p(bits, k)[0]
                b = rng.random() < p
                if b:
                    bits |= np.uint64(1) << np.uint64(model.order[k])
            assert in_sector(bits, model.n, model.n_up, model.n_dn)[0]


def test_bf16x2_split_is_a_pair_of_bf16_within_2_to_minus_16():
    # the compensated form represents a as hi + lo with hi = bf16(a), lo = bf16(a - hi): both
    # bf16 numbers, and |a - (hi + lo)| <= 2^-16 |a| (8 + 8 significant bits, two roundings)
    from oracle.models import _q
    rng = np.random.default_rng(11)
    a = torch.tensor(rng.standard_normal(50000) * 10 ** rng.uniform(-3, 3, 50000))
    r = _q(a, "x2")
    hi = bf16_round(a)
    lo = r - hi
    assert torch.equal(bf16_round(hi), hi) and torch.equal(bf16_round(lo), lo)
    assert torch.all((r - a).abs() <= 2.0 ** -16 * a.abs())
    assert torch.all((bf16_round(a) - a).abs() <= 2.0 ** -8 * a.abs())


def _made_by_degree_rule(P, n, hidden, layers, X):
    """The MADE modulus network and the phase MLP written unit by unit from the connectivity
    rule (Germain et al.; paper Section 4, Architecture): input position t has degree t+1,
    hidden unit k degree (k mod (n-1)) + 1; a hidden unit sees the inputs and previous-layer
    units of degree <= its own, output t sees the last hidden units of degree < t+1 (so output
    0 is its bias alone); ReLU after every hidden layer.  The phase MLP sees the +-1 spins of
    the first n-2 positions through one dense ReLU layer and has 4 outputs."""
    deg_in = [t + 1 for t in range(n)]
    deg_h = [(k % (n - 1)) + 1 for k in range(hidden)]
    B = len(X)
    logits = np.zeros((B, n))
    phase = np.zeros((B, 4))
    pre_min = np.inf
    for b in range(B):
        u = [2.0 * X[b][t] - 1.0 for t in range(n)]
        h = []
        for k in range(hidden):
            s = P["made.b0"][k]
            for t in range(n):
                if deg_h[k] >= deg_in[t]:
                    s += P["made.W0"][k][t] * u[t]
            pre_min = min(pre_min, s)
            h.append(s if s > 0.0 else 0.0)
        for l in range(1, layers):
            nxt = []
            for k in range(hidden):
                s = P[f"made.b{l}"][k]
                for j in range(hidden):
                    if deg_h[k] >= deg_h[j]:
                        s += P[f"made.W{l}"][k][j] * h[j]
                pre_min = min(pre_min, s)
                nxt.append(s if s > 0.0 else 0.0)
            h = nxt
        for t in range(n):
            s = P["made.bout"][t]
            for k in range(hidden):
                if deg_h[k] < deg_in[t]:
                    s += P["made.Wout"][t][k] * h[k]
            logits[b][t] = s
        hp = []
        for k in range(hidden):
            s = P["phase.b0"][k]
            for i in range(n - 2):
                s += P["phase.W0"][k][i] * u[i]
            hp.append(s if s > 0.0 else 0.0)
        for j in range(4):
            s = P["phase.b1"][j]
            for k in range(hidden):
                s += P["phase.W1"][j][k] * hp[k]
            phase[b][j] = s
    return logits, phase, pre_min


def _log_psi_by_hand(logits, phase, X, order, n_up, n_dn):
    """log|psi| = 1/2 sum over unforced positions of log pi, and the phase output picked by the
    last two positions, with the Hamming-weight constraint applied position by position (a
    species' bit is forced to 1 when its remaining positions are needed to reach its count, to 0
    when the count is reached)."""
    B, n = X.shape
    la = np.zeros(B)
    ph = np.zeros(B)
    for b in range(B):
        ones = [0, 0]
        need = [n_up, n_dn]
        total = 0.0
        bad = False
        for t in range(n):
            s = int(order[t]) & 1
            left = sum(1 for u in range(t + 1, n) if (int(order[u]) & 1) == s)
            x = int(X[b][t])
            if ones[s] + left < need[s]:
                bad |= x == 0
            elif ones[s] >= need[s]:
                bad |= x == 1
            else:
                z = logits[b][t] if x == 1 else -logits[b][t]
                total += -math.log1p(math.exp(-z)) if z > 0 else z - math.log1p(math.exp(z))
            ones[s] += x
        la[b] = -math.inf if bad else 0.5 * total
        ph[b] = phase[b][2 * int(X[b][n - 2]) + int(X[b][n - 1])]
    return la, ph


@pytest.mark.parametrize("dims", [SMALL_MADE, dict(arch="made", n=6, n_up=1, n_dn=2, hidden=9, layers=3, seed=8), 1, 2])
def test_made_matches_unit_by_unit_degree_rule(dims):
    # Pins the MADE network values themselves (normalisation holds for any logits): a dropped
    # ReLU, a wrong mask degree, a wrong bias or a wrong phase-MLP input slice changes these.
    cfg = synth.get_config(dims) if isinstance(dims, int) else dims
    model, params = oracle_model(cfg, beta=1.0)
    n, hidden, layers = model.n, model.hidden, model.layers
    P = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
    st = sector_states(n // 2, model.n_up, model.n_dn)
    rng = np.random.default_rng(12)
    free = rng.integers(0, 2, size=(24, n)).astype(np.float64)     # also out-of-sector inputs
    X = np.concatenate([model.positions(st[:40]).numpy(), free])
    want_logits, want_phase, pre_min = _made_by_degree_rule(P, n, hidden, layers, X)
    assert pre_min < 0.0                  # the ReLUs are active on these inputs
    logits, phase_out = model._made(torch.tensor(X))
    np.testing.assert_allclose(logits.numpy(), want_logits, rtol=0, atol=1e-12)
    np.testing.assert_allclose(phase_out.numpy(), want_phase, rtol=0, atol=1e-12)
    la_w, ph_w = _log_psi_by_hand(want_logits, want_phase, X, model.order, model.n_up, model.n_dn)
    la, ph = model.log_psi_t(torch.tensor(X))
    fin = np.isfinite(la_w)
    assert np.array_equal(np.isfinite(la.numpy()), fin)
    np.testing.assert_allclose(la.numpy()[fin], la_w[fin], rtol=0, atol=1e-12)
    np.testing.assert_allclose(ph.numpy(), ph_w, rtol=0, atol=1e-12)


def test_made_degree_rule_catches_planted_mistakes():
    # Each mistake planted in a copy of the oracle's MADE on the CPU must break the agreement
    # with the unit-by-unit restatement above.
    import oracle.models as OM
    model, params = oracle_model(SMALL_MADE, beta=1.0)
    P = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
    X = np.random.default_rng(13).integers(0, 2, size=(16, model.n)).astype(np.float64)
    want_logits, want_phase, _ = _made_by_degree_rule(P, model.n, model.hidden, model.layers, X)

    class NoRelu(OM.Model):
        def _made(self, X):
            saved = torch.relu
            torch.relu = lambda t: t
            try:
                return super()._made(X)
            finally:
                torch.relu = saved

    class PhaseSlice(OM.Model):
        def _made(self, X):
            logits, _ = super()._made(X)
            u = 2.0 * X - 1.0
            hp = torch.relu(u[:, 2:] @ self.p["phase.W0"].T + self.p["phase.b0"])
            return logits, hp @ self.p["phase.W1"].T + self.p["phase.b1"]

    class OutMask(OM.Model):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            n = self.n
            deg_in = np.arange(1, n + 1)
            deg_h = (np.arange(self.hidden) % (n - 1)) + 1
            self.m_out = torch.tensor((deg_in[:, None] >= deg_h[None, :]).astype(np.float64))

    for cls in (NoRelu, PhaseSlice, OutMask):
        bad = cls("made", params, model.n, model.n_up, model.n_dn, model.order, model.hidden, model.layers)
        lg, po = bad._made(torch.tensor(X))
        assert not (np.allclose(lg.numpy(), want_logits, atol=1e-9) and
                    np.allclose(po.numpy(), want_phase, atol=1e-9)), cls.__name__
