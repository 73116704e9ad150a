"""Autoregressive wavefunction models in FP64 (torch CPU ops), paper Section 4.

log f(x) = i phi(x) + 1/2 sum_t log pihat_t(x_t | x_<t)   (Section 4, Architecture)

Positions t = 0..n-1 follow the sampling order: position t holds qubit order[t] (reverse order,
Section 4 Sampling, is order[t] = n-1-t).  Conventions (readings of the paper):
  * network inputs are spins +-1 (bit 1 -> +1, bit 0 -> -1);
  * MADE (Germain et al.): input degree t+1; hidden unit k has degree (k mod (n-1)) + 1;
    hidden<-input iff deg_h >= deg_in; hidden<-hidden iff deg >= deg; output t <- hidden iff
    deg_h < t+1, so output 0 is bias only.  log pi uses log-sigmoid;
  * phase sub-model: a dense two-layer MLP on the first n-2 positions with 4 outputs, and
    phi(x) = out[2 x_{order[n-2]} + x_{order[n-1]}];
  * transformer (not in the paper; used for the larger workloads): tokens [BOS, x_order[0..n-2]],
    token + learned position embeddings, pre-LayerNorm blocks (causal multi-head attention, GELU
    MLP of width 4d), final LayerNorm, a per-position logit head and a 4-way phase head on the
    hidden state of position n-2 (which has seen exactly the first n-2 bits);
  * product model: pi(x_order[t] = 1) = p[t] with p an fp32 parameter vector, phi = 0;
  * Hamming-weight constraint, Eq. modifier (garbled in print; read as): for position t with
    qubit q of spin s = q & 1, let c = ones of spin s already sampled and r = spin-s qubits
    left after t.  Force 1 if c + r < n_s, force 0 if c >= n_s, else use the network.
    Forced positions contribute log 1 = 0; a mismatch (x outside the sector) gives -inf.

quant="bf16" emulates the tensor-core path: the four block GEMMs take bf16-rounded (RNE)
weights and bf16-rounded input activations (LayerNorm outputs, attention output, GELU output);
quant="bf16x2" keeps the bf16 weights but represents each GEMM input activation as the sum of
two bf16 numbers hi = bf16(a), lo = bf16(a - hi) (the compensated tensor-core form).  Rounding
is treated as identity by autograd (straight-through).
"""
import math

import numpy as np
import torch

LN_EPS = 1e-5


def bf16_round(t: torch.Tensor) -> torch.Tensor:
    """Round an fp64 tensor to the nearest bfloat16 value, ties to even (8 significant bits)."""
    m, e = torch.frexp(t)
    return torch.ldexp(torch.round(m * 256.0) / 256.0, e)


def _q(t, on):
    """Straight-through bf16 rounding of a GEMM operand (on: False, True or "x2")."""
    if not on:
        return t
    d = t.detach()
    hi = bf16_round(d)
    r = hi + bf16_round(d - hi) if on == "x2" else hi
    return t + (r - d)


def made_masks(n: int, hidden: int, layers: int):
    deg_in = np.arange(1, n + 1)
    deg_h = (np.arange(hidden) % (n - 1)) + 1
    m_in = (deg_h[:, None] >= deg_in[None, :]).astype(np.float64)
    m_hh = (deg_h[:, None] >= deg_h[None, :]).astype(np.float64)
    m_out = (deg_in[:, None] > deg_h[None, :]).astype(np.float64)
    return m_in, [m_hh] * (layers - 1), m_out


class Model:
    def __init__(self, arch, params, n, n_up, n_dn, order, hidden=0, layers=0, heads=0,
                 quant=None, requires_grad=False):
        self.arch, self.n, self.n_up, self.n_dn = arch, int(n), int(n_up), int(n_dn)
        self.order = np.asarray(order, dtype=np.int64)
        self.hidden, self.layers, self.heads = int(hidden), int(layers), int(heads)
        self.quant = {None: False, "bf16": True, "bf16x2": "x2"}[quant]
        self.p = {k: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=requires_grad)
                  for k, v in params.items()}
        if arch == "made":
            m_in, m_hh, m_out = made_masks(self.n, self.hidden, self.layers)
            self.m_in = torch.tensor(m_in)
            self.m_hh = [torch.tensor(m) for m in m_hh]
            self.m_out = torch.tensor(m_out)
        spec = self.order & 1
        self.spec = torch.tensor(spec)
        # spin-s positions strictly after t, for the species of t
        after = np.array([np.sum(spec[t + 1:] == spec[t]) for t in range(self.n)])
        self.after = torch.tensor(after, dtype=torch.float64)
        self.need = torch.tensor(np.where(spec == 0, self.n_up, self.n_dn), dtype=torch.float64)

    # ----------------------------------------------------------------- inputs
    def positions(self, bits) -> torch.Tensor:
        """[B, n] float64 of x_{order[t]} in {0, 1}; bits uint64 [B] or, for registers of more
        than 64 qubits, [B, W] words (qubit j in bit j % 64 of word j // 64)."""
        b = np.asarray(bits, dtype=np.uint64)
        q = self.order.astype(np.int64)
        if b.ndim == 2:
            X = (b[:, q // 64] >> (q % 64).astype(np.uint64)[None, :]) & np.uint64(1)
        else:
            X = (b[:, None] >> q.astype(np.uint64)[None, :]) & np.uint64(1)
        return torch.tensor(X.astype(np.float64))

    # ----------------------------------------------------------------- networks
    def _made(self, X):
        P = self.p
        u = 2.0 * X - 1.0
        h = torch.relu(u @ (P["made.W0"] * self.m_in).T + P["made.b0"])
        for l in range(1, self.layers):
            h = torch.relu(h @ (P[f"made.W{l}"] * self.m_hh[l - 1]).T + P[f"made.b{l}"])
        logits = h @ (P["made.Wout"] * self.m_out).T + P["made.bout"]
        hp = torch.relu(u[:, : self.n - 2] @ P["phase.W0"].T + P["phase.b0"])
        phase_out = hp @ P["phase.W1"].T + P["phase.b1"]
        return logits, phase_out

    @staticmethod
    def _ln(x, g, b):
        mu = x.mean(-1, keepdim=True)
        var = ((x - mu) ** 2).mean(-1, keepdim=True)
        return (x - mu) / torch.sqrt(var + LN_EPS) * g + b

    @staticmethod
    def _gelu(x):
        return 0.5 * x * (1.0 + torch.tanh(math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3)))

    def _transformer(self, X):
        P, n, d, H = self.p, self.n, self.hidden, self.heads
        dh = d // H
        qz = self.quant                 # activations
        qw = bool(self.quant)           # weights: bf16 in both quantised forms
        B = X.shape[0]
        tok = torch.cat([torch.full((B, 1), 2, dtype=torch.long), X[:, : n - 1].long()], dim=1)
        h = P["tok_emb"][tok] + P["pos_emb"][None, :, :]
        causal = torch.tril(torch.ones(n, n, dtype=torch.bool))
        for l in range(self.layers):
            pre = f"blk{l}."
            a = _q(self._ln(h, P[pre + "ln1_g"], P[pre + "ln1_b"]), qz)
            qkv = a @ _q(P[pre + "wqkv"], qw).T + P[pre + "bqkv"]
            q, k, v = qkv.split(d, dim=-1)
            q = q.reshape(B, n, H, dh).transpose(1, 2)
            k = k.reshape(B, n, H, dh).transpose(1, 2)
            v = v.reshape(B, n, H, dh).transpose(1, 2)
            s = (q @ k.transpose(-1, -2)) / math.sqrt(dh)
            s = s.masked_fill(~causal, float("-inf"))
            att = torch.softmax(s, dim=-1)
            o = (att @ v).transpose(1, 2).reshape(B, n, d)
            h = h + _q(o, qz) @ _q(P[pre + "wo"], qw).T + P[pre + "bo"]
            a2 = _q(self._ln(h, P[pre + "ln2_g"], P[pre + "ln2_b"]), qz)
            m = self._gelu(a2 @ _q(P[pre + "w1"], qw).T + P[pre + "b1"])
            h = h + _q(m, qz) @ _q(P[pre + "w2"], qw).T + P[pre + "b2"]
        hf = self._ln(h, P["lnf_g"], P["lnf_b"])
        logits = hf @ P["head_w"] + P["head_b"]
        phase_out = hf[:, n - 2, :] @ P["phase_w"].T + P["phase_b"]
        return logits, phase_out

    def cond_logp(self, X):
        """(log pi(bit=1), log pi(bit=0), phase outputs) per position, before the constraint."""
        if self.arch == "product":
            p = self.p["p"][None, :].expand(X.shape[0], -1)
            return torch.log(p), torch.log1p(-p), torch.zeros(X.shape[0], 4, dtype=torch.float64)
        logits, phase_out = self._made(X) if self.arch == "made" else self._transformer(X)
        return torch.nn.functional.logsigmoid(logits), torch.nn.functional.logsigmoid(-logits), phase_out

    def cond_p1(self, X):
        """Unconstrained pi(x_t = 1 | x_<t) for every position t (network output only)."""
        if self.arch == "product":
            return self.p["p"][None, :].expand(X.shape[0], -1)
        logits, _ = self._made(X) if self.arch == "made" else self._transformer(X)
        return torch.sigmoid(logits)

    # ----------------------------------------------------------------- constraint
    def forced(self, X):
        """(force1, force0) boolean [B, n] from the prefix of each position (Eq. modifier)."""
        ones_before = torch.zeros_like(X)
        for s in (0, 1):
            sel = (self.spec == s).to(X.dtype)
            cum = torch.cumsum(X * sel, dim=1) - X * sel
            ones_before = ones_before + cum * sel
        force1 = ones_before + self.after < self.need
        force0 = ones_before >= self.need
        return force1, force0

    # ----------------------------------------------------------------- log psi
    def log_psi_t(self, X):
        """(log|psi|, phi) as torch tensors (differentiable in the parameters)."""
        lp1, lp0, phase_out = self.cond_logp(X)
        f1, f0 = self.forced(X)
        free = ~(f1 | f0)
        lp = torch.where(X > 0.5, lp1, lp0)
        lp = torch.where(free, lp, torch.zeros_like(lp))
        bad = (f1 & (X < 0.5)) | (f0 & (X > 0.5))
        log_abs = 0.5 * lp.sum(dim=1)
        log_abs = torch.where(bad.any(dim=1), torch.full_like(log_abs, float("-inf")), log_abs)
        sel = (2 * X[:, self.n - 2] + X[:, self.n - 1]).long()
        phase = phase_out.gather(1, sel[:, None])[:, 0]
        return log_abs, phase

    def log_psi(self, bits, chunk: int = 8192):
        """(log|psi|, phi) as fp64 numpy arrays; out-of-sector inputs give log|psi| = -inf."""
        bits = np.asarray(bits, dtype=np.uint64)
        la = np.empty(len(bits)); ph = np.empty(len(bits))
        with torch.no_grad():
            for lo in range(0, len(bits), chunk):
                a, p = self.log_psi_t(self.positions(bits[lo: lo + chunk]))
                la[lo: lo + chunk] = a.numpy(); ph[lo: lo + chunk] = p.numpy()
        return la, ph

    def sampling_p(self, prefix_bits, k: int) -> np.ndarray:
        """pihat(x_{order[k]} = 1 | prefix) in FP64 for parents whose positions < k are set."""
        return self.sampling_p_positions(self.positions(prefix_bits), k)

    def sampling_p_positions(self, X, k: int) -> np.ndarray:
        """sampling_p from the parents' positions matrix X [B, n] (x_{order[t]} in {0, 1})."""
        X = X.clone()
        X[:, k:] = 0.0
        with torch.no_grad():
            p = self.cond_p1(X)[:, k]
            f1, f0 = self.forced(X)
        p = torch.where(f1[:, k], torch.ones_like(p), p)
        p = torch.where(f0[:, k], torch.zeros_like(p), p)
        return p.numpy()


def in_sector(bits, n: int, n_up: int, n_dn: int) -> np.ndarray:
    """Hamming-weight constraint, Eq. hamming_weight_constraint (up = even bits, down = odd)."""
    b = np.asarray(bits, dtype=np.uint64)
    a_mask = np.uint64(sum(1 << j for j in range(0, n, 2)))
    b_mask = np.uint64(sum(1 << j for j in range(1, n, 2)))
    return (np.bitwise_count(b & a_mask) == n_up) & (np.bitwise_count(b & b_mask) == n_dn)
