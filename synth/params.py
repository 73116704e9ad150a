"""Seeded model parameters (fp32 masters) as named arrays.

Weights ~ N(0, 1/fan_in).  Biases and LayerNorm affines are small seeded perturbations
(N(0, 0.1^2) around 0 or 1) so that a forward that ignored one of them would change its output.
The output-head bias of sampling position t is +beta when qubit order[t] is occupied in the
Hartree-Fock reference (the lowest n_up spin-up and n_dn spin-down orbitals) and -beta
otherwise, plus the same small perturbation: beta = 0 gives a near-uniform model, beta = 2 a
concentrated ("trained-like") one.
"""
import numpy as np

from .rng import SplitMix64


def default_order(n: int) -> np.ndarray:
    """Reverse sampling order: qubit n-1 is sampled first (paper, Section 4, Sampling)."""
    return np.arange(n - 1, -1, -1, dtype=np.int64)


def hf_occupied(n_orb: int, n_up: int, n_dn: int) -> int:
    """Hartree-Fock bitstring: bits 2p (spin up, p < n_up) and 2p+1 (spin down, p < n_dn)."""
    bits = 0
    for p in range(n_up):
        bits |= 1 << (2 * p)
    for p in range(n_dn):
        bits |= 1 << (2 * p + 1)
    return bits


def param_shapes(arch: str, n: int, hidden: int, layers: int, heads: int = 0):
    """Ordered (name, shape) list; the order is the packing order of the flat parameter vector."""
    h = hidden
    if arch == "product":
        return [("p", (n,))]
    if arch == "made":
        out = [("made.W0", (h, n)), ("made.b0", (h,))]
        for l in range(1, layers):
            out += [(f"made.W{l}", (h, h)), (f"made.b{l}", (h,))]
        out += [("made.Wout", (n, h)), ("made.bout", (n,)),
                ("phase.W0", (h, n - 2)), ("phase.b0", (h,)),
                ("phase.W1", (4, h)), ("phase.b1", (4,))]
        return out
    if arch == "transformer":
        d = hidden
        out = [("tok_emb", (3, d)), ("pos_emb", (n, d))]
        for l in range(layers):
            out += [(f"blk{l}.ln1_g", (d,)), (f"blk{l}.ln1_b", (d,)),
                    (f"blk{l}.wqkv", (3 * d, d)), (f"blk{l}.bqkv", (3 * d,)),
                    (f"blk{l}.wo", (d, d)), (f"blk{l}.bo", (d,)),
                    (f"blk{l}.ln2_g", (d,)), (f"blk{l}.ln2_b", (d,)),
                    (f"blk{l}.w1", (4 * d, d)), (f"blk{l}.b1", (4 * d,)),
                    (f"blk{l}.w2", (d, 4 * d)), (f"blk{l}.b2", (d,))]
        out += [("lnf_g", (d,)), ("lnf_b", (d,)), ("head_w", (d,)), ("head_b", (n,)),
                ("phase_w", (4, d)), ("phase_b", (4,))]
        return out
    raise ValueError(f"unknown arch {arch}")


def init_params(arch: str, n: int, n_up: int, n_dn: int, hidden: int, layers: int, heads: int,
                seed: int, beta: float = 2.0, order=None) -> dict:
    """Named fp32 parameter arrays for one model."""
    rng = SplitMix64(seed)
    order = default_order(n) if order is None else np.asarray(order, dtype=np.int64)
    hf = hf_occupied(n // 2, n_up, n_dn)
    head_sign = np.array([1.0 if (hf >> int(q)) & 1 else -1.0 for q in order])
    out = {}
    for name, shape in param_shapes(arch, n, hidden, layers, heads):
        size = int(np.prod(shape))
        leaf = name.split(".")[-1]
        if name == "p":
            logit = beta * head_sign + 0.5 * rng.normal(size)
            v = 1.0 / (1.0 + np.exp(-logit))
        elif name in ("made.bout", "head_b"):
            v = beta * head_sign + 0.1 * rng.normal(size)
        elif leaf.endswith("_g"):
            v = 1.0 + 0.1 * rng.normal(size)
        elif leaf in ("tok_emb", "pos_emb"):
            v = rng.normal(size)
        elif len(shape) == 1:
            v = 0.1 * rng.normal(size)
        else:
            v = rng.normal(size) / np.sqrt(shape[-1])
        out[name] = np.asarray(v, dtype=np.float32).reshape(shape)
    return out
