"""Helpers for the GPU parity tests: the same seeded workload for the library and the oracle."""
import numpy as np

import synth


def lib():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2208_05637_b300 as P
    return P


def dims(cfg_or_dims):
    from tests.common import dims_of
    return dims_of(cfg_or_dims)


def gpu_model(cfg_or_dims, beta=2.0, precision="fp32", compensated=True, order=None):
    """(library Model with bound params, named params) for a config or dims dict."""
    import torch  # noqa: F401
    P = lib()
    d = dims(cfg_or_dims)
    order = synth.default_order(d["n"]) if order is None else np.asarray(order)
    params = synth.init_params(d["arch"], d["n"], d["n_up"], d["n_dn"], d["hidden"], d["layers"],
                               d["heads"], d["seed"], beta=beta, order=order)
    m = P.Model(d["arch"], d["n"], d["n_up"], d["n_dn"], d["hidden"], d["layers"], d["heads"],
                precision=precision, compensated=compensated, order=order)
    m.bind(m.pack(params))
    return m, params


def to_dev_bits(bits):
    import torch
    return torch.tensor(np.asarray(bits, dtype=np.uint64).view(np.int64), device="cuda")


def from_dev_bits(t):
    return t.cpu().numpy().view(np.uint64)
