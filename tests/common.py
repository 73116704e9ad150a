"""Shared test helpers: workload construction for the oracle and the library."""
import numpy as np

import synth


def oracle_model(cfg_or_dims, beta=2.0, quant=None, requires_grad=False, seed=None, order=None):
    """An oracle Model for a WorkloadConfig, or for a dims dict with keys
    arch, n, n_up, n_dn, hidden, layers, heads."""
    from oracle.models import Model
    d = dims_of(cfg_or_dims)
    order = synth.default_order(d["n"]) if order is None else np.asarray(order)
    params = synth.init_params(d["arch"], d["n"], d["n_up"], d["n_dn"], d["hidden"], d["layers"],
                               d["heads"], d["seed"] if seed is None else seed, beta=beta,
                               order=order)
    return Model(d["arch"], params, d["n"], d["n_up"], d["n_dn"], order, d["hidden"], d["layers"],
                 d["heads"], quant=quant, requires_grad=requires_grad), params


def dims_of(c):
    if isinstance(c, dict):
        out = dict(c)
        out.setdefault("seed", 7)
        out.setdefault("heads", 0)
        return out
    return dict(arch=c.arch, n=c.n_qubits, n_up=c.n_up, n_dn=c.n_dn, hidden=c.hidden,
                layers=c.layers, heads=c.heads, seed=c.seed_params)


def rel_norm(a, b, w=None):
    """sqrt(sum w |a-b|^2) / sqrt(sum w |b|^2)."""
    a = np.asarray(a); b = np.asarray(b)
    w = np.ones(len(b)) if w is None else np.asarray(w, dtype=np.float64)
    return float(np.sqrt(np.sum(w * np.abs(a - b) ** 2)) / max(np.sqrt(np.sum(w * np.abs(b) ** 2)), 1e-300))
