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


def elem_metric(got, want, absum):
    """max_i |got_i - want_i| / (|want_i| + A_i 2^-24): the element-wise relative error of the
    local energies, with A_i (the sum of the magnitudes of sample i's terms) times the fp32 unit
    roundoff as the floor where the terms cancel."""
    got = np.asarray(got); want = np.asarray(want)
    return float(np.max(np.abs(got - want) / (np.abs(want) + np.asarray(absum) * 2.0 ** -24)))


# Local-energy gates (spec: relative error 1e-5 in the FP32 path, 1e-4 in the compensated
# BF16 path against the quantisation-aware oracle).  The norm over the batch takes the stated
# tolerance; the element-wise maximum takes ten times it.
TOL_NORM = {"fp32": 1e-5, "bf16": 1e-4}
TOL_ELEM = {"fp32": 1e-4, "bf16": 1e-3}


def check_eloc(got, want, absum, form="fp32", w=None, label=""):
    """Assert both local-energy gates; returns (rel_norm, elem_metric)."""
    rn = rel_norm(got, want, w)
    em = elem_metric(got, want, absum)
    print(f"{label} E_loc rel_norm {rn:.2e} elementwise {em:.2e} ({form})")
    assert rn <= TOL_NORM[form], (label, rn)
    assert em <= TOL_ELEM[form], (label, em)
    return rn, em
