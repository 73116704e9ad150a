"""Energy statistics, VMC gradient and Adam (paper Eqs. total_energy, grad, total_energy_sum;
Section 5.1 training set-up).

Readings: the reported energy is <H> (not the 1/2 <H> objective of Eq. total_energy, whose
gradient differs only by the same factor); the baseline b of Eq. grad is the real scalar
Re(E_bar) with E_bar the count-weighted mean of the local energies.  Then
    grad <H> = 2 Re sum_i (w_i/W) (E_i - b) conj(d log f(x_i))
             = sum_i g_abs_i d log|f(x_i)| + g_phase_i d phi(x_i),
    g_abs_i = 2 (w_i/W) Re(E_i - E_bar),   g_phase_i = 2 (w_i/W) Im(E_i).
"""
import numpy as np
import torch


def energy_stats(eloc, counts):
    """(mean complex, variance) with weights = counts, in FP64 (Eq. total_energy_sum)."""
    e = np.asarray(eloc, dtype=np.complex128)
    w = np.asarray(counts, dtype=np.float64)
    W = w.sum()
    mean = np.sum(w * e) / W
    var = np.sum(w * np.abs(e - mean) ** 2) / W
    return mean, float(var)


def surrogate_weights(eloc, counts):
    """Upstream gradients (g_abs, g_phase) of the surrogate sum_i g_abs log|f| + g_phase phi."""
    e = np.asarray(eloc, dtype=np.complex128)
    w = np.asarray(counts, dtype=np.float64)
    W = w.sum()
    mean = np.sum(w * e) / W
    return 2.0 * w / W * (e.real - mean.real), 2.0 * w / W * e.imag


def logpsi_vjp(model, bits, g_abs, g_phase) -> dict:
    """sum_i g_abs_i d log|f(x_i)|/d theta + g_phase_i d phi(x_i)/d theta, by FP64 autograd.
    The model must have been built with requires_grad=True."""
    for t in model.p.values():
        t.grad = None
    la, ph = model.log_psi_t(model.positions(bits))
    obj = (torch.tensor(np.asarray(g_abs, np.float64)) * la).sum() + \
          (torch.tensor(np.asarray(g_phase, np.float64)) * ph).sum()
    obj.backward()
    return {k: (v.grad.numpy().copy() if v.grad is not None else np.zeros(v.shape))
            for k, v in model.p.items()}


def vmc_gradient(model, bits, counts, eloc) -> dict:
    g_abs, g_phase = surrogate_weights(eloc, counts)
    return logpsi_vjp(model, bits, g_abs, g_phase)


def adam_step(params: dict, grads: dict, m: dict, v: dict, t: int, lr=1e-3, b1=0.9, b2=0.99,
              eps=1e-8):
    """One Adam update (Kingma & Ba), paper Section 5.1: lr 1e-3, beta = (0.9, 0.99).
    t is the 1-based step number; eps (unstated in the paper) is 1e-8.  Returns new dicts."""
    new_p, new_m, new_v = {}, {}, {}
    for k in params:
        g = np.asarray(grads[k], dtype=np.float64)
        mk = b1 * m[k] + (1 - b1) * g
        vk = b2 * v[k] + (1 - b2) * g * g
        mhat = mk / (1 - b1 ** t)
        vhat = vk / (1 - b2 ** t)
        new_p[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
        new_m[k], new_v[k] = mk, vk
    return new_p, new_m, new_v
