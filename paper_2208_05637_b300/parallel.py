"""Data-parallel VMC gradient over L ranks (paper Section 5: the B*K summands of the local
energies are split over L GPUs with replicated models, and the gradients averaged).

Each rank samples with its own seed and keeps its own unique samples, computes their local
energies and two backward sums over them:

    first  = sum_i 2 w_i [Re E_i  d log|f(x_i)| + Im E_i  d phi(x_i)]
    second = sum_i   w_i           d log|f(x_i)|

together with S = [sum w Re E, sum w Im E, sum w |E|^2, W].  One all-reduce of [S, first, second]
gives the totals over all ranks, and the gradient of Eq. grad over the union of the samples,

    g = (first - 2 Re(E_bar) second) / W,   E_bar = (S0 + i S1) / W,

is the same on every rank (the baseline b = Re E_bar of Eq. grad is the global mean).  This
module holds the exchange: packing, the all-reduce and the final combination of the reduced
vectors; the per-rank pieces come from the library (nqs_energy_sums, nqs_logpsi_backward).
"""
import torch
import torch.distributed as dist


def combine(sums, first, second, group=None):
    """One all-reduce of [sums (4), first (P), second (P)] over `group` (any backend; tensors on
    that backend's device) and the gradient of the union of the ranks' samples.

    Returns (grad fp32 [P], stats fp64 [4] = Re E_bar, Im E_bar, Var, W) on first's device."""
    P = first.numel()
    buf = torch.cat([sums.reshape(-1).to(torch.float64), first.reshape(-1).to(torch.float64),
                     second.reshape(-1).to(torch.float64)])
    if group is not None or (dist.is_available() and dist.is_initialized()):
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    S = buf[:4]
    W = S[3]
    mean_re, mean_im = S[0] / W, S[1] / W
    var = S[2] / W - (mean_re * mean_re + mean_im * mean_im)
    grad = (buf[4:4 + P] - 2.0 * mean_re * buf[4 + P:]) / W
    return grad.to(torch.float32), torch.stack([mean_re, mean_im, var, W])


def world(group=None):
    """(rank, size) of `group` (1 process when torch.distributed is not initialised)."""
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)
