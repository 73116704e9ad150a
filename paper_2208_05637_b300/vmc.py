"""The VMC step on top of the C ABI: log psi as a torch.autograd.Function with a hand-written
backward, mini-batch gradient accumulation with forward recomputation, FP64 statistics and Adam
(paper Eqs. total_energy, grad; Section 5.1: Adam lr 1e-3, betas (0.9, 0.99); Section 5.2
gradient accumulation).

The gradient of the VMC surrogate sum_i g_abs_i log|f(x_i)| + g_phase_i phi(x_i) is exactly the
vector-Jacobian product with upstream gradients (g_abs, g_phase).  VMC.step hands those to the
backward entry point directly (the backward recomputes the forward itself); with
``autograd=True`` it goes through LogPsi and torch autograd instead, which also evaluates the
surrogate's forward.  Both give the same gradient.  With one mini-batch the backward's forward
recompute (which needs only the samples) runs on a second stream while the local energy is
computed (nqs_logpsi_backward_phase); the gradient is the same bit for bit.
"""
import torch

from . import (NQS_ERR_UNSUPPORTED, NQSError, OP_BACKWARD, OP_LOCAL_ENERGY, OP_SAMPLE, nqs_adam_step,
               nqs_energy_stats, nqs_energy_sums, nqs_local_energy, nqs_logpsi, nqs_logpsi_backward,
               nqs_logpsi_backward_phase, nqs_sample)
from . import parallel


class LogPsi(torch.autograd.Function):
    """(log|f(x)|, phi(x)) = LogPsi.apply(params, model, bits).

    `params` must be the flat fp32 tensor bound to `model`.  Nothing is saved but the bits: the
    backward recomputes the forward inside nqs_logpsi_backward (activation recomputation) and
    returns sum_i g_abs_i d log|f_i|/d theta + g_phase_i d phi_i/d theta."""

    @staticmethod
    def forward(ctx, params, model, bits):
        la, ph = nqs_logpsi(model, bits)
        ctx.model = model
        ctx.save_for_backward(bits)
        return la, ph

    @staticmethod
    def backward(ctx, g_la, g_ph):
        (bits,) = ctx.saved_tensors
        model = ctx.model
        B = bits.shape[0]
        g_la = torch.zeros(B, dtype=torch.float32, device=bits.device) if g_la is None else g_la.float().contiguous()
        g_ph = torch.zeros(B, dtype=torch.float32, device=bits.device) if g_ph is None else g_ph.float().contiguous()
        grad = torch.zeros_like(model.params)
        nqs_logpsi_backward(model, bits, g_la, g_ph, grad)
        return grad, None, None


class VMC:
    """One variational Monte Carlo step per call: sample -> local energies (mini-batched) ->
    FP64 statistics -> surrogate backward (mini-batched, recomputed) -> Adam."""

    def __init__(self, ham, model, params, n_samples, mini_batches=1, max_unique=None,
                 lr=1e-3, betas=(0.9, 0.99), eps=1e-8, autograd=False, group=None):
        self.ham, self.model = ham, model
        self.params = params.detach().requires_grad_(True)
        model.bind(self.params)
        self.n_samples = int(n_samples)
        self.max_unique = int(max_unique or n_samples)
        self.mini_batches = int(mini_batches)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.autograd = bool(autograd)
        self.m = torch.zeros_like(self.params, requires_grad=False)
        self.v = torch.zeros_like(self.params, requires_grad=False)
        self.t = 0
        self.ws_sample = model.workspace(OP_SAMPLE, self.n_samples)
        self._ws = {}
        self._side = None            # stream of the overlapped backward recompute
        self.overlap_backward = True
        # data parallel over the ranks of `group` (NCCL): own samples per rank, one all-reduce of
        # the gradient pieces per step (paper Section 5); None or one rank: a single replica
        self.group = group
        self.rank, self.world = parallel.world(group) if group is not None else (0, 1)

    def reset(self, params):
        """Restore the parameters and clear the optimiser state (device copies, no sync)."""
        with torch.no_grad():
            self.params.data.copy_(params)
            self.m.zero_()
            self.v.zero_()
        self.t = 0

    def _workspace(self, op, batch):
        key = (op, batch)
        if key not in self._ws:
            self._ws[key] = self.model.workspace(op, batch, self.ham if op == OP_LOCAL_ENERGY else None)
        return self._ws[key]

    def _slices(self, U):
        per = max(1, -(-U // self.mini_batches))
        return [slice(lo, min(U, lo + per)) for lo in range(0, U, per)]

    def _recompute_ahead(self, bits, ws):
        """Phase 1 of the backward on the side stream (True), or False where it does not apply."""
        if self.autograd or not self.overlap_backward or self.mini_batches != 1:
            return False
        main = torch.cuda.current_stream()
        if self._side is None:
            self._side = torch.cuda.Stream()
        self._side.wait_stream(main)
        try:
            nqs_logpsi_backward_phase(self.model, 1, bits, ws=ws, stream=self._side)
        except NQSError as e:
            if e.status != NQS_ERR_UNSUPPORTED:
                raise
            return False
        return True

    def step(self, seed):
        # ranks draw from disjoint seed streams (each keeps its own unique samples)
        seed = seed + 0x9E3779B97F4A7C15 * self.rank if self.world > 1 else seed
        bits, counts, _ = nqs_sample(self.model, self.n_samples, self.max_unique, seed,
                                     ws=self.ws_sample)
        out = self.gradient(bits, counts)
        self.t += 1
        with torch.no_grad():
            nqs_adam_step(self.params, self.params.grad, self.m, self.v, self.t, self.lr,
                          self.betas[0], self.betas[1], self.eps)
        return out

    def gradient(self, bits, counts):
        """Local energies (mini-batched), FP64 statistics and the VMC gradient (Eq. grad) of
        the given unique samples and counts, accumulated into params.grad over the mini-batches
        with the forward recomputed in each; no parameter update."""
        U = bits.shape[0]
        eloc = torch.empty((U, 2), dtype=torch.float32, device="cuda")
        per = max(1, -(-U // self.mini_batches))
        ahead = self._recompute_ahead(bits, self._workspace(OP_BACKWARD, per))
        for sl in self._slices(U):
            nqs_local_energy(self.ham, self.model, bits[sl], ws=self._workspace(OP_LOCAL_ENERGY, per),
                             out=eloc[sl])
        if self.world > 1:
            return self._gradient_parallel(bits, counts, eloc, per, ahead)
        stats, g_abs, g_phase = nqs_energy_stats(eloc, counts)
        if self.params.grad is None:
            self.params.grad = torch.zeros_like(self.params)
        else:
            self.params.grad.zero_()
        if ahead:
            torch.cuda.current_stream().wait_stream(self._side)
            nqs_logpsi_backward_phase(self.model, 2, bits, g_abs, g_phase, self.params.grad,
                                      ws=self._workspace(OP_BACKWARD, per))
        for sl in ([] if ahead else self._slices(U)):
            if self.autograd:
                la, ph = LogPsi.apply(self.params, self.model, bits[sl])
                (la * g_abs[sl]).sum().add((ph * g_phase[sl]).sum()).backward()
            else:
                nqs_logpsi_backward(self.model, bits[sl], g_abs[sl], g_phase[sl], self.params.grad,
                                    ws=self._workspace(OP_BACKWARD, per))
        return dict(bits=bits, counts=counts, eloc=eloc, stats=stats, unique=U)

    def _gradient_parallel(self, bits, counts, eloc, per, ahead):
        """Data-parallel gradient: this rank's two backward sums, one all-reduce (parallel.combine)."""
        sums, ga_e, gp_e, ga_w = nqs_energy_sums(eloc, counts)
        first = torch.zeros_like(self.params)
        second = torch.zeros_like(self.params)
        zero = torch.zeros_like(ga_w)
        if ahead:   # the overlapped recompute served one backward; the second recomputes itself
            torch.cuda.current_stream().wait_stream(self._side)
            nqs_logpsi_backward_phase(self.model, 2, bits, ga_e, gp_e, first, ws=self._workspace(OP_BACKWARD, per))
            nqs_logpsi_backward(self.model, bits, ga_w, zero, second, ws=self._workspace(OP_BACKWARD, per))
        else:
            for sl in self._slices(bits.shape[0]):
                ws = self._workspace(OP_BACKWARD, per)
                nqs_logpsi_backward(self.model, bits[sl], ga_e[sl], gp_e[sl], first, ws=ws)
                nqs_logpsi_backward(self.model, bits[sl], ga_w[sl], zero[sl], second, ws=ws)
        grad, stats = parallel.combine(sums, first, second, self.group)
        if self.params.grad is None:
            self.params.grad = grad
        else:
            self.params.grad.copy_(grad)
        return dict(bits=bits, counts=counts, eloc=eloc, stats=stats, unique=bits.shape[0])
