"""VMC training to convergence on a named synthetic workload, with a choice of sampling order
(paper Section 5.1 set-up: Adam, lr 1e-3, betas (0.9, 0.99), a batch of unique samples per
iteration; Section 4: sampling order, the reverse order being the paper's default; Table 2 top:
the order ablation).

    python -m paper_2208_05637_b300.train --workload 2 --order reverse --iters 10000

Prints one JSON line: the energy trace (every `--every` iterations), the mean energy over the last
10% of the iterations, the wall time and the time per iteration.  The ground energy of the
particle-number sector, where a caller wants to compare, is a separate computation (the library
has no dense or Lanczos eigensolver).
"""
import argparse
import json
import os
import sys
import time

import numpy as np


def orders(n: int, kind: str, seed: int = 0) -> np.ndarray:
    """Sampling order: position t samples qubit order[t].  reverse (the paper's default): n-1 .. 0;
    forward: 0 .. n-1; random: a seeded permutation."""
    if kind == "reverse":
        return np.arange(n - 1, -1, -1)
    if kind == "forward":
        return np.arange(n)
    if kind == "random":
        return np.random.default_rng(seed).permutation(n)
    raise ValueError(f"unknown order {kind}")


def train(workload: int, order_kind: str = "reverse", iters: int = 10000, beta: float = 0.0,
          precision=None, max_unique: int = 1024, lr: float = 1e-3, every: int = 100, seed: int = 0):
    """Runs `iters` VMC steps from the workload's seeded initial parameters; returns a dict with
    the energy trace and timings."""
    import torch
    import paper_2208_05637_b300 as P
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth

    cfg = synth.get_config(workload)
    n = cfg.n_qubits
    order = orders(n, order_kind, seed)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(n, xm, zm, coef)
    named = synth.init_params(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                              cfg.seed_params, beta=beta, order=order)
    prec = precision or ("bf16" if cfg.arch == "transformer" else "fp32")
    model = P.Model(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                    precision=prec, compensated=True, order=order)
    params = model.pack(named)
    vmc = P.VMC(ham, model, params, cfg.n_samples, mini_batches=cfg.mini_batches,
                max_unique=max_unique, lr=lr)
    trace, tail = [], []
    torch.cuda.synchronize()
    t0 = time.time()
    for it in range(iters):
        out = vmc.step(seed=cfg.seed_sampler + 7919 * seed + it)
        if it % every == 0 or it == iters - 1 or it >= iters - max(1, iters // 10):
            e = float(out["stats"][0].item())
            if it % every == 0 or it == iters - 1:
                trace.append((it, e))
            if it >= iters - max(1, iters // 10):
                tail.append(e)
    torch.cuda.synchronize()
    wall = time.time() - t0
    return {"workload": cfg.name, "order": order_kind, "precision": prec, "iters": iters,
            "max_unique": max_unique, "n_samples": cfg.n_samples, "energy_trace": trace,
            "energy_final_mean": float(np.mean(tail)), "energy_final_std": float(np.std(tail)),
            "wall_s": wall, "ms_per_iter": 1e3 * wall / max(1, iters)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--order", default="reverse", choices=["reverse", "forward", "random"])
    ap.add_argument("--iters", type=int, default=10000)
    ap.add_argument("--beta", type=float, default=0.0)
    ap.add_argument("--precision", default=None)
    ap.add_argument("--max-unique", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    print(json.dumps(train(a.workload, a.order, a.iters, a.beta, a.precision, a.max_unique, a.lr, a.every, a.seed)))


if __name__ == "__main__":
    main()
