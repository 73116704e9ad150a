"""Writes the stored expected local energies of the large workloads (oracle only).

    python tests/golden/make_eloc_golden.py --workload 5 --quant none   [--count 64]
    python tests/golden/make_eloc_golden.py --workload 5 --quant bf16x2 [--count 64]

The FP64 oracle takes minutes to hours on these workloads, so the GPU tests read its results
from the files this script writes instead of recomputing them.  Everything here comes from
`oracle/` and the seeded inputs of `synth/`: the oracle's unique-sample sampler (Section 4,
Sampling) runs the benchmark's first step -- the workload's nominal sample count, the
paper's batch of 1024 unique samples (Section 5.1), sampler seed 3000 + workload id, output
bias beta = 2 -- and the `count` samples with the highest occurrence counts (ties: smaller
bitstring first) get their local energy by the per-term definition (Eq. local_energy_auto)
together with the sum of the magnitudes of its terms.  quant "bf16x2" is the
quantisation-aware oracle of the compensated BF16 form, "none" the plain FP64 model.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle.eloc import local_energy  # noqa: E402
from oracle.models import Model  # noqa: E402
from oracle.sampler import model_p_fn, sample  # noqa: E402

BATCH = 1024
BETA = 2.0


def golden_path(cfg, quant):
    return os.path.join(HERE, f"eloc_{cfg.name}_{quant}.txt")


def read_golden(cfg, quant):
    """(bits uint64, counts int64, E complex128, A float64, header dict) of a stored file."""
    head, rows = {}, []
    with open(golden_path(cfg, quant)) as f:
        for line in f:
            if line.startswith("#"):
                if ":" in line:
                    k, v = line[1:].split(":", 1)
                    head[k.strip()] = v.strip()
                continue
            if line.strip():
                rows.append(line.split())
    bits = np.array([int(r[0], 16) for r in rows], dtype=np.uint64)
    counts = np.array([int(r[1]) for r in rows], dtype=np.int64)
    e = np.array([float.fromhex(r[2]) + 1j * float.fromhex(r[3]) for r in rows])
    a = np.array([float.fromhex(r[4]) for r in rows])
    return bits, counts, e, a, head


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, required=True)
    ap.add_argument("--quant", choices=["none", "bf16x2"], required=True)
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--logpsi-chunk", type=int, default=256,
                    help="configurations per oracle log psi batch (speed only; values are per row)")
    args = ap.parse_args()
    cfg = synth.get_config(args.workload)
    n = cfg.n_qubits
    order = synth.default_order(n)
    params = synth.init_params(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                               cfg.seed_params, beta=BETA, order=order)
    model = Model(cfg.arch, params, n, cfg.n_up, cfg.n_dn, order, cfg.hidden, cfg.layers, cfg.heads,
                  quant=None if args.quant == "none" else args.quant)
    log_psi = model.log_psi
    model.log_psi = lambda b, chunk=args.logpsi_chunk: log_psi(b, chunk=chunk)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    t0 = time.time()
    bits, counts = sample(model_p_fn(model), n, order, cfg.n_samples, BATCH, cfg.seed_sampler)
    t_s = time.time() - t0
    print(f"sampler: {len(bits)} unique samples in {t_s:.0f} s", flush=True)
    top = np.lexsort((bits, -counts))[: args.count]
    top = top[np.argsort(bits[top], kind="stable")]
    sel_b, sel_c = bits[top], counts[top]
    cut = np.sort(counts)[::-1][min(args.count, len(counts) - 1)]
    out = []
    t0 = time.time()
    for i, x in enumerate(sel_b):
        e, a = local_energy(model, xm, zm, coef, np.array([x], dtype=np.uint64), return_abs=True)
        out.append((x, sel_c[i], e[0], a[0]))
        print(f"  {i + 1}/{len(sel_b)}  {time.time() - t0:.0f} s", flush=True)
    with open(golden_path(cfg, args.quant), "w") as f:
        f.write(f"# FP64 oracle local energies (Eq. local_energy_auto) of the {len(out)} highest-count samples of\n")
        f.write(f"# the oracle sampler's batch (Section 4, Sampling) on workload {cfg.name}; written by\n")
        f.write("# tests/golden/make_eloc_golden.py from oracle/ and synth/ only.\n")
        f.write(f"# workload: {cfg.name}\n# quant: {args.quant}\n# beta: {BETA}\n")
        f.write(f"# n_samples: {cfg.n_samples}\n# max_unique: {BATCH}\n# seed: {cfg.seed_sampler}\n")
        f.write(f"# batch_unique: {len(bits)}\n# next_count_below: {cut}\n")
        f.write("# columns: bits (hex), count, Re E_loc, Im E_loc, sum of |term| (float hex)\n")
        for x, c, e, a in out:
            f.write(f"{int(x):016x} {int(c)} {float(e.real).hex()} {float(e.imag).hex()} {float(a).hex()}\n")
    print("wrote", golden_path(cfg, args.quant))


if __name__ == "__main__":
    main()
