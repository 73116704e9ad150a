"""Benchmark: one VMC step of the NQS local-energy hot path per timed step.

A step runs every part of the path on one batch of synthetic input: unique-sample sampling with
counts, the grouped popcount term sweep, the network on every connected x' with the fused
ratio-weighted reduction (mini-batched), FP64 energy statistics, the log psi backward with
recomputation (mini-batched) and one Adam update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload ID] [--impl ours|reference]

metric: sample.Pauli-term local-energy evaluations per second = sum over the step's local-energy
calls of (unique samples x Hamiltonian terms K), divided by the step time.  Under torchrun each
rank runs an independent replica (own sampler seed); the value is the sum over ranks divided
by the slowest rank's time (weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

DEFAULT_WORKLOAD = 3          # 20-qubit transformer: the first workload with BF16 and FP32 forms
FFMA_PER_SM_PER_CLK = 128      # fp32 lanes per SM (sm_100 family)

# DRAM bytes (read + write) per algorithmic byte of each transformer scope's big-pass launch, from
# the committed ncu capture named beside it (traffic = ratio x the scope's bytes per launch); an
# entry is removed once its kernel changes.
NCU_TRAFFIC = {
    ("n2_like_20q_tf64x2", "tf_qkv_attention"): (0.46, "profiles/qkv_attention_tf20q_bf16_ncu.md"),
    ("n2_like_20q_tf64x2", "tf_resid_ln"): (0.74, "profiles/resid_ln_tf20q_bf16_ncu.md"),
    ("n2_like_20q_tf64x2", "tf_mlp"): (0.85, "profiles/tc_mlp_tf20q_bf16_ncu.md"),
    ("n2_like_20q_tf64x2", "tf_layernorm"): (0.74, "profiles/layernorm_tf20q_bf16_ncu.md"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", type=int, default=DEFAULT_WORKLOAD)
    ap.add_argument("--beta", type=float, default=0.0,
                    help="output-head bias toward Hartree-Fock; 0 = untrained (near uniform)")
    ap.add_argument("--max-unique", type=int, default=1024,
                    help="unique-sample cap of the sampler; the paper fixes 1024 (Section 5.1)")
    ap.add_argument("--precision", default=None, help="bf16 (compensated) or fp32; default: the "
                    "workload's fastest form (bf16 for transformers)")
    ap.add_argument("--fp32-steps", type=int, default=5, help="steps of the FP32 form timed beside "
                    "the BF16 one for the speedup (0: skip)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    import paper_2208_05637_b300 as P

    torch.cuda.set_device(local)
    cfg = synth.get_config(args.workload)
    n = cfg.n_qubits
    xm, zm, coef = synth.hamiltonian_for(cfg)
    ham = P.Hamiltonian(n, xm, zm, coef)
    K_terms, G = ham.info()
    order = synth.default_order(n)
    named = synth.init_params(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                              cfg.seed_params, beta=args.beta, order=order)
    prec = args.precision or ("bf16" if cfg.arch == "transformer" else "fp32")
    model = P.Model(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                    precision=prec, compensated=True, order=order)
    params0 = model.pack(named)
    vmc = P.VMC(ham, model, params0.clone(), cfg.n_samples, mini_batches=cfg.mini_batches,
                max_unique=args.max_unique)
    seed0 = cfg.seed_sampler + 7919 * rank
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MB > 126 MB L2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(k, first_seed, e2e=False, host=None):
        # every step starts from the same parameters and optimiser state (a stationary workload:
        # the same distribution, a new seed), reset outside the timed events except that the
        # end-to-end form uploads the parameters from pinned host memory inside them
        times, evals, units = [], 0, []
        for i in range(k):
            flush.random_(0, 255)        # evict L2 between steps (outside the timed events)
            vmc.reset(params0)
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if e2e:
                vmc.params.data.copy_(host["params"], non_blocking=True)
            out = vmc.step(seed=first_seed + i)
            if e2e:
                host["stats"].copy_(out["stats"], non_blocking=True)
                U = out["unique"]
                host["eloc"][:U].copy_(out["eloc"], non_blocking=True)
            b.record(stream)
            if e2e:
                torch.cuda.synchronize()
            times.append((a, b))
            units.append(out["unique"])
            evals += out["unique"] * K_terms
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in times]
        return ms, evals, units

    # warmup
    for i in range(args.warmup):
        vmc.reset(params0)
        vmc.step(seed=seed0 + 100000 + i)
    barrier()

    # timed region (no profiling)
    launches0 = P.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        ms, evals, units = timed_steps(args.steps, seed0)
        barrier()
    launches = (P.launch_count() - launches0) / max(args.steps, 1)
    step_ms = float(np.mean(ms))
    tot_ms = float(np.sum(ms))
    # max over ranks of the time; sum over ranks of the work
    if world > 1:
        t = torch.tensor([tot_ms, float(evals)], dtype=torch.float64, device="cuda")
        tmax = t.clone(); dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t.clone(); dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        tot_ms_all, evals_all = tmax[0].item(), tsum[1].item()
    else:
        tot_ms_all, evals_all = tot_ms, float(evals)
    value = evals_all / (tot_ms_all / 1e3)

    # second pass with per-kernel events on the launching stream
    P.profile_reset(); P.profile_enable(True)
    ms_p, _, units_p = timed_steps(args.steps, seed0)
    P.profile_enable(False)
    kern = {}
    for name in ("sample", "local_energy", "logpsi_rows", "sweep_count", "term_sweep", "eloc_rows", "made_backward",
                 "grad_reduce", "energy_stats", "adam", "product_backward", "tf_gemm", "tf_qkv_attention", "tf_resid_ln", "tf_mlp", "tf_attention",
                 "tf_heads", "tf_layernorm", "tf_tok_table", "tf_step_fused", "dedup", "dedup_contrib", "tf_backward",
                 "tf_backward_recompute", "bwd_recompute",
                 "bwd_heads", "bwd_mlp", "bwd_attention", "bwd_embed"):
        tms, cnt = P.profile_read(name)
        if cnt:
            kern[name] = {"ms_total": tms, "launches": cnt, "ms_per_launch": tms / cnt}
    rows_per_step = None

    # roofline of the dominant hot-path kernel: the transformer scope with the largest time
    # among those whose algorithmic bytes are recorded, and the same figures for the others
    roofline = None
    rooflines = {}
    peaks, peak_kind = load_peaks()
    clk_mhz = peaks.get("sm_max_mhz", 2032.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    ffma_peak = sms * FFMA_PER_SM_PER_CLK * 2 * clk_mhz * 1e6 / 1e12
    tf_scopes = {"tf_gemm": "tc_gemm_kernel (tcgen05 GEMM: QKV projection)",
                 "tf_qkv_attention": "tc_qkv_attn_kernel (fused QKV projection + causal attention; first block "
                                     "gathers q|k|v from the token-position table)",
                 "tf_resid_ln": "tc_gemm_kernel<RESID_LN> (attention output + residual + LayerNorm 2)",
                 "tf_mlp": "tc_mlp_res_kernel (fused tcgen05 MLP block; the last one with LNf and the output head)",
                 "tf_attention": "attention_grp_kernel (causal attention)",
                 "tf_layernorm": "layernorm_kernel (LayerNorm 1 of the second block)",
                 "tf_heads": "heads_reduce_kernel (constraint, log-sigmoid sums, phase head, ratio-weighted contribution)"}
    if cfg.arch == "transformer" and prec == "bf16":
        peak_b = peaks.get("hbm_gbs", 6400.0)
        peak_t = peaks.get("bf16_tflops_sustained", 1400.0)
        for name, desc in tf_scopes.items():
            if name not in kern:
                continue
            work, wbytes = P.profile_work(name)
            if wbytes <= 0:
                continue
            k = kern[name]
            sec = k["ms_per_launch"] / 1e3
            ach_b = wbytes / k["launches"] / sec / 1e9
            tr = NCU_TRAFFIC.get((cfg.name, name))
            r = {"kernel": desc, "bound": "hbm", "achieved": ach_b, "peak": peak_b, "unit": "GB/s",
                 "frac": ach_b / peak_b, "ms_per_step": k["ms_total"] / max(1, args.steps),
                 "bytes_per_launch": wbytes / k["launches"],
                 "traffic": tr[0] * wbytes / k["launches"] if tr else None,
                 "traffic_source": tr[1] if tr else None,
                 "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json)"}
            if work > 0:
                # useful FLOPs (2MNK); the compensated split issues twice that on the tensor pipe
                r["flops_per_launch"] = work / k["launches"]
                r["flop_per_byte"] = work / wbytes
                r["tensor_tflops"] = work / k["launches"] / sec / 1e12
                r["tensor_frac"] = r["tensor_tflops"] / peak_t
            rooflines[name] = r
        if rooflines:
            top = max(rooflines, key=lambda nm: kern[nm]["ms_total"])
            roofline = dict(rooflines[top])
            roofline["note"] = ("dominant kernel of the step by time; bytes = compulsory operand reads + "
                                "result writes per launch; traffic = ncu DRAM bytes of the same launch "
                                "shape scaled to the mean launch")
    elif cfg.arch == "transformer" and "tf_gemm" in kern:
        work, wbytes = P.profile_work("tf_gemm")
        k = kern["tf_gemm"]
        sec = k["ms_per_launch"] / 1e3
        ach = work / k["launches"] / sec / 1e12
        roofline = {"kernel": "sgemm_kernel (fp32 SIMT)", "bound": "alu", "achieved": ach, "peak": ffma_peak,
                    "unit": "TFLOP/s", "frac": ach / ffma_peak, "traffic": None,
                    "peak_source": f"fp32 FFMA: {sms} SMs x {FFMA_PER_SM_PER_CLK} lanes x 2 x {clk_mhz:.0f} MHz",
                    "flops_per_launch": work / k["launches"], "bytes_per_launch": wbytes / k["launches"]}
    elif "eloc_rows" in kern and cfg.arch == "made":
        # rows = connected in-sector x' other than x itself, counted on one step's samples
        out = vmc.step(seed=seed0 + 999)
        bits = out["bits"]
        ro, xp, _, _ = P.nqs_term_sweep(ham, cfg.n_up, cfg.n_dn, bits)
        rows = int(xp.numel()) - int(bits.numel())
        h, L = cfg.hidden, cfg.layers
        macs = n * h + (L - 1) * h * h + n * h + (n - 2) * h + h
        launches_per_step = kern["eloc_rows"]["launches"] / max(1, args.steps)
        flops_launch = 2.0 * macs * rows / max(1.0, launches_per_step)
        per_launch_s = kern["eloc_rows"]["ms_per_launch"] / 1e3
        ach = flops_launch / per_launch_s / 1e12
        roofline = {"kernel": "eloc_rows", "bound": "alu", "achieved": ach, "peak": ffma_peak,
                    "unit": "TFLOP/s", "frac": ach / ffma_peak, "traffic": None,
                    "peak_source": f"fp32 FFMA: {sms} SMs x {FFMA_PER_SM_PER_CLK} lanes x 2 x "
                                   f"{clk_mhz:.0f} MHz (max clock)",
                    "flops_per_row": 2 * macs, "rows_per_launch": rows / max(1.0, launches_per_step)}

    # end to end through the public API with host buffers
    import torch as _t
    host = {"params": params0.detach().cpu().pin_memory(),
            "stats": _t.empty(4, dtype=_t.float64).pin_memory(),
            "eloc": _t.empty((cfg.n_samples, 2), dtype=_t.float32).pin_memory()}
    vmc.params.data.copy_(params0)
    ms_e, evals_e, units_e = timed_steps(args.steps, seed0, e2e=True, host=host)
    e2e_value = evals_e / (np.sum(ms_e) / 1e3)
    if world > 1:
        t = _t.tensor([e2e_value], dtype=_t.float64, device="cuda")
        dist.all_reduce(t)
        e2e_value = t.item()

    fp32_form = None
    if prec == "bf16" and args.fp32_steps > 0:
        m32 = P.Model(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                      precision="fp32", compensated=True, order=order)
        v32 = P.VMC(ham, m32, params0.clone(), cfg.n_samples, mini_batches=cfg.mini_batches,
                    max_unique=args.max_unique)
        v32.step(seed=seed0 + 50000)
        torch.cuda.synchronize()
        ms32, ev32 = [], 0
        for i in range(args.fp32_steps):
            flush.random_(0, 255)
            v32.reset(params0)
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            o32 = v32.step(seed=seed0 + i)
            b.record(stream)
            torch.cuda.synchronize()
            ms32.append(a.elapsed_time(b))
            ev32 += o32["unique"] * K_terms
        fp32_form = {"ms_per_step": float(np.mean(ms32)), "value": ev32 / (np.sum(ms32) / 1e3),
                     "steps": args.fp32_steps, "speedup_of_bf16": float(np.mean(ms32)) / step_ms}
        del v32, m32

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, args, budget_s=args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "sample.Pauli-term local-energy evals/sec (VMC step)",
            "value": value, "unit": "sample.term/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (hi+lo activations, fp32 accumulate)" if prec == "bf16" else "f32",
            "data": "synthetic",
            "config": {"workload": cfg.name, "n_qubits": n, "electrons": [cfg.n_up, cfg.n_dn],
                       "terms_K": K_terms, "groups_G": G, "model": f"{cfg.arch} h={cfg.hidden} L={cfg.layers}",
                       "n_samples": cfg.n_samples, "max_unique": args.max_unique,
                       "mini_batches": cfg.mini_batches,
                       "unique_samples_mean": float(np.mean(units)), "beta": args.beta,
                       "precision": prec, "compensated": True,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "rooflines": rooflines or None,
            "kernels": kern,
            "connected_rows_per_step": rows_per_step,
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "sample.term/s",
                    "h2d_bytes_per_step": int(host["params"].numel() * 4),
                    "d2h_bytes_per_step": int(32 + 8 * float(np.mean(units_e)))},
            "fp32_form": fp32_form,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "peaks_source": peak_kind,
        }
        print(json.dumps(line))


# ----------------------------------------------------------------------------- oracle timing
def cpu_baseline(cfg, args, budget_s=15.0):
    """The FP64 oracle as it stands on this host, on a bounded sample of the workload: local
    energies (per-term definition, FP64 network) of seeded in-sector configurations, one at a
    time until the time budget is used.  Sampling and the gradient are not included, which
    favours the CPU figure."""
    import torch
    from oracle.eloc import local_energy
    from oracle.models import Model

    n = cfg.n_qubits
    order = synth.default_order(n)
    named = synth.init_params(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                              cfg.seed_params, beta=args.beta, order=order)
    xm, zm, coef = synth.hamiltonian_for(cfg)
    om = Model(cfg.arch, named, n, cfg.n_up, cfg.n_dn, order, cfg.hidden, cfg.layers, cfg.heads)
    bits = synth.random_sector_bits(cfg.n_orb, cfg.n_up, cfg.n_dn, 4096, seed=cfg.seed_sampler)
    done, t = 0, 0.0
    while done < len(bits) and t < budget_s:
        t0 = time.perf_counter()
        local_energy(om, xm, zm, coef, bits[done: done + 1])
        t += time.perf_counter() - t0
        done += 1
    return {"value": done * len(coef) / t, "unit": "sample.term/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle local energy of {done} seeded in-sector samples of the workload "
                      f"({t:.1f} s; K = {len(coef)} terms each); sampling and gradient excluded"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = synth.get_config(args.workload)
    import torch
    per_step = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    vals = []
    for i in range(args.warmup + args.steps):
        v = cpu_baseline(cfg, args, budget_s=per_step)
        if i >= args.warmup:
            vals.append(v)
    value = float(np.mean([v["value"] for v in vals]))
    line = {"impl": "reference", "metric": "sample.Pauli-term local-energy evals/sec (VMC step)",
            "value": value, "unit": "sample.term/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name},
            "cpu_baseline": {"kind": "oracle", "cores": torch.get_num_threads(), "value": value,
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": "sample.term/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
