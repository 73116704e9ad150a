"""Benchmark: one VMC step of the NQS local-energy hot path per timed step.

A step runs every part of the path on one batch of synthetic input: unique-sample sampling with
counts, the grouped popcount term sweep, the network on every connected x' (prefix reuse or x'
deduplication) with the ratio-weighted reduction, in the workload's mini-batches, FP64 energy
statistics, the log psi backward with recomputation (mini-batched) and one Adam update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload ID] [--impl ours|reference]

Default workload: the 52-qubit one (26 orbitals, 8+8 electrons, 669,579 Pauli strings,
transformer d_model 128, 4 layers, 8 heads, 2^18 nominal samples in 16 mini-batches), in the
compensated BF16 form, output bias beta = 2 ("trained-like"), the paper's batch of 1024 unique
samples (Section 5.1).  The FP32 form is timed beside it on the same workload.

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

DEFAULT_WORKLOAD = 5

# DRAM bytes (read + write) per algorithmic byte of a scope's launch, from one ncu capture of the
# same kernel on the same workload shape (an entry is removed when its kernel changes).
NCU_TRAFFIC = {
    ("large_52q_tf128x4", "bf16", "tf_mlp"): 0.98,
    ("large_52q_tf128x4", "bf16", "tf_gemm"): 1.0,
    ("large_52q_tf128x4", "bf16", "tf_layernorm"): 0.91,
    ("large_52q_tf128x4", "bf16", "ch_attention"): 1.18,
}

# The library's profiled scopes that record their algorithmic FLOPs and compulsory bytes, with
# the kernels behind each (bf16 form, fp32 form).
SCOPE_KERNELS = {
    "tf_gemm": ("tc_gemm_kernel (tcgen05 + TMA + TMEM: QKV and attention-output projections)",
                "sgemm_kernel (fp32 SIMT)"),
    "tf_mlp": ("tc_mlp_kernel / tc_mlp_res_kernel (fused tcgen05 MLP block, hidden layer on chip)",
               "sgemm_kernel (fp32 SIMT, W1 + GELU and W2 + residual)"),
    "tf_qkv_attention": ("tc_qkv_attn_kernel (fused QKV projection + causal attention, d_model 64)", None),
    "tf_resid_ln": ("tc_gemm_kernel<RESID_LN> (attention output + residual + LayerNorm 2, d_model 64)", None),
    "ch_attention": ("ch_attention_mma_kernel (causal attention of the prefix-sharing jobs, mma.sync m16n8k16, "
                     "compensated bf16 products)",
                     "ch_attention_kernel (causal attention of the prefix-sharing jobs, fp32 SIMT)"),
    "tf_layernorm": ("layernorm_kernel / ch_embed_ln_kernel (LayerNorm and embedding rows)",) * 2,
    "ch_cache": ("ch_cache_fill_kernel (key/value caches of the prefix-sharing jobs)",) * 2,
    "eloc_rows": (None, "eloc_rows_kernel (MADE / product log psi of every connected x' with the ratio-weighted "
                        "reduction fused, fp32 FFMA, one row per thread)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", type=int, default=DEFAULT_WORKLOAD)
    ap.add_argument("--beta", type=float, default=2.0,
                    help="output-head bias toward Hartree-Fock; 2 = trained-like, 0 = near uniform")
    ap.add_argument("--max-unique", type=int, default=1024,
                    help="unique-sample cap of the sampler; the paper fixes 1024 (Section 5.1)")
    ap.add_argument("--precision", default=None, help="bf16 (compensated) or fp32; default: the "
                    "workload's fastest form (bf16 for transformers)")
    ap.add_argument("--fp32-steps", type=int, default=1, help="steps of the FP32 form timed beside "
                    "the BF16 one for the speedup (0: skip)")
    ap.add_argument("--sweep-samples", type=int, default=1 << 16,
                    help="samples of the term-sweep microbenchmark (0: skip)")
    ap.add_argument("--mode", default="step", choices=["step", "sweep", "eloc"],
                    help="step: the VMC-step benchmark (the JSON line); sweep: the term-sweep "
                         "microbenchmark alone on --sweep-samples samples; eloc: the local energy alone on "
                         "--eloc-samples seeded in-sector samples (each its own JSON line; small cases for "
                         "profiler captures)")
    ap.add_argument("--eloc-samples", type=int, default=64, help="samples of the local-energy microbenchmark")
    ap.add_argument("--pass-bytes", type=int, default=0,
                    help="activation bytes of one prefix-sharing sub-pass (0: the library default)")
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
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

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


def golden(cfg, quant):
    """Stored FP64 oracle local energies of the benchmark's first batch (tests/golden), or None."""
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        from make_eloc_golden import golden_path, read_golden
        if not os.path.exists(golden_path(cfg, quant)):
            return None
        return read_golden(cfg, quant)
    except Exception:
        return None


def err_vs_oracle(bits, eloc, gold):
    """rel_norm and element-wise error of a step's local energies on the stored samples."""
    if gold is None:
        return None
    gb, _, ge, ga, _ = gold
    idx = np.searchsorted(bits, gb)
    ok = (idx < len(bits))
    ok[ok] &= bits[idx[ok]] == gb[ok]
    if not np.any(ok):
        return None
    got = eloc[idx[ok], 0].astype(np.float64) + 1j * eloc[idx[ok], 1]
    want, absum = ge[ok], ga[ok]
    rn = float(np.sqrt(np.sum(np.abs(got - want) ** 2) / np.sum(np.abs(want) ** 2)))
    em = float(np.max(np.abs(got - want) / (np.abs(want) + absum * 2.0 ** -24)))
    return {"rel_norm": rn, "elementwise": em, "samples": int(ok.sum())}


# ----------------------------------------------------------------------------- our arm
def scope_roofline(name, k, prec, cfg_name, ceilings):
    """Roofline entry of one profiled scope ({ms_total, launches, ms_per_step, flops, bytes} over
    the profiled steps), or None when the scope records no work or has no kernel of this form.
    The scope has two ceilings: its arithmetic (the sustained bf16 tensor peak for the bf16 form,
    the FFMA pipe for the fp32 form) and HBM; `bound` is the one whose time at peak is larger.
    `traffic` is the measured DRAM-bytes ratio of NCU_TRAFFIC times the launch's compulsory bytes."""
    sec = k["ms_total"] / 1e3
    if sec <= 0 or name not in SCOPE_KERNELS or (k["flops"] <= 0 and k["bytes"] <= 0):
        return None
    kernel = SCOPE_KERNELS[name][0 if prec == "bf16" else 1]
    if kernel is None:
        return None
    per = k["launches"]
    tr = NCU_TRAFFIC.get((cfg_name, prec, name))
    peak_b = ceilings["hbm_gbs"]
    if prec == "bf16":
        pk_c, bound_c = ceilings["tensor_tflops"], "tensor"
        src_c = f"{ceilings['peak_kind']} sustained bf16 cuBLAS (MEASURED_PEAKS.json); useful FLOPs (the " \
                "compensated hi+lo split issues twice as many products)"
    else:
        pk_c, bound_c = ceilings["ffma_tflops"], "alu"
        src_c = ceilings["ffma_src"]
    t_c = k["flops"] / (pk_c * 1e12)
    t_m = k["bytes"] / (peak_b * 1e9)
    ach_c = k["flops"] / sec / 1e12
    ach_m = k["bytes"] / sec / 1e9
    if t_c >= t_m:
        r = {"kernel": kernel, "bound": bound_c, "achieved": ach_c, "peak": pk_c, "unit": "TFLOP/s",
             "frac": ach_c / pk_c, "peak_source": src_c}
    else:
        r = {"kernel": kernel, "bound": "hbm", "achieved": ach_m, "peak": peak_b, "unit": "GB/s",
             "frac": ach_m / peak_b, "peak_source": f"{ceilings['peak_kind']} HBM copy bandwidth (MEASURED_PEAKS.json)"}
    r["flops_per_launch"] = k["flops"] / per
    r["bytes_per_launch"] = k["bytes"] / per
    r["compute_frac"] = ach_c / pk_c if k["flops"] > 0 else None
    r["hbm_frac"] = ach_m / peak_b if k["bytes"] > 0 else None
    r["intensity_flop_per_byte"] = k["flops"] / k["bytes"] if k["bytes"] > 0 else None
    r["ms_per_step"] = k["ms_per_step"]
    r["traffic"] = tr * (k["bytes"] / per) if (tr and k["bytes"] > 0) else None
    return r


def dominant_roofline(rooflines):
    """The entry of the scope with the largest time per step (the line's `roofline`), or None."""
    if not rooflines:
        return None
    top = max(rooflines, key=lambda nm: rooflines[nm]["ms_per_step"])
    roofline = dict(rooflines[top])
    roofline["scope"] = top
    roofline["note"] = ("dominant kernel of the step by time; achieved = the scope's algorithmic FLOPs (or "
                        "bytes) over its CUDA-event time on the launching stream in a profiled pass of the "
                        "timed steps")
    return roofline


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    import paper_2208_05637_b300 as P

    torch.cuda.set_device(local)
    cfg = synth.get_config(args.workload)
    n = cfg.n_qubits
    xm, zm, coef = hamiltonian_of(cfg)
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

    def timed_steps(v, k, first_seed, e2e=False, host=None, keep_first=False):
        # every step starts from the same parameters and optimiser state (a stationary workload:
        # the same distribution, a new seed), reset outside the timed events except that the
        # end-to-end form uploads the parameters from pinned host memory inside them
        times, evals, units, first = [], 0, [], None
        for i in range(k):
            flush.random_(0, 255)        # evict L2 between steps (outside the timed events)
            v.reset(params0)
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if e2e:
                v.params.data.copy_(host["params"], non_blocking=True)
            out = v.step(seed=first_seed + i)
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
            if keep_first and i == 0:
                first = (out["bits"].clone(), out["eloc"].clone())
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in times]
        return ms, evals, units, first

    # warmup
    for i in range(args.warmup):
        vmc.reset(params0)
        vmc.step(seed=seed0 + 100000 + i)
    barrier()

    # timed region (no profiling)
    launches0 = P.launch_count()
    with ClockSampler(local) as clk:
        barrier()
        ms, evals, units, first = timed_steps(vmc, args.steps, seed0, keep_first=True)
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
    fb = first[0].cpu().numpy().view(np.uint64)
    fe = first[1].cpu().numpy()
    g_main = golden(cfg, "bf16x2" if prec == "bf16" else "none")
    g_fp64 = golden(cfg, "none")
    errors = {"form": err_vs_oracle(fb, fe, g_main)}
    if prec == "bf16":
        errors["form_vs_unquantised_fp64"] = err_vs_oracle(fb, fe, g_fp64)

    # second pass with per-kernel events on the launching stream
    P.profile_reset(); P.profile_enable(True)
    ms_p, _, units_p, _ = timed_steps(vmc, args.steps, seed0)
    P.profile_enable(False)
    kern = {}
    names = ("sample", "local_energy", "sweep_count", "term_sweep", "eloc_rows", "made_backward", "grad_reduce",
             "energy_stats", "adam", "product_backward", "tf_gemm", "tf_qkv_attention", "tf_resid_ln", "tf_mlp",
             "tf_attention", "tf_heads", "tf_layernorm", "tf_tok_table", "tf_step_fused", "dedup", "dedup_contrib",
             "ch_build", "ch_cache", "ch_attention", "ch_heads", "tf_backward", "tf_backward_recompute",
             "bwd_recompute", "bwd_heads", "bwd_mlp", "bwd_attention", "bwd_embed")
    for name in names:
        tms, cnt = P.profile_read(name)
        if cnt:
            w, by = P.profile_work(name)
            kern[name] = {"ms_total": tms, "launches": cnt, "ms_per_launch": tms / cnt,
                          "ms_per_step": tms / max(1, args.steps), "flops": w, "bytes": by}

    peaks, peak_kind = load_peaks()
    clk_mhz = peaks.get("sm_max_mhz", 2032.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pipes = P.probe_pipes()
    ffma_peak = sms * 2 * pipes["ffma"] * clk_mhz * 1e6 / 1e12
    popc_peak = sms * pipes["popc"] * clk_mhz * 1e6 / 1e9
    rooflines = {}
    peak_t = peaks.get("bf16_tflops_sustained", 1400.0)
    peak_b = peaks.get("hbm_gbs", 6400.0)
    ceilings = {"tensor_tflops": peak_t, "hbm_gbs": peak_b, "ffma_tflops": ffma_peak, "peak_kind": peak_kind,
                "ffma_src": f"fp32 FFMA: {sms} SMs x {pipes['ffma']:.1f}/clk (probe) x 2 x {clk_mhz:.0f} MHz"}
    for name, k in kern.items():
        r = scope_roofline(name, k, prec, cfg.name, ceilings)
        if r is not None:
            rooflines[name] = r
    # backward: tensor roofline from the layer shapes (forward recompute + two backward GEMMs per
    # forward GEMM on U x n rows), the backward scope's time
    if cfg.arch == "transformer" and "tf_backward" in kern:
        d, L = cfg.hidden, cfg.layers
        rows = float(np.mean(units_p)) * n
        fl = 3.0 * 2.0 * rows * 12.0 * d * d * L
        sec = kern["tf_backward"]["ms_total"] / max(1, args.steps) / 1e3
        if "tf_backward_recompute" in kern:
            sec += kern["tf_backward_recompute"]["ms_total"] / max(1, args.steps) / 1e3
        ach = fl / sec / 1e12
        pk = peak_t if prec == "bf16" else ffma_peak
        rooflines["tf_backward"] = {"kernel": "tf_backward (recompute + backward GEMMs, tb_gemm on mma.sync)",
                                    "bound": "tensor" if prec == "bf16" else "alu", "achieved": ach, "peak": pk,
                                    "unit": "TFLOP/s", "frac": ach / pk, "ms_per_step": sec * 1e3,
                                    "flops_per_step": fl, "traffic": None,
                                    "peak_source": "FLOPs from the layer shapes: 3 x forward"}
    roofline = dominant_roofline(rooflines)

    # term-sweep microbenchmark (B random in-sector samples, 1024 per call)
    sweep = None
    if args.sweep_samples > 0 and rank == 0:
        sweep = sweep_microbench(P, torch, cfg, ham, args.sweep_samples, popc_peak, pipes, sms, clk_mhz)

    # end to end through the public API with host buffers
    import torch as _t
    host = {"params": params0.detach().cpu().pin_memory(),
            "stats": _t.empty(4, dtype=_t.float64).pin_memory(),
            "eloc": _t.empty((cfg.n_samples, 2), dtype=_t.float32).pin_memory()}
    vmc.params.data.copy_(params0)
    ms_e, evals_e, units_e, _ = timed_steps(vmc, args.steps, seed0, e2e=True, host=host)
    e2e_value = evals_e / (np.sum(ms_e) / 1e3)
    if world > 1:
        t = _t.tensor([e2e_value], dtype=_t.float64, device="cuda")
        dist.all_reduce(t)
        e2e_value = t.item()

    fp32_form = None
    if prec == "bf16" and args.fp32_steps > 0:
        del vmc, model
        torch.cuda.empty_cache()
        m32 = P.Model(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                      precision="fp32", compensated=True, order=order)
        v32 = P.VMC(ham, m32, params0.clone(), cfg.n_samples, mini_batches=cfg.mini_batches,
                    max_unique=args.max_unique)
        v32.step(seed=seed0 + 50000)
        torch.cuda.synchronize()
        ms32, ev32, _, f32 = timed_steps(v32, args.fp32_steps, seed0, keep_first=True)
        e32 = err_vs_oracle(f32[0].cpu().numpy().view(np.uint64), f32[1].cpu().numpy(), g_fp64)
        fp32_form = {"ms_per_step": float(np.mean(ms32)), "value": ev32 / (np.sum(ms32) / 1e3),
                     "steps": args.fp32_steps, "speedup_of_bf16": float(np.mean(ms32)) / step_ms,
                     "err_vs_oracle": e32}
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
            "data": "synthetic (seeded molecule-shaped integrals, Jordan-Wigner strings, random-init weights)",
            "config": dict(workload_config(cfg, args, K_terms, G), unique_samples_mean=float(np.mean(units)),
                           precision=prec, compensated=True, l2="flushed between steps (256 MB write)",
                           parallelism=f"replicas x{world}"),
            "err_vs_oracle": errors,
            "roofline": roofline,
            "rooflines": rooflines or None,
            "pipes_per_sm_per_clk": pipes,
            "term_sweep_microbench": sweep,
            "kernels": kern,
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


def hamiltonian_of(cfg):
    """The workload's Pauli strings: one-word masks up to 64 qubits, two-word masks beyond."""
    return synth.hamiltonian_for(cfg) if cfg.n_qubits <= 64 else synth.hamiltonian_words_for(cfg)


def sector_bits_of(cfg, count, seed):
    """Seeded in-sector configurations of the workload ([count] or [count, 2] uint64)."""
    if cfg.n_qubits <= 64:
        return synth.random_sector_bits(cfg.n_orb, cfg.n_up, cfg.n_dn, count, seed=seed)
    return synth.random_sector_bits_words(cfg.n_orb, cfg.n_up, cfg.n_dn, count, seed=seed, words=2)


def sweep_microbench(P, torch, cfg, ham, B, popc_peak, pipes, sms, clk_mhz):
    """The grouped term sweep alone on B seeded in-sector samples (1024 per nqs_term_sweep call),
    count and emit kernels timed with CUDA events; performed (sample, term) pairs counted from the
    emitted rows.  POPC work per (sample, group): one per spin species and word (the two 32-bit
    halves of a word folded into one 32-bit word), so 2 for one-word and 4 for two-word registers;
    per performed (sample, term): 1 for the parity (all halves XOR-folded into one word)."""
    W = ham.words
    ex = ham.export()
    gsz = torch.tensor(np.diff(ex["group_offset"]), device="cuda")
    gm = torch.tensor(np.ascontiguousarray(ex["group_mask"]).view(np.int64), device="cuda")
    if W > 1:
        gm = gm.reshape(-1, W)
    K, G = ham.info()
    chunk = 1024
    bits_all = sector_bits_of(cfg, B, 4242)

    def dev(b):
        t = torch.tensor(np.ascontiguousarray(b).view(np.int64), device="cuda")
        return t if W == 1 else t.reshape(-1, W)
    # one warm-up call
    P.nqs_term_sweep(ham, cfg.n_up, cfg.n_dn, dev(bits_all[:chunk]))
    t_ms, terms, rows = 0.0, 0, 0
    for lo in range(0, B, chunk):
        bt = dev(bits_all[lo: lo + chunk])
        P.profile_reset(); P.profile_enable(True)
        ro, xp, _, _ = P.nqs_term_sweep(ham, cfg.n_up, cfg.n_dn, bt)
        P.profile_enable(False)
        t_ms += P.profile_read("sweep_count")[0] + P.profile_read("term_sweep")[0]
        cnt = ro[1:] - ro[:-1]
        m = torch.repeat_interleave(bt, cnt, dim=0) ^ xp
        if W == 1:
            terms += int(gsz[torch.searchsorted(gm, m)].sum())
        else:
            # group of each row's flip mask: unique over group masks and row masks together
            _, inv = torch.unique(torch.cat([gm, m]), dim=0, return_inverse=True)
            size_of_key = torch.zeros(int(inv.max()) + 1, dtype=gsz.dtype, device="cuda")
            size_of_key[inv[:G]] = gsz
            terms += int(size_of_key[inv[G:]].sum())
        rows += xp.shape[0]
    sec = t_ms / 1e3
    popc_ops = 2.0 * W * B * G + terms
    ach = popc_ops / sec / 1e9
    return {"samples": B, "chunk": chunk, "ms": t_ms,
            "nominal_pairs_per_s": B * K / sec, "performed_terms_per_s": terms / sec,
            "performed_terms_per_sample": terms / B, "rows_per_sample": rows / B,
            "roofline": {"bound": "alu", "kernel": "sweep_count_kernel + sweep_emit_kernel", "achieved": ach,
                         "peak": popc_peak, "unit": "Gpopc/s", "frac": ach / popc_peak,
                         "peak_source": f"POPC: {sms} SMs x {pipes['popc']:.1f}/clk (probe) x {clk_mhz:.0f} MHz",
                         "work": f"{2 * W} POPC per (sample, group) + 1 per performed (sample, term)"}}


def run_sweep(args, local):
    """The term-sweep microbenchmark alone (one JSON line)."""
    import torch
    import paper_2208_05637_b300 as P
    torch.cuda.set_device(local)
    cfg = synth.get_config(args.workload)
    xm, zm, coef = hamiltonian_of(cfg)
    ham = P.Hamiltonian(cfg.n_qubits, xm, zm, coef)
    peaks, _ = load_peaks()
    clk_mhz = peaks.get("sm_max_mhz", 2032.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pipes = P.probe_pipes()
    popc_peak = sms * pipes["popc"] * clk_mhz * 1e6 / 1e9
    with ClockSampler(local) as clk:
        res = sweep_microbench(P, torch, cfg, ham, max(1024, args.sweep_samples), popc_peak, pipes, sms, clk_mhz)
    K, G = ham.info()
    print(json.dumps({"metric": "term-sweep (sample, Pauli term) pairs/s", "workload": cfg.name, "terms_K": K,
                      "groups_G": G, "pipes_per_sm_per_clk": pipes, "term_sweep_microbench": res,
                      "clocks": clk.summary()}))


def run_eloc(args, local):
    """The local energy alone (nqs_local_energy) on seeded in-sector samples of the workload: one
    warm-up call, then one profiled call; per-scope CUDA-event times (one JSON line)."""
    import torch
    import paper_2208_05637_b300 as P
    torch.cuda.set_device(local)
    cfg = synth.get_config(args.workload)
    n = cfg.n_qubits
    xm, zm, coef = hamiltonian_of(cfg)
    ham = P.Hamiltonian(n, xm, zm, coef)
    order = synth.default_order(n)
    named = synth.init_params(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                              cfg.seed_params, beta=args.beta, order=order)
    prec = args.precision or ("bf16" if cfg.arch == "transformer" else "fp32")
    model = P.Model(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                    precision=prec, compensated=True, order=order)
    model.bind(model.pack(named))
    if args.pass_bytes and cfg.arch == "transformer":
        model.set_pass_bytes(args.pass_bytes)
    bits = sector_bits_of(cfg, args.eloc_samples, 77)
    bt = torch.tensor(np.ascontiguousarray(bits).view(np.int64), device="cuda")
    if bits.ndim == 2:
        bt = bt.reshape(-1, bits.shape[1])
    P.nqs_local_energy(ham, model, bt)
    torch.cuda.synchronize()
    P.profile_reset(); P.profile_enable(True)
    a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
    a.record()
    e = P.nqs_local_energy(ham, model, bt)
    b.record()
    torch.cuda.synchronize()
    P.profile_enable(False)
    scopes = {}
    for name in ("term_sweep", "sweep_count", "ch_build", "ch_cache", "ch_attention", "ch_heads", "tf_gemm", "tf_mlp",
                 "tf_layernorm", "dedup", "dedup_contrib", "tf_qkv_attention", "tf_resid_ln", "eloc_rows"):
        ms, c = P.profile_read(name)
        if c:
            fl, by = P.profile_work(name)
            scopes[name] = {"ms": ms, "launches": c, "flops": fl, "bytes": by}
    print(json.dumps({"metric": "local energy (sample.term/s)", "workload": cfg.name, "precision": prec,
                      "samples": args.eloc_samples, "ms": a.elapsed_time(b),
                      "value": args.eloc_samples * ham.info()[0] / (a.elapsed_time(b) / 1e3),
                      "pass_bytes": args.pass_bytes, "finite": bool(torch.isfinite(e).all().item()),
                      "scopes": scopes}))


def workload_config(cfg, args, K, G):
    """The workload keys of the JSON line's config (the same for both arms)."""
    return {"workload": cfg.name, "n_qubits": cfg.n_qubits, "electrons": [cfg.n_up, cfg.n_dn],
            "terms_K": int(K), "groups_G": int(G),
            "model": f"{cfg.arch} d={cfg.hidden} L={cfg.layers} H={cfg.heads}",
            "n_samples": cfg.n_samples, "max_unique": args.max_unique,
            "batch": "capped: the paper's 1024 unique samples per step (Section 5.1); the sampler "
                     "draws the nominal count and keeps the 1024 most frequent",
            "mini_batches": cfg.mini_batches, "beta": args.beta}


# ----------------------------------------------------------------------------- oracle timing
def cpu_baseline(cfg, args, budget_s=15.0):
    """The FP64 oracle as it stands on this host, on a bounded sample of the workload: local
    energies (per-term definition, FP64 network) of seeded in-sector configurations, one at a
    time until the time budget is used; on workloads where one sample over all terms exceeds the
    budget, one sample over a seeded subset of the terms (the rate is per evaluated term).
    Sampling and the gradient are not included, which favours the CPU figure."""
    import torch
    from oracle.eloc import local_energy as local_energy_one_word
    from oracle.models import Model
    from oracle.wide import local_energy_words

    n = cfg.n_qubits
    order = synth.default_order(n)
    named = synth.init_params(cfg.arch, n, cfg.n_up, cfg.n_dn, cfg.hidden, cfg.layers, cfg.heads,
                              cfg.seed_params, beta=args.beta, order=order)
    xm, zm, coef = hamiltonian_of(cfg)
    om = Model(cfg.arch, named, n, cfg.n_up, cfg.n_dn, order, cfg.hidden, cfg.layers, cfg.heads)
    bits = sector_bits_of(cfg, 4096, cfg.seed_sampler)
    local_energy = local_energy_one_word if n <= 64 else local_energy_words
    # terms per call: all of them, or the share one call can do in about a third of the budget
    frac = 1.0
    if cfg.n_qubits >= 30:
        t0 = time.perf_counter()
        sub = np.random.default_rng(1).choice(len(coef), max(64, len(coef) // 256), replace=False)
        local_energy(om, xm[sub], zm[sub], coef[sub], bits[:1])
        per_term = (time.perf_counter() - t0) / len(sub)
        frac = min(1.0, (budget_s / 3) / (per_term * len(coef)))
    sub = np.sort(np.random.default_rng(2).choice(len(coef), max(1, int(frac * len(coef))), replace=False)) \
        if frac < 1.0 else np.arange(len(coef))
    done, t = 0, 0.0
    while done < len(bits) and t < budget_s:
        t0 = time.perf_counter()
        local_energy(om, xm[sub], zm[sub], coef[sub], bits[done: done + 1])
        t += time.perf_counter() - t0
        done += 1
    what = "all" if frac >= 1.0 else f"a seeded subset of {len(sub)} of the"
    return {"value": done * len(sub) / t, "unit": "sample.term/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle local energy of {done} seeded in-sector samples over {what} {len(coef)} "
                      f"terms of the workload ({t:.1f} s); sampling and gradient excluded"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = synth.get_config(args.workload)
    xm_, _, _ = hamiltonian_of(cfg)
    K = len(xm_)
    G = len(np.unique(xm_, axis=0)) if xm_.ndim == 2 else len(np.unique(xm_))
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
            "config": dict(workload_config(cfg, args, K, G), precision="f64 (oracle)"),
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
    elif args.mode == "sweep":
        run_sweep(args, local)
    elif args.mode == "eloc":
        run_eloc(args, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
