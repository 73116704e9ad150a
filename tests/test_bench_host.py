"""Host logic of the benchmark's roofline reporting (no GPU): the binding ceiling of a scope, the
fractions, the traffic scaling and the choice of the dominant scope."""
import math

import bench

CEIL = {"tensor_tflops": 1400.0, "hbm_gbs": 6500.0, "ffma_tflops": 75.0, "peak_kind": "measured",
        "ffma_src": "probe"}


def scope(ms_total, launches, flops, nbytes, steps=5):
    return {"ms_total": ms_total, "launches": launches, "ms_per_step": ms_total / steps,
            "flops": flops, "bytes": nbytes}


def test_high_intensity_scope_is_bound_by_the_tensor_ceiling():
    # 1e15 FLOP over 1e12 B (1000 FLOP/B, above the 215 FLOP/B ridge) in 2 s
    r = bench.scope_roofline("tf_mlp", scope(2000.0, 10, 1e15, 1e12), "bf16", "some_workload", CEIL)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["achieved"], 500.0) and math.isclose(r["frac"], 500.0 / 1400.0)
    assert math.isclose(r["hbm_frac"], 0.5e3 / 6500.0)
    assert math.isclose(r["intensity_flop_per_byte"], 1000.0)
    assert math.isclose(r["flops_per_launch"], 1e14) and math.isclose(r["bytes_per_launch"], 1e11)
    assert r["traffic"] is None                       # no capture for this workload


def test_low_intensity_scope_is_bound_by_hbm_and_carries_measured_traffic():
    # 10 FLOP/B: HBM-bound; 1.3e12 B in 1 s = 1300 GB/s
    k = scope(1000.0, 4, 1.3e13, 1.3e12)
    r = bench.scope_roofline("ch_attention", k, "bf16", "large_52q_tf128x4", CEIL)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6500.0
    assert math.isclose(r["achieved"], 1300.0) and math.isclose(r["frac"], 0.2)
    ratio = bench.NCU_TRAFFIC[("large_52q_tf128x4", "bf16", "ch_attention")]
    assert math.isclose(r["traffic"], ratio * 1.3e12 / 4)


def test_fp32_form_uses_the_ffma_ceiling():
    r = bench.scope_roofline("tf_mlp", scope(1000.0, 1, 3e13, 1e10), "fp32", "w", CEIL)
    assert r["bound"] == "alu" and math.isclose(r["frac"], 30.0 / 75.0)


def test_scopes_without_work_or_kernel_are_skipped():
    assert bench.scope_roofline("tf_mlp", scope(1.0, 1, 0.0, 0.0), "bf16", "w", CEIL) is None
    assert bench.scope_roofline("not_a_scope", scope(1.0, 1, 1.0, 1.0), "bf16", "w", CEIL) is None
    assert bench.scope_roofline("tf_mlp", scope(0.0, 1, 1.0, 1.0), "bf16", "w", CEIL) is None


def test_dominant_scope_is_the_slowest_per_step():
    rl = {"a": {"ms_per_step": 1.0, "frac": 0.9}, "b": {"ms_per_step": 3.0, "frac": 0.2},
          "c": {"ms_per_step": 2.0, "frac": 0.5}}
    top = bench.dominant_roofline(rl)
    assert top["scope"] == "b" and top["frac"] == 0.2 and "note" in top
    assert "scope" not in rl["b"]                     # the per-scope table is not modified
    assert bench.dominant_roofline({}) is None


def test_traffic_ratios_name_profiled_scopes():
    for (_, prec, name), ratio in bench.NCU_TRAFFIC.items():
        assert name in bench.SCOPE_KERNELS and prec in ("bf16", "fp32")
        assert 0.3 < ratio < 3.0
