"""The benchmark's headline line: the last stdout line must stay short enough for a reader
that keeps only the tail of the output, and carry the contract's keys.  CPU only (the line
is built from synthetic values)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "geodesic_steps_per_s", "roofline", "cpu_baseline", "e2e",
            "gpu_launches", "clocks")


def _line(digits=17):
    x = float("0." + "3" * digits)  # long repr
    paths = ("mlp_df", "mlp", "mixed_df", "mixed", "fp64")
    return {
        "metric": bench.METRIC, "value": 5.1e7 + x, "unit": "rays/s", "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 20.5 + x, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+df64+bf16", "data": "synthetic (analytic plasma, deterministic)",
        "config": {"workload": bench.WORKLOAD, "precision": "mlp_df", "pixels": 1048576, "freqs_hz": [230e9],
                   "parallelism": "replicas x1", "l2": "flushed (256 MB write) before every timed render"},
        "geodesic_steps_per_s": 1.1e10 + x,
        "roofline": {"bound": "alu", "kernel": "mixed_fp64_long", "pipe": "fp32 (double-float)", "achieved": x,
                     "peak": 5 + x, "unit": "TFLOP/s", "frac": x, "traffic": 1958656,
                     "peak_source": "FP32 FMA-chain probe 73.5 TFLOP/s / (2 x 6.73 FP32 instr per flop, double-float)",
                     "frac_of_fp64_native": x, "counters": dict(bench.NCU_PIPES["mixed_fp64_long"])},
        "cpu_baseline": {"value": 22924.0 + x, "unit": "rays/s", "cores": 16, "kind": "oracle",
                         "sample": "16384 rays: every 8th pixel per axis of the 1024^2 image"},
        "e2e": {"value": 5e7 + x, "unit": "rays/s", "h2d_bytes_per_step": 8, "d2h_bytes_per_step": 8388616},
        "gpu_launches": 380, "clocks": {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"]},
        "rays_per_s": {p: 1e7 + x for p in paths},
        "flux_rel_err_vs_fp64": {p: x for p in paths if p != "fp64"},
        "oracle_max_rel_err_sampled": {p: x for p in paths},
        "detail": "bench_part lines above; bench_detail.json",
    }


def test_headline_line_fits_and_keeps_the_contract():
    for digits in (5, 17):
        out = bench._final_line(_line(digits))
        assert "\n" not in out
        assert len(out) <= bench.FINAL_LINE_MAX, len(out)
        d = json.loads(out)
        for k in REQUIRED:
            assert k in d, k
        assert d["config"]["workload"] == bench.WORKLOAD
        for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
            assert k in d["roofline"], k
        for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
            assert k in d["e2e"], k


def test_only_optional_keys_are_dropped():
    line = _line(17)
    line["detail"] = "x" * 3000  # too long on its own: dropping it (third) makes the line fit
    out = bench._final_line(line)
    d = json.loads(out)
    assert len(out) <= bench.FINAL_LINE_MAX
    assert "detail" not in d and "flux_rel_err_vs_fp64" in d
    assert all(k in d for k in REQUIRED)
