"""The bench's headline line: compact (the driver keeps only a tail of stdout), with the
top-level value and step time at full precision, and the same config on both arms."""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line():
    """A headline line of the full shape, every field filled, floats at full width."""
    args = argparse.Namespace(precision="f16", resampler="systematic")
    f = 1.0 / 3.0
    return {
        "metric": bench.METRIC, "value": 42247914167.38247, "unit": bench.METRIC, "n_gpus": 1, "steps": 200,
        "warmup": 3, "ms_per_step": 2.481959217786789, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic", "config": bench._config(args, 1),
        "roofline": {"bound": "hbm", "achieved": 844.9582833476494, "peak": 6795.8, "unit": "GB/s", "frac": f,
                     "traffic": 6428928.0, "kernel": "step_kernel<f16>", "peak_source": "measured",
                     "bytes_per_particle_step": 20, "launch_us": 24.81959217786789, "fused_frac": f},
        "roofline_issue": {"bound": "alu", "frac": f, "instructions_per_particle_step": 458.98788452148},
        "e2e": {"value": 38289633123.92059, "unit": bench.METRIC, "h2d_bytes_per_step": 26214400,
                "d2h_bytes_per_step": 1600},
        "gpu_launches": 20000,
        "accuracy": {"rmse_px_vs_ref64_gpu": f, "rmse_px_vs_ground_truth": f, "rmse_px_vs_oracle": f},
        "per_precision": {p: {"value": 4.1e10 + f, "us_per_frame": 24.0 + f} for p in ("ref64", "f32", "bf16", "f16")},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
        "batched": {"value": 4.2e10 + f, "us_per_frame": 350.0 + f, "autotuned_value": 4.2e10 + f, "trackers": 256},
        "serving": {"seconds": 20.0, "streams": 1024, "p50_ms": f, "p99_ms": 1.0 + f, "saturated_value": 2.3e10 + f,
                    "rejected": 0, "overloaded": {"p50_ms": 1500.0 + f, "p99_ms": 2400.0 + f, "rejected": 275,
                                                  "admitted": 749}},
        "cpu_baseline": {"value": 5.2e7 + f, "unit": bench.METRIC, "cores": 16, "kind": "oracle",
                         "sample": "whole workload (100 frames, N = 2^20), 16 threads"},
    }


def test_headline_line_is_compact_and_keeps_the_value():
    out = json.dumps(bench._rounded(_line()), separators=(",", ":"))
    assert len(out) < 2048
    back = json.loads(out)
    assert back["value"] == 42247914167.38247 and back["ms_per_step"] == 2.481959217786789
    assert back["roofline"]["frac"] == 0.33333 and back["e2e"]["value"] == 3.829e10


def test_both_arms_print_the_same_config():
    args = argparse.Namespace(precision="f16", resampler="systematic")
    assert bench._config(args, 1) == _line()["config"]
    assert bench._config(args, 1)["workload"] == bench.WORKLOAD_SHORT
