"""bench.py's headline line stays compact and complete (CPU only): the default run prints one
JSON line last, and a harness that keeps only the tail of stdout must be able to parse it."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_headline_is_one_compact_json_line_with_the_contract_keys():
    per_method = {f"{m}_fp32": 8.0 + i for i, m in enumerate(("mri", "erk", "mri_adapt", "rk4"))}
    line = bench.headline(
        value=2216.5, n_gpus=1, steps=20, warmup=5, ms_per_step=9.2,
        config={"workload": bench.WORKLOAD, "step": "x" * 160, "precision": "y" * 90, "l2": "z" * 120,
                "channel_entries": 283379292, "parallelism": "replicas x1", "split_weight": 320,
                "attempts": "device-loop CUDA graph"},
        sim_ps_per_s=5.4, sim_ps_at_1e6={"value": 8.2, "method": "mri_fp32", "t_end_ps": 0.5,
                                         "reference": "FP64 sums, Zonneveld rtol 1e-9, atol 1e-15",
                                         "per_method": per_method},
        roofline={"bound": "hbm", "achieved": 5452.1, "peak": 6650.7, "unit": "GB/s", "frac": 0.82,
                  "traffic": 2333000000.0, "kernel": "rhs_kernel (full RHS: e-ph + ph-e + ph-ph)",
                  "avg_launch_ms": 0.4157, "launches_timed": 20, "alg_bytes_per_launch": 2267034336.0,
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured"},
        e2e={"value": 2190.0, "unit": bench.UNIT, "h2d_bytes_per_step": 1654000, "d2h_bytes_per_step": 1654000,
             "how": "rtbte_advance_to on a pinned host state vector (library stages it in and out per call)"},
        mri={"sim_ps_per_s": 3.7, "h_s_fs": 20.0, "rhs_fast": 300, "rhs_slow": 15},
        ensemble={"instances": 64, "instance_rhs_evals_per_s": 23000.0, "rhs_kernel_frac": 0.6,
                  "rhs_kernel_ms": 1.1},
        clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 5, "samples_how": "inside the timed region",
                "power_w_max": 1100.0, "reasons": []},
        gpu_launches=1234,
        cpu_baseline={"value": 0.0048, "unit": bench.UNIT, "cores": 16, "kind": "oracle", "sample": "s" * 300})
    assert "\n" not in line
    assert len(line) < 4096
    d = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "cpu_baseline", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] and d["roofline"]["frac"] == 0.82
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"]
