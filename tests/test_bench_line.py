"""bench.py's printed line on CPU: from a full record of the shape run_gpu builds (synthetic values),
compact_line keeps every key of the benchmark contract, the roofline of the dominant kernel, the CPU
baseline and the comparison numbers, stays valid JSON, and stays short enough that the last lines of
the output hold it whole."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CONTRACT = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "clocks", "e2e", "gpu_launches")


def _record():
    prof = {c: {"ms_per_step": 1.0 + i, "launches_per_step": 3.0, "share_of_kernel_time": 0.05}
            for i, c in enumerate(("residual", "outer_op64", "outer_op32", "mg_op0_picard", "smooth", "krylov_vec",
                                   "filter", "mg_stencil", "mg_stencil_l1", "mg_setup_fine"))}
    roof = {"bound": "alu", "kernel_class": "residual", "arith": "fp64", "achieved": 0.84, "peak": 1.259,
            "unit": "TFLOP/s", "frac": 0.667, "traffic": 110.5e6, "per_launch_us": 1567.0, "launches": 15,
            "timed": "x"}
    return {
        "metric": "state solves/s at 128^3", "value": 33.7, "unit": "solves/s", "n_gpus": 1, "steps": 5,
        "warmup": 3, "ms_per_step": 29.7, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64", "data": "synthetic", "config": {"workload": "128^3", "grid": [128, 128, 128]},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3},
        "e2e": {"value": 33.0, "unit": "solves/s", "h2d_bytes_per_step": 16777216, "d2h_bytes_per_step": 16777224},
        "gpu_launches": 6265, "roofline": roof,
        "roofline_level0": dict(roof, bound="hbm", kernel_class="mg_op0_picard", unit="GB/s"),
        "cpu_baseline": {"value": 6e-4, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": "s"},
        "solver": {"newton_its": [3] * 5, "krylov_its": [15] * 5, "adjoint_krylov_its": [14] * 5,
                   "rel_residual": [9e-10] * 5},
        "kernel_time_share_warmup": prof,
        "rooflines_warmup": {c: dict(roof, bound="hbm" if i % 2 else "alu", frac=0.1 * i)
                             for i, c in enumerate(prof)},
        "fp64_path": {"value": 2.5, "ms_per_step": 397.0, "newton_its": [3], "krylov_its": [16],
                      "rel_residual": [2e-10]},
        "mixed_fast": {"value": 41.6, "ms_per_step": 24.0, "krylov_its": [14, 14]},
        "concurrent": {"in_flight": 2, "value": 40.0},
        "cavity": [{"alpha": 1e3, "settings": {}, "ms_per_state_solve": 26.1, "newton_its": [4], "krylov_its": [21],
                    "ms_adjoint": 9.0, "adjoint_krylov_its": 14},
                   {"alpha": 1e6, "settings": {"mg_smoother": 1}, "ms_per_state_solve": 69.9, "newton_its": [7],
                    "krylov_its": [78], "ms_adjoint": 22.6, "adjoint_krylov_its": 32}],
        "serving": {"requests": 300, "errors": 0, "p50_ms": 20.0, "p99_ms": 45.8, "requests_per_s": 20.3,
                    "state_solves_per_s": 20.3, "adjoint_solves_per_s": 10.2, "slots": 6, "peak_pool_gb": 8.8,
                    "latencies_ms": list(range(300))},
    }


def test_compact_line_keeps_the_contract_and_stays_short():
    sys.path.insert(0, ROOT)
    import bench
    out = bench.compact_line(_record())
    text = json.dumps(out)
    back = json.loads(text)
    for k in CONTRACT:
        assert k in back
    for k in ("roofline", "roofline_level0", "cpu_baseline", "fp64_path", "mixed_fast", "concurrent", "cavity",
              "serving", "mixed_over_fp64"):
        assert k in back
    assert back["roofline"]["frac"] == 0.667 and back["roofline"]["traffic"] == 110.5e6
    assert back["cavity"][1]["smoother"] == "zline" and back["cavity"][0]["smoother"] == "jacobi"
    assert "latencies_ms" not in back["serving"]          # per-request data stays out of the line
    assert len(text) < 4000
    # the comparison numbers come last
    keys = list(back)
    assert keys.index("serving") > keys.index("roofline") and keys.index("cavity") > keys.index("cpu_baseline")
