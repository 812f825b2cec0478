"""The benchmark's last stdout line stays small and carries every key of the contract.

A reader of the output sees only its tail, so the final JSON line must be short
whatever the run measured: tuner trials, filter tables and the other workloads'
sections go to the detail file, and the line keeps one digest of each.  The
detail below has the shape of a full default run (every section present, the
tuner lists at their real lengths).
"""
import json
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _clocks():
    return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 60}


def _prec(ms, frac):
    return {"value": 1.81e9 / (ms * 1e-3), "ms_per_step": ms, "speedup_vs_f64": 542.0 / ms,
            "err_col": 3.3e-3, "err_elem": 1.1e-2, "clocks": _clocks(), "gpu_launches": 180,
            "roofline": {"bound": "hbm", "frac": frac, "achieved": 100.0, "peak": 6789.6, "unit": "GB/s",
                         "tune_ms_per_config": [1.0] * 7}}


def _full_detail():
    trials = [{"threads": 512, "blocks_per_sm": 2, "tile_f64": 0, "tile_f32": 1, "cells_per_item": 2,
               "ms": 5.998}] * 62
    batched = {"ms_per_step": 161.6, "speedup_vs_separate": 0.9, "tuning_trials": trials, "value": 1e10,
               "one_launch_per_system": {"ms_per_step": 144.7}}
    flt = {p: {"lanczos_ms": 95.0, "rayleigh_ritz_ms": 694.0, "filter_ms": 851.0, "pass_ms": 1640.0}
           for p in ("f64", "f64_pairs", "mixed", "mixed_bf16", "mixed_f16", "mixed_bf16x2")}
    flt.update({"speedup_filter_mixed_vs_f64": 13.1, "speedup_pass_mixed_vs_f64": 8.8,
                "f64_apply_ms_by_n_v": {1: 3.0, 8: 20.0, 64: 140.0},
                "converged": {"workload": "24^3 cells, p=8, N_v=256, lowest 240 to residual 1e-9",
                              "passes_f64": 31, "passes_mixed": 32, "speedup": 7.7,
                              "max_eig_diff_Ha": 3e-12, "max_residual": 8e-10},
                "converged_6cubed": {"speedup": 3.6, "max_eig_diff_mixed_vs_f64_Ha": 4.7e-14,
                                     "generalised_consistent_mass": {"f64": {"ms": 1.0}}}})
    return {
        "f64": {"value": 3.34e9, "ms_per_step": 542.0, "clocks": _clocks(), "gpu_launches": 180,
                "roofline": {"bound": "alu", "achieved": 0.8, "peak": 1.25, "unit": "TFLOP/s", "frac": 0.64,
                             "traffic": 7.9e9, "kernel": "fe_local_kernel (FP64 DFMA pipe)",
                             "peak_source": "nominal FP64 1.25 TFLOP/s; live DFMA probe 1.251 TFLOP/s",
                             "frac_of_live_probe": 0.64, "avg_launch_ms": 65.4, "tile_config": 1,
                             "tune_ms_per_config": [600.0] * 7}},
        "f64_pairs_of_fp32": {"value": 1e10, "ms_per_step": 178.0, "speedup_vs_f64": 3.05, "err_col": 1e-14,
                              "err_elem": 2e-14, "frac_of_nominal_fp64": 1.9, "tune_ms_per_config": [1.0] * 7},
        "f32": _prec(26.5, 0.21), "bf16_tensor_core": _prec(28.3, 0.077), "f16_tensor_core": _prec(29.7, 0.074),
        "bf16x2_tensor_core": _prec(40.0, 0.05),
        "e2e": {"value": 3.09e9, "unit": bench.UNIT, "h2d_bytes_per_step": 14495514624,
                "d2h_bytes_per_step": 14495514624, "ms_per_step": 587.0, "steps": 10,
                "one_step_serial_ms": {"h2d": 69.0, "apply": 542.0, "d2h": 75.0}},
        "cpu_baseline": {"value": 3.06e5, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                         "sample": "36 of 13824 cells in 15.1 s (cell-matrix method: H^(e) by quadrature then "
                                   "H^(e) X^(e), local terms, all 256 vectors), scaled to the whole operator"},
        "filter": flt,
        "batched": batched, "batched_small_systems": dict(batched, ms_per_step=1.6, speedup_vs_separate=4.15),
        "all_electron_like": {k: {"ms_per_step": 10.0} for k in ("f64", "f32", "bf16_tensor_core")},
        "cell_matrix_baseline": {"f64": {"ms_per_step": 3537.0, "tune": trials}},
        "quadrature_n_p_plus_2": {"f64": {"ms_per_step": 960.0, "tune_ms_per_config": [1.0] * 7}},
    }


def _config():
    return {"workload": "C4: L=30 bohr, 24^3 cells, p=8, n_q=9, N_v=256, real, GGA=True, atoms=64",
            "n_dofs": 7077888, "n_v": 256, "degree": 8, "n_q": 9,
            "l2": "inputs larger than L2 (X = 14.5 GB), no flush", "parallelism": "replicas x1"}


def test_final_line_is_compact_and_complete():
    args = types.SimpleNamespace(steps=20, warmup=5)
    line = bench.compact_line(_full_detail(), args, _config(), 1)
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) < 3000, len(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "gpu_launches",
                "e2e", "cpu_baseline"):
        assert key in line, key
    assert line["value"] > 0 and line["dtype"] == "f64"
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in line["roofline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in line["e2e"], key
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in line["cpu_baseline"], key
    assert set(line["precisions"]) >= {"f64_pairs", "f32", "bf16_tc", "f16_tc"}
    assert line["precisions"]["bf16_tc"]["err_col"] == 3.3e-3
    assert line["filter"]["converged"]["speedup"] == 7.7
    assert line["batched_c5"]["x_separate"] == 0.9
    assert json.loads(text) == line


def test_minimal_run_line():
    """A run with every optional section switched off still prints the contract's keys."""
    d = _full_detail()
    d = {"f64": d["f64"]}
    line = bench.compact_line(d, types.SimpleNamespace(steps=3, warmup=3), _config(), 1)
    assert "precisions" not in line and "filter" not in line
    assert line["roofline"]["frac"] == 0.64
