"""bench.py's output contract on CPU: the last stdout line is one compact JSON
object that a driver keeping only the tail of the output can parse (at most
2 KB, the headline keys present), built from a complete record whose legs and
kernel tables are far larger; and the per-result backward-error helper that
the line reports (zero on an exact factor, large when an entry is wrong)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1305_2353_gb300 import inputs  # noqa: E402


def _fake_record():
    kern = {f"kernel_with_a_long_name_{i}": (3, 1.2345678 * i) for i in range(40)}
    roof = {"kernel": "form_fp64", "bound": "alu", "achieved": 1.2491, "peak": 1.17, "unit": "TFLOP/s",
            "frac": 1.0676, "traffic": 1.717e11, "peak_source": "measured in this run: torch.matmul "
            "float64 6144^3, best of 10" * 3, "work_per_launch": 1.02e13, "launch_ms": 8179.0,
            "alu_peak": 1.2586, "frac_of_alu_peak": 0.9925}
    err = {"factor": {"raw": 1.2e-12, "growth_normalised": 3.4e-17, "growth": 1.7e4},
           "form": {"entries_sampled": 4096, "max_rel_to_scale": 2.2e-16}, "a21_rows_sampled": 2049}
    main = {"value": 1247.61234567, "ms": 3 * 8197.123, "e": 256, "roofline": roof, "errors": err,
            "e2e": {"value": 1229.1, "unit": "GFLOP/s", "h2d_bytes_per_step": 409600000,
                    "d2h_bytes_per_step": 409606148},
            "launches": 15, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 99},
            "kern": kern, "kernels": kern}
    mixed = {"value": 347000.0, "ms_per_step": 29.45, "roofline": {"frac": 0.66, "hbm_frac": 0.48},
             "errors": err, "kernels": kern, "autotune": {"candidates_ms": {str(i): 1.0 for i in range(50)}}}
    batch = {k: {"ms_per_batch": v, "accuracy": {"max_bwd_err": 8.8e-15, "max_corrections": 3},
                 "kernels": kern} for k, v in (("fp64", 60.7), ("mixed", 42.2))}
    return {"metric": "Supernode LDL^T GFLOP/s", "n_gpus": 1, "steps": 3, "warmup": 3, "dtype": "f64",
            "config": {"workload": bench.workload_name(bench.parse_args([])), "n": 200000, "p": 256,
                       "u": 0.01, "pivot": "relaxed", "prec": "fp64", "solve": "fp64", "S": "fp64_packed",
                       "nelim": 256, "flops_per_step": 10227000000000, "l2": "inputs larger than L2",
                       "parallelism": "replicas x1"},
            "main": main, "mixed": mixed, "batch": batch,
            "cpu_baseline": {"value": 2.63, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": "oracle factor+solve on the first 20000 A21 rows " * 5},
            "multifrontal": {"kernels": kern}, "complete_system": {"kernels": kern}}


def test_headline_is_compact_and_complete():
    rec = _fake_record()
    assert len(json.dumps(rec, default=str)) > 8000      # the full record is large
    s = bench.headline(rec)
    assert len(s) <= 2000
    line = json.loads(s)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in line, k
    assert line["config"]["workload"].startswith("single supernode n=200000 p=256")
    assert line["roofline"]["bound"] == "alu" and 0 < line["roofline"]["frac"]
    assert line["cpu_baseline"]["cores"] == 1
    assert line["config"]["batch_8192_mixed_vs_fp64"]["speedup"] > 1
    assert "\n" not in s


def test_parse_args_defaults():
    a = bench.parse_args([])
    assert (a.gpus, a.n, a.p, a.pivot, a.prec) == (1, 200000, 256, "relaxed", "fp64")
    assert a.full_out.endswith("bench_full.json")


def test_factor_errors_exact_and_planted():
    """The backward-error helper on the oracle's factor (FP64 rounding only) and
    on the same factor with one planted wrong entry of L21."""
    A = inputs.supernode(300, 24, seed=3)
    for method in ("strict", "relaxed", "tpp"):
        r = O.factor(A, 24, method)
        rows = np.arange(276)
        ok = bench.factor_errors(A, r["A"], r["perm"], r["piv"], r["D"], r["nelim"], 24, rows)
        assert ok["growth_normalised"] < 1e-14 and ok["raw"] < 1e-12
        bad = r["A"].copy()
        bad[24 + 100, 0] += 1e-6
        b = bench.factor_errors(A, bad, r["perm"], r["piv"], r["D"], r["nelim"], 24, rows)
        assert b["raw"] > 1e-8


def test_s_index_layouts():
    m = 300
    # packed: column j starts after the lengths of columns 0..j-1
    assert bench.s_index(0, 0, m, "fp64_packed") == 0
    assert bench.s_index(m - 1, 0, m, "fp64_packed") == m - 1
    assert bench.s_index(1, 1, m, "fp64_packed") == m
    # tiled: 128 x 128 blocks of the lower block triangle, column-major inside
    nb = 3
    assert bench.s_index(0, 0, m, "fp32_tiled") == 0
    assert bench.s_index(128, 0, m, "fp32_tiled") == 16384
    assert bench.s_index(128, 128, m, "fp32_tiled") == 16384 * nb
    assert bench.s_index(5, 3, m, "fp32_tiled") == 3 * 128 + 5
