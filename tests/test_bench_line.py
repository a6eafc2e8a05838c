"""The benchmark line's short forms (host logic, no device): the compact
sections carry the keys the record needs, figures are rounded to four
significant digits, and the sections stay within a couple of kilobytes."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def serve_row(p50, p99, batch=1.0):
    return {"p50_ms": p50, "p99_ms": p99, "mean_batch": batch, "submit_lag_max_ms": 0.5}


def fake_extra():
    uneven = {"value": 1.603e8, "ms_per_solve": 43.75, "threads": 384, "launches_per_solve": 3.0,
              "one_launch_per_problem": {"value": 1.197e8, "ms_per_solve": 58.58},
              "bf16": {"value": 1.641e8, "ms_per_solve": 42.74},
              "auto": {"value": 2.409e8, "ms_per_solve": 29.12, "warp_slots_cap": 7,
                       "frac_of_fp32_peak": 0.63321234, "frac_finer_count": 0.46812345}}
    precision = {k: {"value": v, "coef_dev_vs_fp32_after_10": {"max": 1e-2, "median": 1e-3}}
                 for k, v in (("tf32", 2.1e8), ("bf16", 2.1e8), ("split_bf16", 2.0e8), ("fp32_warp_pair", 3.56e8))}
    precision["fp32"] = {"value": 2.07e8}
    precision["workload"] = "text"
    large = {f"B={b}": {"large": {"value": 4.1e8, "kernel_ms": 3.97, "frac_of_fp32_peak": 0.7},
                        "small_tile": {"value": 2.0e8}, "warp_pair": {"value": 4.0e8}} for b in (16384, 18944)}
    large["profile"] = {"tensor_pipe_pct": 10.6, "traffic": 8596224}
    serving = {"batched": serve_row(0.56, 1.2), "sequential_fused": serve_row(0.57, 1.4),
               "batched_auto": serve_row(0.43, 0.9), "sequential_auto": serve_row(0.44, 1.0),
               "sequential_plain_fp32_loop": serve_row(1272.0, 1916.0),
               "high_load": {"offered_per_s": 2500.0, "runs": 3,
                             **{k: [serve_row(0.6, 3.0 + r, 1.5) for r in range(3)]
                                for k in ("batched", "sequential_fused", "batched_auto", "sequential_auto")}}}
    return {"uneven": uneven, "precision": precision, "large": large, "serving": serving}


def test_summary_sections_keys_and_size():
    out = bench.compact(bench.summary_sections(fake_extra()))
    u = out["uneven"]
    assert u["auto_value"] == 2.409e8 and u["auto_slots_cap"] == 7
    assert u["auto_frac"] == 0.6332 and u["auto_frac_finer"] == 0.4681  # four significant digits
    assert set(out["precision_b4096"]) == {"fp32", "tf32", "bf16", "split_bf16", "fp32_warp_pair"}
    assert out["large_batch"]["profile"]["tensor_pipe_pct"] == 10.6
    s = out["serving_p50_p99_ms"]
    assert s["400/s"]["batched_auto"] == [0.43, 0.9]
    assert s["2500/s"]["seq_auto"] == [[0.6, 0.6, 0.6], [3.0, 4.0, 5.0]]
    assert out["serving_mean_batch"]["2500/s"] == [1.5, 1.5, 1.5]
    assert out["serving_submit_lag_max_ms"] == 0.5
    assert len(json.dumps(out)) < 2000


def test_sig_rounds_and_passes_other_values():
    assert bench.sig(123456.789) == 123500.0 and bench.sig(0.000123456) == 0.0001235
    assert bench.sig(None) is None and bench.sig(True) is True and bench.sig(0) == 0
