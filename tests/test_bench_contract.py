"""The JSON line of bench.py's reference arm (the FP64 oracle on the host
cores), checked against the bench contract on the small workload (no GPU)."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_line_has_the_contract_keys():
    import bench

    class A:
        workload = "fp64_fullbox_32x32x64"
        steps, warmup, cpu_budget, tol = 1, 0, 2.0, 1e-8

    line = bench.reference_arm(A, 0, 1)
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and math.isfinite(line["value"])
    assert abs(line["ms_per_step"] - 1e3 / line["value"]) < 1e-9 * line["ms_per_step"]
    assert line["config"]["workload"] == A.workload and line["vs_baseline"] is None
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
