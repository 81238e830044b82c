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
    # a step is one bounded sample, timed as it ran; value is the complete oracle
    # step that sample estimates (so the timed region is steps x ms_per_step)
    assert line["ms_per_step"] > 0 and math.isfinite(line["ms_per_step"])
    assert line["config"]["workload"] == A.workload and line["vs_baseline"] is None
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _dict_keys_assigned(fn_name, var):
    """String keys of the dict literal assigned to `var` inside bench.fn_name."""
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    for node in ast.walk(tree):
        if isinstance(node, ast.FunctionDef) and node.name == fn_name:
            for sub in ast.walk(node):
                if isinstance(sub, ast.Assign) and any(isinstance(t, ast.Name) and t.id == var
                                                       for t in sub.targets) and isinstance(sub.value, ast.Dict):
                    return {k.value for k in sub.value.keys if isinstance(k, ast.Constant)}
    return set()


def test_gpu_arm_line_names_every_contract_key():
    """The GPU arm cannot run here; its JSON line is checked from the source:
    the base keys plus roofline, cpu_baseline, e2e, gpu_launches and clocks."""
    keys = _dict_keys_assigned("gpu_arm", "line")
    need = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
            "gpu_launches", "clocks"}
    assert need <= keys, need - keys


def test_roofline_object_has_the_contract_fields():
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    fn = next(n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef) and n.name == "roofline_for")
    returned = [r.value for r in ast.walk(fn) if isinstance(r, ast.Return) and isinstance(r.value, ast.Dict)]
    assert returned
    for d in returned:
        keys = {k.value for k in d.keys if isinstance(k, ast.Constant)}
        assert {"bound", "achieved", "peak", "unit", "frac"} <= keys, keys
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'smooth["traffic"] =' in src            # traffic: from the ncu summary, or null
