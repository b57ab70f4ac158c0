"""bench.py's reference arm (the FP64 oracle on the host, no GPU) prints one JSON line with the
contract's keys, and the helpers behind the GPU line behave (no NaN in JSON, byte model)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.strip().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["warmup"] >= 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_json_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._finite({"a": float("nan"), "b": [1.0, float("inf")]}) == {"a": None, "b": [1.0, None]}
    a = {"n": 3, "E": 0.5, "G_inst": float("nan")}
    assert bench.same_result(a, dict(a)) and not bench.same_result(a, dict(a, E=0.5000000001))


def test_both_arms_name_the_same_metric_and_config():
    """The driver divides the two arms' values only when they measure the same thing."""
    sys.path.insert(0, ROOT)
    import bench
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    d = json.loads([x for x in r.stdout.strip().splitlines() if x.startswith("{")][0])
    assert d["metric"] == bench.METRIC
    assert d["config"] == bench.workload_config(bench.WORKLOAD, "fp64", "staggered", 1)


def test_roofline_of_dominant_kernel():
    """The projection instance stands for the column-pass template; the largest candidate wins."""
    sys.path.insert(0, ROOT)
    import bench
    bd = {"classes": {
        "k_axis": {"ms_per_step": 12.0, "bytes_per_launch": 4e6, "avg_launch_us": 10.0, "launches_per_step": 500,
                   "share": 0.3, "GB_s": 400.0, "TFLOP_s": 0.5},
        "k_x_fwd": {"ms_per_step": 3.0, "bytes_per_launch": 5e6, "avg_launch_us": 6.0, "launches_per_step": 500,
                    "share": 0.2, "GB_s": 800.0, "TFLOP_s": 0.4},
        "projection_pass": {"ms_per_step": 9.0, "bytes_per_launch": 6e6, "avg_launch_us": 12.0,
                            "launches_per_step": 100, "share": 0.1, "GB_s": 500.0, "TFLOP_s": 0.6},
        "fp64_residual": {"ms_per_step": 20.0, "bytes_per_launch": 6e6, "avg_launch_us": 12.0,
                          "launches_per_step": 100, "share": 0.1, "GB_s": 50.0, "TFLOP_s": 0.1}}}
    f64 = {"tflops": 1.0}
    r = bench.roofline_of(bd, "fp64", "w", 6000.0, "measured", f64)
    assert r["kernel"].startswith("k_axis<OpProj>") and r["bound"] == "alu" and abs(r["frac"] - 0.6) < 1e-12
    assert r["avg_launch_us"] == 12.0 and r["algorithmic_bytes"] == 6e6
    r = bench.roofline_of(bd, "fp32r", "w", 6000.0, "measured", f64)
    assert r["bound"] == "hbm" and abs(r["frac"] - 500.0 / 6000.0) < 1e-12 and r["traffic"] is None
    bd["classes"]["k_x_fwd"]["ms_per_step"] = 10.0
    r = bench.roofline_of(bd, "fp32r", "w", 6000.0, "measured", f64)
    assert r["kernel"] == "k_x_fwd" and abs(r["frac"] - 800.0 / 6000.0) < 1e-12
    # the CG x pass stands for its template once the library times it on its own
    bd["classes"]["cg_x_fwd"] = {"ms_per_step": 9.5, "bytes_per_launch": 9e6, "avg_launch_us": 8.0,
                                 "launches_per_step": 400, "share": 0.2, "GB_s": 1125.0, "TFLOP_s": 0.3}
    r = bench.roofline_of(bd, "fp32r", "w", 6000.0, "measured", f64)
    assert r["kernel"].startswith("k_x_fwd<ProCGCG>") and abs(r["frac"] - 1125.0 / 6000.0) < 1e-12
