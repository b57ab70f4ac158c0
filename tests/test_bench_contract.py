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
    b2, f2 = bench.axis_kernel_model(512, 512, 3, 4)
    assert b2 == 2 * 3 * 257 * 512 * 2 * 4 and f2 > 0
    b3, f3 = bench.axis_kernel_model(64, 64, 6, 4, 64)
    assert b3 == 2 * 6 * 33 * 64 * 64 * 2 * 4 and f3 != f3      # 3D: flops not modelled (NaN)
