"""The benchmark's reference arm on the host, no GPU: ``bench.py --impl
reference`` times the FP64 oracle per step on a bounded sample of the
2048x1024 workload's medium and prints one JSON line with the keys the
benchmark contract fixes (metric, value, unit, impl, the CPU baseline it
describes, and an end-to-end record with no host-device copies)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("2-comp D2Q9 MLUPS") and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == "MLUPS"
    assert cb["cores"] >= 1 and "2048x" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == "MLUPS"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["nx"] == 2048 and 16 <= d["config"]["ny"] <= 1024
    # the per-step time and the throughput describe the same sample
    nodes = d["config"]["nx"] * d["config"]["ny"]
    assert abs(nodes / (d["ms_per_step"] * 1e-3) / 1e6 - d["value"]) <= 0.02 * d["value"]
