"""The benchmark's reference arm (the oracle timed on the host cores) runs
without a GPU: its one JSON line follows the contract of the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--oracle-rows", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    b = json.loads(lines[0])
    assert b["impl"] == "reference"
    assert b["metric"].startswith("GF(p) GEMM effective 2mnk/s")
    assert b["unit"] == "T(2mnk)/s" and b["higher_is_better"] is True
    assert b["value"] > 0 and b["ms_per_step"] > 0
    assert b["n_gpus"] == 1 and b["steps"] == 1 and b["warmup"] >= 3
    assert b["config"]["workload"] and b["config"]["m"] == b["config"]["k"] == b["config"]["n"] == 16384
    assert b["config"]["p"] == 5
    cb = b["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == b["value"] and cb["sample"]
    assert b["e2e"] == {"value": b["value"], "unit": b["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
