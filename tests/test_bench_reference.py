"""The bench's reference arm on the CPU: `bench.py --impl reference` times the oracle as it
stands on a bounded sample of the headline workload and prints one JSON line in the bench
contract (no GPU involved)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "particles/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert abs(d["ms_per_step"] - d["sample"]["N"] / d["value"] * 1e3) < 1e-6 * d["ms_per_step"]
    # the same workload as the GPU arm's default line, timed on a bounded sample of it
    assert d["config"]["workload"].startswith("plummer") and d["config"]["N"] == 1 << 20
    assert d["config"]["p"] == 4 and d["config"]["theta"] == 0.6 and d["config"]["leaf_size"] == 32
    assert 0 < d["sample"]["N"] < d["config"]["N"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
