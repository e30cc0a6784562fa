"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the one-line JSON
contract: runs on CPU with a small image."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--size", "96",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600, check=True).stdout.strip().splitlines()
    lines = [l for l in out if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ns/photon/step" and d["value"] > 0
    assert d["higher_is_better"] is False and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["image"] == "96x96"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
