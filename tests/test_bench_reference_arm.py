"""bench.py --impl reference on the host: the CPU oracle timed on the GPU arm's workload prints one
JSON line with the GPU arm's metric, unit and direction, its measured step time, a cpu_baseline
describing the run (value equal to the line's) and an e2e entry that moves no bytes."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "s/k-point" and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s/k-point", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value = measured time per apply x the GPU arm's apply count per k-point
    assert d["extrapolation"]["applies_per_kpoint"] == bench.APPLIES_PER_KPOINT_MEASURED
