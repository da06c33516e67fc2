"""bench.py's reference arm (the CPU oracle) keeps the bench's JSON contract.

Runs on the CPU: `--impl reference` on the tiny workload, one JSON line with
the arm's metric and unit for that workload, a positive value, and the
cpu_baseline and e2e objects the contract asks for.
"""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_on_the_tiny_workload():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "3", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    n_frames, desc, metric = bench.WORKLOADS["tiny"]
    assert d["impl"] == "reference" and d["metric"] == metric and d["unit"] == "frames/s"
    assert d["config"]["workload"] == desc
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["voxel_updates_per_s"] > 0
