"""bench.py's host-side helpers (CPU): the committed traffic is reported only
while the integration source matches the captured one, the roofline peak
comes from the measured file (else the stated fallback), and throughput is
the whole job's units over the slowest rank's time."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_traffic_follows_the_integration_source(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "integrate_kinect_traffic.json")) as f:
        d = json.load(f)
    want = (d["dram_bytes_per_launch_mean"], d["frames"], d["traffic_over_algorithmic"])
    if d["integrate_source_sha256_16"] == bench.integrate_source_hash():
        assert bench.committed_traffic() == want and want[0] > 0
    else:  # the kernel changed since the capture: no traffic is reported
        assert bench.committed_traffic() is None
    monkeypatch.setattr(bench, "integrate_source_hash", lambda: d["integrate_source_sha256_16"])
    assert bench.committed_traffic() == want
    monkeypatch.setattr(bench, "integrate_source_hash", lambda: "0" * 16)
    assert bench.committed_traffic() is None


def test_committed_traffic_pairs_the_same_frames():
    """The summary's ratio is DRAM bytes over the algorithmic bytes of the
    same launches: the bench's default timed frames (warm-up 5, 20 steps)."""
    with open(os.path.join(ROOT, "profiles", "integrate_kinect_traffic.json")) as f:
        d = json.load(f)
    assert d["frames"] == [5, 24] and d["captured_launches"] == 20
    assert abs(d["dram_bytes_per_launch_mean"] / d["algorithmic_bytes_per_launch_same_frames"]
               - d["traffic_over_algorithmic"]) < 1e-3


def test_peak_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6781.4, "bf16_tflops": 1900.0}))
    assert bench.load_peaks() == (6781.4, "measured")


def test_job_throughput_counts_all_ranks_over_the_slowest():
    assert bench.job_throughput(290, 1, 58.0) == 290 / 0.058
    assert bench.job_throughput(290, 4, 60.0) == 4 * 290 / 0.060


def test_frames_jsonl(tmp_path):
    import json
    import numpy as np
    import bench
    p = tmp_path / "f.jsonl"
    bench.write_frames_jsonl(str(p), [10, 11], np.array([[0.05, 0.03, 0.1], [0.06, 0.02, 0.2]]))
    rows = [json.loads(l) for l in p.read_text().splitlines()]
    assert rows == [{"frame": 10, "u16_to_f32_and_allocate_ms": 0.05, "integrate_ms": 0.03, "raycast_ms": 0.1},
                    {"frame": 11, "u16_to_f32_and_allocate_ms": 0.06, "integrate_ms": 0.02, "raycast_ms": 0.2}]
