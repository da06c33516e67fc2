"""The seeded synthetic inputs follow the stated recipe (CPU).

The paper has no public benchmark; seeded analytic scenes stand in for its
Kinect-style sequences.  These checks keep the generators to the recipe the
design notes state: image sizes, intrinsics and scene parameters of the three
configurations; frames reproducible from the seed; the room trajectory's speed
and turn-rate limits and its distance from the walls; the sensor model (noise
level against the stated sigma(z), flying pixels only on depth edges and at
the stated fraction capped by the edge count, depth range, the float frame equal to the millimetre
frame / 1000).
"""

import numpy as np

from synth import kinect_workload, large_workload, tiny_workload
from synth.scenes import depth_edges, sensor_sigma


def test_configurations():
    t, k, l = tiny_workload(), kinect_workload(n_frames=5), large_workload(n_frames=5)
    assert (t.intr.width, t.intr.height, t.intr.fx, t.intr.cx, t.intr.cy) == (160, 120, 140.0, 80.0, 60.0)
    assert (k.intr.width, k.intr.height, k.intr.fx, k.intr.cx, k.intr.cy) == (640, 480, 525.0, 319.5, 239.5)
    assert (l.intr.width, l.intr.height, l.intr.fx) == (640, 480, 525.0)
    assert t.params == dict(voxel_size=0.01, mu=0.04, max_w=100, num_buckets=1 << 16, num_excess=1 << 14,
                            num_blocks=1 << 16, z_min=0.2, z_max=5.0)
    assert k.params == dict(voxel_size=0.005, mu=0.02, max_w=100, num_buckets=1 << 20, num_excess=1 << 17,
                            num_blocks=1 << 19, z_min=0.4, z_max=5.0)
    assert l.params["voxel_size"] == 0.002 and l.params["mu"] == 0.01 and l.params["num_blocks"] == 1 << 21
    assert t.n_frames == 10 and kinect_workload().n_frames == 300 and large_workload().n_frames == 1000


def test_frames_reproducible_from_the_seed():
    a, b, c = kinect_workload(seed=3, n_frames=20), kinect_workload(seed=3, n_frames=20), kinect_workload(seed=4)
    fa, fb, fc = a.frame(7), b.frame(7), c.frame(7)
    assert np.array_equal(fa.depth_u16, fb.depth_u16) and np.array_equal(fa.T_wc, fb.T_wc)
    assert not np.array_equal(fa.T_wc, fc.T_wc)


def test_room_trajectory_limits():
    """Speed <= 0.5 m/s and turn rate <= 30 deg/s at 30 fps; camera at least
    0.5 m from the walls of the 4 x 3 x 2.5 m room."""
    w = kinect_workload(seed=0)
    T = np.stack([w.pose(k) for k in range(w.n_frames)]).astype(np.float64)
    p = T[:, :3, 3]
    speed = np.linalg.norm(np.diff(p, axis=0), axis=1) * 30.0
    assert speed.max() <= 0.5 * 1.02
    R = T[:, :3, :3]
    cosang = np.clip((np.einsum("kij,kij->k", R[:-1], R[1:]) - 1.0) / 2.0, -1.0, 1.0)
    turn = np.degrees(np.arccos(cosang)) * 30.0
    assert turn.max() <= 30.0 * 1.05
    lo, hi = np.array([-2.0, 0.0, -1.5]), np.array([2.0, 2.5, 1.5])
    assert np.all(p - lo >= 0.5 - 1e-9) and np.all(hi - p >= 0.5 - 1e-9)


def test_sensor_model():
    w = kinect_workload(seed=1, n_frames=40)
    resid, sig = [], []
    for k in (0, 13, 27):
        f = w.frame(k)
        assert np.array_equal(f.depth, (f.depth_u16.astype(np.float64) / 1000.0).astype(np.float32))
        d = f.depth_u16.astype(np.float64) / 1000.0
        valid = d > 0
        assert np.all((d[valid] >= 0.4 - 5e-4) & (d[valid] <= 5.0 + 5e-4))
        assert not np.any(f.flying & ~depth_edges(f.depth_true))
        # 1% of the valid pixels, capped by the number of edge pixels; a few
        # may then fall outside the depth range
        want = min(round(0.01 * int((f.depth_true > 0).sum())), int(depth_edges(f.depth_true).sum()))
        assert 0.9 * want <= int(f.flying.sum()) <= want
        m = valid & ~f.flying & (f.depth_true > 0)
        resid.append(d[m] - f.depth_true[m])
        sig.append(sensor_sigma(f.depth_true[m]))
    r, s = np.concatenate(resid), np.concatenate(sig)
    z = r / np.sqrt(s ** 2 + (0.001 ** 2) / 12.0)  # the millimetre quantisation adds 1/12 mm^2
    assert abs(float(np.mean(z))) < 0.02 and abs(float(np.std(z)) - 1.0) < 0.03
