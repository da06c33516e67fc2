"""Seeded layout of the batched workload: rigid submaps and many small scenes.

* 16 submaps of the Kinect room sequence (seed 0), each with its own hash
  size between 2^16 and 2^20 buckets and a world-from-submap pose rotated by
  up to 15 degrees and offset by up to 0.5 m; every frame goes to 1-3 active
  submaps (a primary one that advances along the sequence, plus neighbours).
* 64 independent rooms (seeds 100..163) at uneven resolutions (80x60 to
  640x480, same field of view) and voxel sizes (5-20 mm, mu = 4 voxels).
"""

from __future__ import annotations

import numpy as np

from .scenes import kinect_workload

RESOLUTIONS = [(80, 60), (160, 120), (320, 240), (640, 480)]


def submap_poses(n, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        a = np.radians(rng.uniform(0, 15))
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        R = np.eye(3) + np.sin(a) * K + (1 - np.cos(a)) * K @ K
        P = np.eye(4)
        P[:3, :3] = R
        t = rng.normal(size=3)
        P[:3, 3] = t / np.linalg.norm(t) * rng.uniform(0, 0.5)
        out.append(P)
    return out


def submaps(n=16, seed=0):
    """(workload of the shared sequence, [(params, world_from_submap)])."""
    rng = np.random.default_rng([seed, 21])
    w = kinect_workload(seed=seed)
    out = []
    for P in submap_poses(n, seed=seed + 3):
        nb = 1 << int(rng.integers(16, 21))
        out.append((dict(w.params, num_buckets=nb, num_excess=1 << 16, num_blocks=1 << 17), P))
    return w, out


def active_submaps(k, n=16, seed=0):
    """1-3 submaps that frame k is fused into."""
    rng = np.random.default_rng([seed, 22, k])
    primary = (k // 19) % n
    extra = int(rng.integers(0, 3))
    return [(primary + j) % n for j in range(extra + 1)]


def small_scenes(n=64, seed=100):
    """Workloads of n independent rooms at uneven resolutions and voxel sizes."""
    rng = np.random.default_rng([seed, 23])
    out = []
    for i in range(n):
        W, H = RESOLUTIONS[int(rng.integers(0, len(RESOLUTIONS)))]
        vs = float(np.round(rng.uniform(0.005, 0.020), 4))
        nb = 1 << (16 if W <= 160 else 17 if W == 320 else 18)
        nv = 1 << (15 if W <= 160 else 16 if W == 320 else 17)
        p = dict(voxel_size=vs, mu=4 * vs, num_buckets=nb, num_excess=1 << 15, num_blocks=nv)
        out.append(kinect_workload(seed=seed + i, width=W, height=H, params=p))
    return out
