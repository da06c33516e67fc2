"""Seeded training data for the learned per-pixel confidence weight.

Frames of seeded analytic rooms (the Kinect-like sequence generator with
other seeds) carry both the measured depth and the exact depth, so each pixel
gets a label: 1 when the measurement lies within two standard deviations of
the sensor model around the truth and is not a flying pixel, else 0.  Half of
the sampled pixels are drawn uniformly from the valid pixels, half from the
valid pixels within three pixels of a depth edge, where flying pixels live.
"""

from __future__ import annotations

import numpy as np

from .scenes import depth_edges, kinect_workload, sensor_sigma


def training_frames(n_scenes=4, frames_per_scene=3, seed=1000):
    out = []
    for sc in range(n_scenes):
        w = kinect_workload(seed=seed + sc)
        for k in np.linspace(0, w.n_frames - 1, frames_per_scene).astype(int):
            out.append((w, w.frame(int(k))))
    return out


def pixel_labels(frame):
    """(labels float32 [H, W], valid bool [H, W])."""
    d = frame.depth.astype(np.float64)
    t = frame.depth_true
    valid = (d > 0) & (t > 0)
    good = valid & (np.abs(d - t) <= 2.0 * sensor_sigma(t)) & ~frame.flying
    return good.astype(np.float32), valid


def sample_pixels(frame, n, rng):
    """n linear pixel indices of one frame, half near depth edges."""
    from scipy import ndimage
    _, valid = pixel_labels(frame)
    near = ndimage.binary_dilation(depth_edges(frame.depth_true), iterations=3) & valid
    all_idx = np.flatnonzero(valid)
    near_idx = np.flatnonzero(near)
    half = n // 2 if near_idx.size else 0
    a = rng.choice(all_idx, size=n - half, replace=all_idx.size < n - half)
    b = rng.choice(near_idx, size=half, replace=near_idx.size < half) if half else np.zeros(0, np.int64)
    return np.concatenate([a, b]).astype(np.int32)
