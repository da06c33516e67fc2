"""Pins of the oracle's colour voxels (Sec. 3.1).

The paper's voxel types with colour carry an RGB value and a colour weight;
it does not print their update.  Readings (recorded with the others in the
design notes): a voxel that gets a depth update within the band |eta| <= mu
takes the colour of its projection into the RGB image (depth camera -> colour
camera by the extrinsic map, colour intrinsics, bilinear sampling of the 2x2
pixels at the floor of the position); each channel keeps the running mean
(w c + c_obs) / (w + 1) rounded half up to 8 bits, the colour weight counting
observations up to max_w; the colour of a point (a raycast hit) is that of its
nearest voxel.  Each test checks the oracle against something other than
itself: exact closed forms of the running mean and its rounding, a linear
colour ramp whose bilinear sample is the analytic projection, an extrinsic
shift of a known number of pixels, a brute-force nearest-voxel lookup, and
the depth fusion without colour.
"""

import numpy as np
import pytest

import oracle
from synth.scenes import Intrinsics
from tests.test_oracle_pins import scene_params

INTR = Intrinsics(64, 48, 60.0, 60.0, 31.5, 23.5)
EYE = np.eye(4, dtype=np.float32)


def _plane(z=1.0):
    return np.full((INTR.height, INTR.width), z, np.float32)


def _scene(**kw):
    sc = oracle.Scene(**scene_params(**kw))
    sc.colour_enable()
    return sc


def _voxels(coords, s):
    """World positions (fp64) of every voxel of the exported blocks [n, 512, 3]."""
    l = np.arange(512)
    local = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    g = coords.astype(np.int64)[:, None, :] * 8 + local[None]
    return g.astype(np.float64) * np.float64(np.float32(s))


def _fuse(sc, rgb, frames=1, depth=None, T_d2c=None, intr_c=None):
    d = _plane() if depth is None else depth
    ia = INTR.as_array()
    for _ in range(frames):
        sc.allocate(d, ia, EYE)
        sc.integrate_colour(d, ia, EYE, rgb, ia if intr_c is None else intr_c, T_d2c)


def _band(sc, mu, margin=2e-4):
    """Exported colours, voxel positions and masks of the voxels surely inside
    the band (|1 - z| < mu - margin, projected well inside the image) and surely
    in front of it (z < 1 - mu - margin)."""
    c, C = sc.export_colour()
    P = _voxels(c, sc.params["voxel_size"])
    z = P[..., 2]
    u = INTR.fx * P[..., 0] / z + INTR.cx
    v = INTR.fy * P[..., 1] / z + INTR.cy
    inside = (u > 2) & (u < INTR.width - 3) & (v > 2) & (v < INTR.height - 3)
    band = inside & (np.abs(1.0 - z) < mu - margin)
    front = inside & (z < 1.0 - mu - margin) & (z > 0.2)
    return C, P, band, front


def test_first_observation_takes_the_colour_inside_the_band_only():
    """Blocks of a nearer plane (z = 0.9) are allocated first, so the frame of
    the plane z = 1 also updates free space in front of its surface."""
    sc = _scene()
    sc.allocate(_plane(0.9), INTR.as_array(), EYE)
    rgb = np.zeros((INTR.height, INTR.width, 3), np.uint8)
    rgb[...] = (10, 200, 77)
    _fuse(sc, rgb)
    c, F, W = sc.export()
    assert np.any((W > 0) & (F == 1.0))  # free-space voxels were updated
    C, _, band, front = _band(sc, sc.params["mu"])
    assert band.sum() > 10000 and front.sum() > 1000
    assert np.all(C[band] == (10, 200, 77, 1))
    assert np.all(C[front] == 0)  # free space in front of the surface: depth updated, no colour


def test_running_mean_rounds_half_up_and_the_weight_counts():
    """(10,20,30) then (21,20,33): means 15.5, 20, 31.5 -> 16, 20, 32 (half up),
    weight 2; a third frame (16,20,35): (2*16+16)/3 = 16, 20, (2*32+35)/3 = 33."""
    sc = _scene()
    rgb = np.zeros((INTR.height, INTR.width, 3), np.uint8)
    for col in ((10, 20, 30), (21, 20, 33)):
        rgb[...] = col
        _fuse(sc, rgb)
    C, _, band, _ = _band(sc, sc.params["mu"])
    assert np.all(C[band] == (16, 20, 32, 2))
    rgb[...] = (16, 20, 35)
    _fuse(sc, rgb)
    C, _, band, _ = _band(sc, sc.params["mu"])
    assert np.all(C[band] == (16, 20, 33, 3))


def test_colour_weight_stops_at_max_w():
    sc = _scene(max_w=3)
    rgb = np.zeros((INTR.height, INTR.width, 3), np.uint8)
    rgb[...] = (5, 6, 7)
    _fuse(sc, rgb, frames=6)
    C, _, band, _ = _band(sc, sc.params["mu"])
    assert np.all(C[band] == (5, 6, 7, 3))


def _ramp():
    """r = column, g = row, b = 100: bilinear sampling of a linear ramp is the
    position itself."""
    rgb = np.zeros((INTR.height, INTR.width, 3), np.uint8)
    rgb[..., 0] = np.arange(INTR.width)[None, :]
    rgb[..., 1] = np.arange(INTR.height)[:, None]
    rgb[..., 2] = 100
    return rgb


def _check_ramp(C, u, v, sel):
    ru, rv = np.floor(u + 0.5), np.floor(v + 0.5)
    # away from a rounding boundary the fp32 chain agrees with fp64 exactly
    clear = sel & (np.abs(u - np.round(u - 0.5) - 0.5) > 1e-3) & (np.abs(v - np.round(v - 0.5) - 0.5) > 1e-3)
    assert clear.sum() > 5000
    assert np.all(C[..., 0][clear] == ru[clear]) and np.all(C[..., 1][clear] == rv[clear])
    assert np.all(np.abs(C[..., 0][sel].astype(int) - ru[sel]) <= 1)
    assert np.all(C[..., 2][sel] == 100)


def test_bilinear_sample_is_the_analytic_projection():
    sc = _scene()
    _fuse(sc, _ramp())
    C, P, band, _ = _band(sc, sc.params["mu"])
    u = INTR.fx * P[..., 0] / P[..., 2] + INTR.cx
    v = INTR.fy * P[..., 1] / P[..., 2] + INTR.cy
    _check_ramp(C, u, v, band)


def test_extrinsic_map_shifts_the_sample():
    """A colour camera 5 cm along +x of the depth camera (points map by
    x - 0.05): on the plane z = 1 the sample moves by fx * 0.05 = 3 pixels."""
    T = np.eye(4, dtype=np.float32)
    T[0, 3] = -0.05
    sc = _scene()
    _fuse(sc, _ramp(), T_d2c=T)
    C, P, band, _ = _band(sc, sc.params["mu"])
    u = INTR.fx * (P[..., 0] - 0.05) / P[..., 2] + INTR.cx
    v = INTR.fy * P[..., 1] / P[..., 2] + INTR.cy
    sel = band & (u > 1) & (u < INTR.width - 2)
    _check_ramp(C, u, v, sel)
    assert np.all(C[band & (u < -0.5)] == 0)  # projects outside the colour image: no colour


def test_colour_integration_leaves_the_depth_fusion_unchanged():
    a, b = _scene(), oracle.Scene(**scene_params())
    rgb = _ramp()
    d = _plane()
    d[10:20, 30:40] = 0.8  # a step
    ia = INTR.as_array()
    for T in (EYE, np.array([[1, 0, 0, 0.02], [0, 1, 0, 0], [0, 0, 1, 0.03], [0, 0, 0, 1]], np.float32)):
        a.allocate(d, ia, T)
        b.allocate(d, ia, T)
        assert a.integrate_colour(d, ia, T, rgb, ia) == b.integrate(d, ia, T)
    ca, Fa, Wa = a.export()
    cb, Fb, Wb = b.export()
    assert np.array_equal(ca, cb) and np.array_equal(Fa, Fb) and np.array_equal(Wa, Wb)


def test_colour_at_is_the_nearest_voxel():
    sc = _scene()
    _fuse(sc, _ramp(), frames=2)
    vtx, _ = sc.raycast(INTR.width, INTR.height, INTR.as_array(), EYE)
    got = sc.colour_at(vtx)
    c, C = sc.export_colour()
    table = {tuple(int(x) for x in k): C[i] for i, k in enumerate(c)}
    inv_s = np.float32(1.0 / np.float64(sc.params["voxel_size"]))
    hits = vtx[..., 3] > 0
    assert hits.sum() > 2000
    for y, x in zip(*np.nonzero(hits)):
        g = np.floor(vtx[y, x, :3] * inv_s + np.float32(0.5)).astype(np.int64)
        b = tuple(int(t) for t in g >> 3)
        want = table[b][int((g[0] & 7) + 8 * (g[1] & 7) + 64 * (g[2] & 7))] if b in table else np.zeros(4, np.uint8)
        assert np.array_equal(got[y, x], want), (y, x)
    assert np.all(got[~hits] == 0)
    # hits sit in coloured voxels, except at the image border (bilinear needs the next pixel)
    assert np.mean(got[hits][:, 3] == 2) > 0.95
