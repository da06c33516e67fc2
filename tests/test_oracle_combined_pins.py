"""Pins of the oracle's combined-map raycast (Sec. 7.2).

The paper defines the combined TSDF of posed submaps as the sum over submaps
of weight times TSDF at P_i X, and renders the global map by raycasting it.
Readings (recorded with the others in the design notes): P_i maps world to
submap coordinates; F and its weight are interpolated trilinearly in each
submap (unallocated voxels: value 1, weight 0); the sum is divided by the
weight sum (value 1 where nothing was observed), which keeps its zero set and
the raycast's step rule; the march is the Sec. 4.4 state machine in world
coordinates.  Each test checks the oracle against something other than
itself: the weighted mean in closed form, a linear field under a known rigid
map, the single-map raycast, the analytic scene geometry, and the union of
submaps that saw disjoint halves of the images.
"""

import numpy as np
import pytest

import oracle
from synth import tiny_workload
from tests.test_oracle_pins import _silhouettes, scene_params

S = 0.01


def _scene():
    return oracle.Scene(**scene_params(voxel_size=S))


def _rot(axis, deg):
    a = np.radians(deg)
    c, s = np.cos(a), np.sin(a)
    i, j = [k for k in range(3) if k != axis]
    R = np.eye(3)
    R[i, i], R[i, j], R[j, i], R[j, j] = c, -s, s, c
    return R


def _pose(R, t):
    P = np.eye(4)
    P[:3, :3] = R
    P[:3, 3] = t
    return P


def test_combined_value_is_the_weight_normalised_sum():
    """F^(X) = sum_i W_i F_i / sum_i W_i, with unobserved submaps ignored and
    the default 1 where no submap has weight."""
    a, b, c = _scene(), _scene(), _scene()
    a.set_block((0, 0, 0), 0.3, 2.0)
    b.set_block((0, 0, 0), -0.5, 5.0)
    c.set_block((0, 0, 0), 0.9, 0.0)
    P = np.stack([np.eye(4)] * 3)
    X = np.array([3.3, 2.1, 4.7]) * S
    want = (2.0 * 0.3 + 5.0 * -0.5) / 7.0
    for order in ([a, b, c], [c, b, a], [b, c, a]):
        v, den = oracle.combined_value(order, P, X)
        assert v == pytest.approx(want, abs=1e-6) and den == pytest.approx(7.0)
    v, den = oracle.combined_value([c], P[:1], X)
    assert v == 1.0 and den == 0.0
    v, den = oracle.combined_value([a, b], P[:2], np.array([50.0, 50.0, 50.0]) * S)   # no block there
    assert v == 1.0 and den == 0.0


def test_combined_weight_is_interpolated_trilinearly():
    """The weight enters as its trilinear interpolation at P_i X, like the
    TSDF: a weight growing along x shifts the blend continuously."""
    a, b = _scene(), _scene()
    g = np.arange(512)
    a.set_block((0, 0, 0), 0.2, (g % 8 + 1).astype(np.float32))   # W_a = x + 1
    b.set_block((0, 0, 0), -0.6, 3.0)
    P = np.stack([np.eye(4)] * 2)
    for x in (1.0, 2.25, 4.5, 6.75):
        X = np.array([x, 3.0, 3.0]) * S
        wa = x + 1.0
        v, den = oracle.combined_value([a, b], P, X)
        assert den == pytest.approx(wa + 3.0, rel=1e-6)
        assert v == pytest.approx((wa * 0.2 + 3.0 * -0.6) / (wa + 3.0), abs=2e-6)


@pytest.mark.parametrize("axis,deg,t", [(2, 90.0, (0.02, 0.03, 0.01)), (0, -35.0, (-0.1, 0.05, 0.2)),
                                        (1, 150.0, (0.3, -0.2, 0.0))])
def test_combined_value_maps_world_points_into_the_submap(axis, deg, t):
    """P_i maps world to submap coordinates: with F linear in the submap's x
    (F = (x - 3.5) / 4 over one block), F^ at world X equals that line at
    Y = P_i X."""
    sc = _scene()
    g = np.arange(512)
    sc.set_block((0, 0, 0), ((g % 8) - 3.5) / 4.0, 1.0)
    P = _pose(_rot(axis, deg), t)
    for y in ([3.25, 2.5, 4.75], [1.5, 6.0, 0.5], [5.875, 1.25, 2.0]):
        Y = np.array(y) * S
        X = P[:3, :3].T @ (Y - P[:3, 3])
        v, den = oracle.combined_value([sc], P[None], X)
        assert den == pytest.approx(1.0, abs=1e-6)
        assert v == pytest.approx((y[0] - 3.5) / 4.0, abs=2e-5)


def _fuse(w, frames, P=None, mask=None):
    """An oracle scene fused in submap coordinates (camera poses P T_wc)."""
    sc = oracle.Scene(**w.params)
    intr = w.intr.as_array()
    for k in frames:
        f = w.frame(k)
        T = f.T_wc if P is None else (P @ f.T_wc.astype(np.float64)).astype(np.float32)
        d = f.depth if mask is None else np.where(mask, f.depth, 0.0).astype(np.float32)
        sc.allocate(d, intr, T)
        sc.integrate(d, intr, T)
    return sc


@pytest.fixture(scope="module")
def noise_free():
    return tiny_workload(noise_scale=0.0)


def _camera_z(vtx, T):
    T = T.astype(np.float64)
    return (((vtx[..., :3].reshape(-1, 3).astype(np.float64) - T[:3, 3]) @ T[:3, :3])[:, 2]).reshape(vtx.shape[:2])


def test_one_submap_at_identity_is_the_single_map_raycast(noise_free):
    """With one submap at the identity the combined value is that submap's
    TSDF wherever it has weight (W F / W up to one rounding), so the combined
    raycast reproduces the Sec. 4.4 raycast."""
    w = noise_free
    sc = _fuse(w, range(w.n_frames))
    f = w.frame(4)
    intr = w.intr.as_array()
    v1, n1 = sc.raycast(w.intr.width, w.intr.height, intr, f.T_wc)
    vc, nc = oracle.raycast_combined([sc], np.eye(4)[None], w.intr.width, w.intr.height, intr, f.T_wc)
    h1, hc = v1[..., 3] > 0, vc[..., 3] > 0
    assert h1.sum() > 10000 and np.mean(h1 == hc) >= 0.999
    both = h1 & hc
    dz = np.abs(_camera_z(v1, f.T_wc) - _camera_z(vc, f.T_wc))[both]
    assert np.mean(dz <= 5e-4) >= 0.999
    nb = both & (n1[..., 3] > 0) & (nc[..., 3] > 0)
    cosang = np.clip(np.sum(n1[..., :3][nb].astype(np.float64) * nc[..., :3][nb], axis=1), -1, 1)
    assert np.mean(np.degrees(np.arccos(cosang)) <= 0.5) >= 0.999


POSES = [_pose(_rot(1, 12.0) @ _rot(0, -7.0), (0.15, -0.05, 0.2)), _pose(_rot(2, -20.0), (-0.3, 0.1, 0.05))]


def _check_on_analytic_surface(w, vtx, nrm, T, min_cover=0.97):
    s = w.params["voxel_size"]
    z_true, pid = w.scene.render(w.intr, T.astype(np.float64))
    z = _camera_z(vtx, T)
    hit = vtx[..., 3] > 0
    ok = (z_true > 0) & (z_true < 4.5) & ~_silhouettes(pid, z_true)
    assert (hit & ok).sum() / ok.sum() > min_cover
    gy, gx = np.gradient(z_true)
    smooth = ok & hit & (np.hypot(gx, gy) <= 0.5 * s)
    err = np.abs(z - z_true)
    assert smooth.sum() > 1500
    assert np.mean(err[smooth] <= 0.25 * s) >= 0.99
    sph = hit & ok & (nrm[..., 3] > 0) & (pid == 1) & (z_true < 2.5)
    P = vtx[..., :3][sph].astype(np.float64)
    c = np.array([-0.35, 0.3, 0.0])
    radial = (P - c) / np.linalg.norm(P - c, axis=1, keepdims=True)
    ang = np.degrees(np.arccos(np.clip(np.sum(nrm[..., :3][sph] * radial, axis=1), -1, 1)))
    assert sph.sum() > 500 and np.median(ang) <= 1.5
    return hit, ok


def test_posed_submaps_render_the_analytic_surface(noise_free):
    """Two submaps, each fused in its own rotated and shifted frame: the
    combined raycast from a world camera finds the analytic surfaces (depth
    within s/4, sphere normals radial)."""
    w = noise_free
    subs = [_fuse(w, range(w.n_frames), P) for P in POSES]
    f = w.frame(4)
    vtx, nrm = oracle.raycast_combined(subs, np.stack(POSES), w.intr.width, w.intr.height, w.intr.as_array(),
                                       f.T_wc)
    _check_on_analytic_surface(w, vtx, nrm, f.T_wc)


def test_submaps_of_disjoint_halves_render_their_union(noise_free):
    """A submap that only saw the left halves of the images and one that only
    saw the right halves: the combined map renders both halves."""
    w = noise_free
    W = w.intr.width
    left = np.zeros((w.intr.height, W), dtype=bool)
    left[:, :W // 2] = True
    subs = [_fuse(w, range(w.n_frames), POSES[0], left), _fuse(w, range(w.n_frames), POSES[1], ~left)]
    f = w.frame(4)
    vtx, nrm = oracle.raycast_combined(subs, np.stack(POSES), W, w.intr.height, w.intr.as_array(), f.T_wc)
    hit, ok = _check_on_analytic_surface(w, vtx, nrm, f.T_wc, min_cover=0.9)
    u = np.arange(W)[None, :] * np.ones_like(hit)
    for side in (u < W // 2 - 12, u > W // 2 + 12):
        assert (hit & ok & side).sum() / (ok & side).sum() > 0.95
    # each submap alone covers only its own side
    for sub, side in ((subs[0], u > W // 2 + 12), (subs[1], u < W // 2 - 12)):
        vs, _ = oracle.raycast_combined([sub], np.stack(POSES)[[subs.index(sub)]], W, w.intr.height,
                                        w.intr.as_array(), f.T_wc)
        assert ((vs[..., 3] > 0) & ok & side).sum() / (ok & side).sum() < 0.5
