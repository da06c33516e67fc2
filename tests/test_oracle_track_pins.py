"""Pins of the oracle's depth tracker (Sec. 4.1.1, ITMDepthTracker).

The paper states the method: render vertex and normal maps from the initial
guess, project the depth points onto them, minimise the sum of squared
point-to-plane distances (R p + t - V(p'))^T N(p') by solving a linear
system, iterate, over a resolution hierarchy of the depth image.  Readings
(recorded in the design notes): nearest-pixel projective association into the
reference view, an outlier distance per level, the linearised motion applied
on the world side, J = (T p x N, N), a pyramid of 2x2 means of the valid
depths.  The reference maps here are analytic (exact depth and SDF-gradient
normals of the synthetic scenes), not the oracle's own raycast; each test
checks the oracle against something other than itself: exact means, the
closed form of a plane offset, finite differences of the energy, and
convergence to the known true pose.
"""

import numpy as np
import pytest

import oracle
from synth import tiny_workload
from synth.scenes import AnalyticScene, Intrinsics, RoomInside, look_at


def analytic_maps(scene, intr, T):
    """World vertex and unit normal maps (float4, w = 1 on a hit) of an
    analytic scene seen from camera-to-world pose T."""
    T = np.asarray(T, np.float64)
    z, _ = scene.render(intr, T)
    H, W = z.shape
    u = np.arange(W)[None, :] * np.ones_like(z)
    v = np.arange(H)[:, None] * np.ones_like(z)
    rays = np.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, np.ones_like(z)], -1)
    Pw = (z[..., None] * rays) @ T[:3, :3].T + T[:3, 3]
    hit = z > 0
    P = Pw.reshape(-1, 3)
    g = np.zeros_like(P)
    h = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        g[:, a] = (scene.sdf(P + e) - scene.sdf(P - e)) / (2 * h)
    n = (g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-12)).reshape(Pw.shape)
    V = np.zeros((H, W, 4), np.float32)
    N = np.zeros((H, W, 4), np.float32)
    V[hit, :3], V[hit, 3] = Pw[hit], 1.0
    N[hit, :3], N[hit, 3] = n[hit], 1.0
    return V, N


def exp_pose(x, T):
    """[R(omega) | tau] T for x = (omega, tau), Rodrigues in fp64."""
    w = np.asarray(x[:3], np.float64)
    th = np.linalg.norm(w)
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    a = np.sin(th) / th if th > 0 else 1.0
    c = (1 - np.cos(th)) / th ** 2 if th > 0 else 0.5
    D = np.eye(4)
    D[:3, :3] = np.eye(3) + a * K + c * K @ K
    D[:3, 3] = x[3:]
    return (D @ np.asarray(T, np.float64)).astype(np.float32)


def pose_error(A, B):
    """(translation distance in m, rotation angle in degrees)."""
    A, B = np.asarray(A, np.float64), np.asarray(B, np.float64)
    R = A[:3, :3].T @ B[:3, :3]
    return np.linalg.norm(A[:3, 3] - B[:3, 3]), np.degrees(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)))


def test_depth_halve_means_valid_pixels():
    """Each output pixel is the float nearest to the exact mean of the valid
    depths of its 2x2 block (their sums are exact for these dyadic values, so
    one rounded division gives it), 0 when none is valid; odd edges are
    dropped."""
    from fractions import Fraction
    rng = np.random.default_rng(0)
    D = (rng.integers(1, 64, size=(9, 13)) / 8.0).astype(np.float32)
    D[rng.uniform(size=D.shape) < 0.3] = 0.0
    D[0:2, 0:2] = 0.0
    out = oracle.depth_halve(D)
    assert out.shape == (4, 6)
    for j in range(4):
        for i in range(6):
            blk = D[2 * j:2 * j + 2, 2 * i:2 * i + 2]
            valid = [Fraction(float(x)) for x in blk.ravel() if x > 0]
            if not valid:
                assert out[j, i] == 0.0
                continue
            exact = sum(valid) / len(valid)
            o = float(out[j, i])
            ulp = float(np.spacing(np.float32(o)))
            assert abs(Fraction(o) - exact) <= Fraction(ulp) / 2


def _plane_setup(W=48, H=36, z=2.0):
    intr = Intrinsics(W, H, 40.0, 40.0, (W - 1) / 2, (H - 1) / 2)
    u = np.arange(W)[None, :] * np.ones((H, 1))
    v = np.arange(H)[:, None] * np.ones((1, W))
    V = np.zeros((H, W, 4), np.float32)
    N = np.zeros((H, W, 4), np.float32)
    V[..., 0] = (u - intr.cx) / intr.fx * z
    V[..., 1] = (v - intr.cy) / intr.fy * z
    V[..., 2] = z
    V[..., 3] = 1.0
    N[..., 2] = -1.0
    N[..., 3] = 1.0
    D = np.full((H, W), z, np.float32)
    return intr, V, N, D


def test_plane_offset_closed_form():
    """A plane z = 2 seen from the identity, the estimate moved 1 cm along the
    normal: every pixel's distance is -1 cm, so sum r^2 = n delta^2, the
    translation gradient is n delta N, sum N_z^2 = n; in-plane components
    vanish; a threshold below the offset rejects every pixel."""
    intr, V, N, D = _plane_setup()
    delta = 0.01
    Tg = np.eye(4, dtype=np.float32)
    Tg[2, 3] = delta
    s, _ = oracle.icp_reduce(D, intr.as_array(), Tg, V, N, intr.as_array(), np.eye(4), 0.05)
    n = D.size
    assert s[28] == n
    assert s[27] == pytest.approx(n * delta ** 2, rel=1e-5)
    assert s[21 + 5] == pytest.approx(n * delta, rel=1e-5)           # sum N_z r
    assert s[21 + 3] == 0.0 and s[21 + 4] == 0.0                       # N_x = N_y = 0
    assert s[20] == n                                                  # sum N_z N_z
    assert abs(s[21 + 0]) < 1e-6 * n and abs(s[21 + 1]) < 1e-6 * n     # symmetric image
    s, _ = oracle.icp_reduce(D, intr.as_array(), Tg, V, N, intr.as_array(), np.eye(4), 0.009)
    assert s[28] == 0
    # a single plane constrains 3 of 6 motions: the step is refused, T kept
    s, _ = oracle.icp_reduce(D, intr.as_array(), Tg, V, N, intr.as_array(), np.eye(4), 0.05)
    T2, _, ok = oracle.icp_update(s, Tg)
    assert not ok and np.array_equal(T2, Tg)


def test_pixels_without_a_vertex_or_normal_are_not_used():
    """The reduction uses a reference pixel only when both its vertex and its
    normal are valid (w > 0): on the offset plane, pixels whose normal (or
    vertex) is marked invalid drop out of the count and of every sum."""
    intr, V, N, D = _plane_setup()
    delta = 0.01
    Tg = np.eye(4, dtype=np.float32)
    Tg[2, 3] = delta
    full, _ = oracle.icp_reduce(D, intr.as_array(), Tg, V, N, intr.as_array(), np.eye(4), 0.05)
    N2, V2 = N.copy(), V.copy()
    N2[:, ::2, 3] = 0.0          # every other column has no normal
    V2[::3, :, 3] = 0.0          # every third row has no vertex
    s, _ = oracle.icp_reduce(D, intr.as_array(), Tg, V2, N2, intr.as_array(), np.eye(4), 0.05)
    used = (N2[..., 3] > 0) & (V2[..., 3] > 0)
    n = int(used.sum())
    assert 0 < n < D.size and s[28] == n
    assert s[27] == pytest.approx(n * delta ** 2, rel=1e-5)
    assert s[20] == n and s[21 + 5] == pytest.approx(n * delta, rel=1e-5)
    assert full[28] == D.size


def _box_view():
    scene = AnalyticScene([RoomInside((-1.0, 0.0, -1.5), (1.5, 2.0, 1.0))])
    intr = Intrinsics(64, 48, 50.0, 50.0, 31.5, 23.5)
    T = look_at((0.2, 1.1, 0.1), (1.5, 0.0, -1.5)).astype(np.float32)
    return scene, intr, T


def test_gradient_matches_finite_differences_of_the_energy():
    """Inside a box (three planes in view) the point-to-plane distance does
    not depend on which point of the plane the association picks, so the
    energy sum r^2 is smooth in the motion and its central differences give
    2 sum J r (up to pixels that change plane at an edge)."""
    scene, intr, Tref = _box_view()
    V, N = analytic_maps(scene, intr, Tref)
    D = scene.render(intr, Tref.astype(np.float64))[0].astype(np.float32)
    Tg = exp_pose(np.array([0.002, -0.003, 0.001, 0.004, -0.002, 0.003]), Tref)
    a = intr.as_array()
    s, _ = oracle.icp_reduce(D, a, Tg, V, N, a, Tref, 0.1)
    g = s[21:27]
    assert s[28] > 2000 and np.all(np.abs(g) > 0.1)
    h = 1e-4
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        Ep = oracle.icp_reduce(D, a, exp_pose(e, Tg), V, N, a, Tref, 0.1)[0][27]
        Em = oracle.icp_reduce(D, a, exp_pose(-e, Tg), V, N, a, Tref, 0.1)[0][27]
        assert (Ep - Em) / (2 * h) == pytest.approx(2 * g[i], rel=0.1), i


def test_hessian_is_the_sum_of_outer_products_of_the_gradient_rows():
    """With one usable pixel, sum J J^T = J J^T and sum J r = J r, so
    H = g g^T / r^2 (rank one)."""
    scene, intr, Tref = _box_view()
    V, N = analytic_maps(scene, intr, Tref)
    D = np.zeros((intr.height, intr.width), np.float32)
    D[20, 30] = scene.render(intr, Tref.astype(np.float64))[0][20, 30]
    Tg = exp_pose(np.array([0.0, 0.0, 0.0, 0.01, 0.0, 0.0]), Tref)
    s, _ = oracle.icp_reduce(D, intr.as_array(), Tg, V, N, intr.as_array(), Tref, 0.1)
    assert s[28] == 1
    H = np.zeros((6, 6))
    k = 0
    for i in range(6):
        for j in range(i, 6):
            H[i, j] = H[j, i] = s[k]
            k += 1
    g, r2 = s[21:27], s[27]
    np.testing.assert_allclose(H, np.outer(g, g) / r2, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("k,pert", [(4, (0, 0, 0, 0, 0, 0)), (4, (0.02, -0.03, 0.01, 0.03, -0.02, 0.02)),
                                    (7, (-0.03, 0.02, 0.02, -0.02, 0.03, 0.01))])
def test_tracking_recovers_the_true_pose(k, pert):
    """Reference maps rendered at the previous frame's pose, the depth of
    frame k, the estimate started at the previous pose moved by up to 3
    degrees and 4 cm: coarse-to-fine tracking lands on frame k's true pose
    within 0.5 mm and 0.1 degree."""
    w = tiny_workload(noise_scale=0.0)
    Tref, Ttrue = w.frame(k - 1).T_wc, w.frame(k).T_wc
    V, N = analytic_maps(w.scene, w.intr, Tref)
    Tinit = exp_pose(np.array(pert, np.float64), Tref)
    T, steps = oracle.track(w.frame(k).depth, w.intr.as_array(), [10, 5, 4], [0.05, 0.1, 0.2], V, N,
                            w.intr.as_array(), Tref, Tinit)
    t0, a0 = pose_error(Tinit, Ttrue)
    t1, a1 = pose_error(T, Ttrue)
    assert t0 > 0.02 and steps > 10
    assert t1 < 5e-4 and a1 < 0.1, (t1, a1)


@pytest.mark.parametrize("level,tol_m", [(1, 1.5e-3), (2, 3e-3)])
def test_each_pyramid_level_alone_tracks(level, tol_m):
    """A half- or quarter-resolution level alone (its depth the 2x2 means,
    its intrinsics f/2 and (c - 1/2)/2, as pixel i covers pixels 2i, 2i+1)
    recovers the true pose to within a fraction of its pixel footprint; a
    centre off by a quarter pixel biases it by several millimetres."""
    w = tiny_workload(noise_scale=0.0)
    for k in (4, 7):
        Tref, Ttrue = w.frame(k - 1).T_wc, w.frame(k).T_wc
        V, N = analytic_maps(w.scene, w.intr, Tref)
        iters = [0, 0, 0]
        iters[level] = 10
        T, steps = oracle.track(w.frame(k).depth, w.intr.as_array(), iters, [0.05, 0.1, 0.2], V, N,
                                w.intr.as_array(), Tref, Tref)
        t1, a1 = pose_error(T, Ttrue)
        assert steps == 10 and t1 < tol_m and a1 < 0.1, (k, t1, a1)
