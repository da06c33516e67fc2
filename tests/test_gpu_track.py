"""Depth tracker (Sec. 4.1.1) on the GPU against the oracle.

* pyramid level: bit-exact (same float operations);
* ICP sums: the pixel count is exact (the per-pixel decisions are the same
  float operations on both sides); every other sum within 2e-6 of the sum of
  its terms' magnitudes (the GPU adds a thread's ~8 products and then a
  warp's 32 lanes in float, at most 13 roundings of 2^-24 relative to that
  magnitude; the oracle adds exact products in double);
* host step: the oracle's step (both in double) to 1e-6;
* tracking: the oracle's final pose matrix within 1e-5 per element (an
  angle from the trace of R^T R' is no finer than ~0.02 degree for float
  matrices), and the true pose within 0.5 mm / 0.1 degree on noise-free
  analytic maps.
"""

import numpy as np
import pytest

import oracle
from synth import Intrinsics, kinect_workload, tiny_workload
from tests.test_oracle_track_pins import analytic_maps, exp_pose, pose_error

pytestmark = pytest.mark.gpu

ITERS = [10, 5, 4]
THRESH = [0.05, 0.1, 0.2]


@pytest.fixture(scope="module")
def itm():
    import torch
    assert torch.cuda.is_available()
    import paper_1708_00783_gb300 as m
    return m


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def intr_of(m, intr: Intrinsics):
    return m.make_intrinsics(intr.width, intr.height, intr.fx, intr.fy, intr.cx, intr.cy)


@pytest.mark.parametrize("shape", [(120, 160), (37, 53), (480, 640), (3, 2)])
def test_depth_halve_bit_exact(itm, shape):
    import torch
    rng = np.random.default_rng(shape[0])
    D = rng.uniform(0.3, 5.0, size=shape).astype(np.float32)
    D[rng.uniform(size=shape) < 0.2] = 0.0
    D[rng.uniform(size=shape) < 0.02] = -1.0
    D[rng.uniform(size=shape) < 0.02] = np.nan
    out = torch.full((shape[0] // 2, shape[1] // 2), 7.0, dtype=torch.float32, device="cuda")
    itm.itm_depth_halve(dev(D), shape[1], shape[0], out)
    torch.cuda.synchronize()
    want = oracle.depth_halve(D)
    assert np.array_equal(out.cpu().numpy(), want)


def _check_sums(g, o, a):
    assert g[28] == o[28]
    tol = 2e-6 * np.asarray(a) + 1e-12
    bad = np.nonzero(np.abs(g[:28] - o[:28]) > tol)[0]
    assert bad.size == 0, [(int(k), g[k], o[k], tol[k]) for k in bad]


def _tiny_case(k=4, pert=(0.01, -0.02, 0.01, 0.02, -0.01, 0.015)):
    w = tiny_workload(noise_scale=0.0)
    Tref = w.frame(k - 1).T_wc
    V, N = analytic_maps(w.scene, w.intr, Tref)
    return w, Tref, V, N, exp_pose(np.array(pert), Tref)


def test_icp_reduce_matches_oracle_tiny(itm):
    import torch
    w, Tref, V, N, Tg = _tiny_case()
    ci = intr_of(itm, w.intr)
    work = torch.zeros(itm.ITM_ICP_WORK_DOUBLES, dtype=torch.float64, device="cuda")
    d = w.frame(4).depth
    for thresh in (0.02, 0.1, 1.0):
        itm.itm_icp_reduce(dev(d), ci, Tg, dev(V), dev(N), ci, Tref, thresh, work)
        torch.cuda.synchronize()
        g = work[:29].cpu().numpy()
        o, a = oracle.icp_reduce(d, w.intr.as_array(), Tg, V, N, w.intr.as_array(), Tref, thresh)
        assert o[28] > 1000
        _check_sums(g, o, a)


def _fused_kinect(itm, frames=range(0, 10)):
    """A GPU volume of the noisy room and the raycast maps of its last pose."""
    import torch
    w = kinect_workload(seed=2)
    sc = itm.Scene(**w.params)
    ci = intr_of(itm, w.intr)
    H, W = w.intr.height, w.intr.width
    V = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    N = torch.zeros_like(V)
    for k in frames:
        f = w.frame(k)
        sc.process(dev(f.depth), ci, f.T_wc, V, N)
    torch.cuda.synchronize()
    return w, sc, ci, V, N


def test_icp_reduce_matches_oracle_kinect(itm):
    import torch
    w, sc, ci, V, N = _fused_kinect(itm)
    Tref = w.frame(9).T_wc
    f = w.frame(10)
    work = torch.zeros(itm.ITM_ICP_WORK_DOUBLES, dtype=torch.float64, device="cuda")
    for Tg in (Tref, exp_pose(np.array([0.01, 0.0, -0.01, 0.01, 0.02, 0.0]), Tref)):
        itm.itm_icp_reduce(dev(f.depth), ci, Tg, V, N, ci, Tref, 0.1, work)
        torch.cuda.synchronize()
        g = work[:29].cpu().numpy()
        o, a = oracle.icp_reduce(f.depth, w.intr.as_array(), Tg, V.cpu().numpy(), N.cpu().numpy(), w.intr.as_array(),
                                 Tref, 0.1)
        assert o[28] > 100000
        _check_sums(g, o, a)


def test_host_step_matches_oracle(itm):
    w, Tref, V, N, Tg = _tiny_case()
    o, _ = oracle.icp_reduce(w.frame(4).depth, w.intr.as_array(), Tg, V, N, w.intr.as_array(), Tref, 0.1)
    T1, x1 = itm.itm_icp_step(o, Tg)
    T2, x2, ok = oracle.icp_update(o, Tg)
    assert ok
    np.testing.assert_allclose(x1, x2, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(T1, T2, atol=1e-6)
    bad = o.copy()
    bad[28] = 3.0
    with pytest.raises(itm.ItmError):
        itm.itm_icp_step(bad, Tg)


def _track_pair(itm, w, depth, V, N, Tref, Tinit, intr=None, iters=ITERS, thresh=THRESH):
    import torch
    intr = intr or w.intr
    ci = intr_of(itm, intr)
    H, W = depth.shape
    nbytes = itm.itm_track_scratch_bytes(W, H, len(iters))
    scratch = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-scratch.data_ptr()) % 256
    Vd = V if hasattr(V, "data_ptr") else dev(V)
    Nd = N if hasattr(N, "data_ptr") else dev(N)
    Tg, steps = itm.itm_track_depth(dev(depth), ci, iters, thresh, Vd, Nd, ci, Tref, Tinit, scratch.data_ptr() + off)
    Vh = V.cpu().numpy() if hasattr(V, "cpu") else V
    Nh = N.cpu().numpy() if hasattr(N, "cpu") else N
    To, steps_o = oracle.track(depth, intr.as_array(), iters, thresh, Vh, Nh, intr.as_array(), Tref, Tinit)
    return Tg, steps, To, steps_o


@pytest.mark.parametrize("k,pert", [(4, (0, 0, 0, 0, 0, 0)), (7, (-0.03, 0.02, 0.02, -0.02, 0.03, 0.01))])
def test_track_matches_oracle_and_truth(itm, k, pert):
    w = tiny_workload(noise_scale=0.0)
    Tref, Ttrue = w.frame(k - 1).T_wc, w.frame(k).T_wc
    V, N = analytic_maps(w.scene, w.intr, Tref)
    Tinit = exp_pose(np.array(pert, np.float64), Tref)
    Tg, steps, To, steps_o = _track_pair(itm, w, w.frame(k).depth, V, N, Tref, Tinit)
    assert steps == steps_o == sum(ITERS)
    assert np.abs(Tg - To).max() < 1e-5, np.abs(Tg - To).max()
    t1, a1 = pose_error(Tg, Ttrue)
    assert t1 < 5e-4 and a1 < 0.1


def test_track_kinect_noisy_room(itm):
    """Frame 10 of the noisy room tracked against the raycast of the volume
    fused from frames 0..9, started at frame 9's pose."""
    w, sc, ci, V, N = _fused_kinect(itm)
    Tref, Ttrue = w.frame(9).T_wc, w.frame(10).T_wc
    Tg, steps, To, steps_o = _track_pair(itm, w, w.frame(10).depth, V, N, Tref, Tref)
    assert steps == steps_o and np.abs(Tg - To).max() < 1e-5, np.abs(Tg - To).max()
    t0, a0 = pose_error(Tref, Ttrue)
    t1, a1 = pose_error(Tg, Ttrue)
    assert t1 < 0.25 * t0 + 1e-3 and t1 < 3e-3 and a1 < 0.2, (t0, a0, t1, a1)


def test_track_degenerate_and_invalid(itm):
    """A single plane constrains only 3 motions: every level stops at once and
    the pose is returned unchanged; bad arguments are rejected."""
    import torch
    W, H, z = 48, 36, 2.0
    intr = Intrinsics(W, H, 40.0, 40.0, (W - 1) / 2, (H - 1) / 2)
    u = np.arange(W)[None, :] * np.ones((H, 1))
    v = np.arange(H)[:, None] * np.ones((1, W))
    V = np.zeros((H, W, 4), np.float32)
    N = np.zeros((H, W, 4), np.float32)
    V[..., 0], V[..., 1], V[..., 2], V[..., 3] = (u - intr.cx) / intr.fx * z, (v - intr.cy) / intr.fy * z, z, 1
    N[..., 2], N[..., 3] = -1.0, 1.0
    D = np.full((H, W), z, np.float32)
    Tinit = np.eye(4, dtype=np.float32)
    Tinit[2, 3] = 0.01
    Tg, steps, To, steps_o = _track_pair(itm, None, D, V, N, np.eye(4, dtype=np.float32), Tinit, intr=intr)
    assert steps == steps_o == 0 and np.array_equal(Tg, Tinit)
    ci = intr_of(itm, intr)
    scratch = torch.empty(itm.itm_track_scratch_bytes(W, H, 3), dtype=torch.uint8, device="cuda")
    Dd, Vd, Nd = dev(D), dev(V), dev(N)
    for args in (dict(iters=[1] * 9, thresh=[0.1] * 9), dict(iters=[-1, 1, 1], thresh=THRESH),
                 dict(iters=ITERS, thresh=[0.1, 0.0, 0.1]), dict(iters=ITERS, thresh=[0.1, np.nan, 0.1])):
        with pytest.raises(itm.ItmError):
            itm.itm_track_depth(Dd, ci, args["iters"], args["thresh"], Vd, Nd, ci, np.eye(4), Tinit,
                                scratch.data_ptr())
    with pytest.raises(itm.ItmError):   # misaligned scratch
        itm.itm_track_depth(Dd, ci, ITERS, THRESH, Vd, Nd, ci, np.eye(4), Tinit, scratch.data_ptr() + 8)
    work = torch.zeros(itm.ITM_ICP_WORK_DOUBLES, dtype=torch.float64, device="cuda")
    with pytest.raises(itm.ItmError):
        itm.itm_icp_reduce(Dd, ci, Tinit, Vd, Nd, ci, np.eye(4), -1.0, work)
