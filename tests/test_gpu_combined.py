"""Combined-map raycast (Sec. 7.2) on the GPU against the oracle.

The same submaps are fused on both sides (each submap in its own frame, the
camera poses mapped by P_i); the two volumes are bit-identical per submap, so
the combined raycasts must agree at the raycast tolerance: hit/miss on
>= 99.9% of pixels, depth <= 0.5 mm and normals <= 0.5 degrees where both
hit.  Cases: posed submaps that overlap, submaps that saw disjoint image
halves, one submap at the identity, novel views, uneven submap counts up to
the maximum, and argument errors.
"""

import numpy as np
import pytest

import oracle
from synth import Intrinsics, kinect_workload, tiny_workload
from tests.parity_util import compare_raycast

pytestmark = pytest.mark.gpu


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


POSES = [_pose(_rot(1, 12.0) @ _rot(0, -7.0), (0.15, -0.05, 0.2)), _pose(_rot(2, -20.0), (-0.3, 0.1, 0.05)),
         _pose(_rot(0, 30.0), (0.05, 0.4, -0.2)), np.eye(4)]


def fuse_pair(itm, w, frames, P, mask=None, params=None):
    """One submap fused on the GPU and in the oracle, camera poses P T_wc."""
    p = dict(params or w.params)
    g = itm.Scene(**p)
    o = oracle.Scene(**p)
    ci = intr_of(itm, w.intr)
    for k in frames:
        f = w.frame(k)
        T = (P @ f.T_wc.astype(np.float64)).astype(np.float32)
        d = f.depth if mask is None else np.where(mask, f.depth, 0.0).astype(np.float32)
        D = dev(d)
        g.allocate(D, ci, T)
        g.integrate(D, ci, T)
        o.allocate(d, w.intr.as_array(), T)
        o.integrate(d, w.intr.as_array(), T)
    return g, o


def combined_pair(itm, w, subs, P, T, intr=None):
    import torch
    intr = intr or w.intr
    ci = intr_of(itm, intr)
    vtx = torch.full((intr.height, intr.width, 4), 7.0, dtype=torch.float32, device="cuda")
    nrm = torch.full_like(vtx, 7.0)
    itm.itm_raycast_combined([g.handle for g, _ in subs], np.stack(P).astype(np.float32), ci, T, vtx, nrm)
    torch.cuda.synchronize()
    vo, no = oracle.raycast_combined([o for _, o in subs], np.stack(P), intr.width, intr.height, intr.as_array(), T)
    return vtx.cpu().numpy(), nrm.cpu().numpy(), vo, no


def _novel(T, yaw_deg, back):
    a = np.radians(yaw_deg)
    Ry = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    N = np.asarray(T, dtype=np.float64).copy()
    N[:3, :3] = N[:3, :3] @ Ry
    N[:3, 3] = N[:3, 3] - back * N[:3, 2]
    return N.astype(np.float32)


@pytest.fixture(scope="module")
def tiny_submaps(itm):
    w = tiny_workload()
    subs = [fuse_pair(itm, w, range(w.n_frames), P) for P in POSES[:3]]
    return w, subs


@pytest.mark.parametrize("yaw,back", [(0.0, 0.0), (15.0, 0.3), (-25.0, -0.4)])
def test_posed_submaps_match_oracle(itm, tiny_submaps, yaw, back):
    w, subs = tiny_submaps
    T = _novel(w.frame(5).T_wc, yaw, back)
    vg, ng, vo, no = combined_pair(itm, w, subs, POSES[:3], T)
    rep = compare_raycast(vg, ng, vo, no, T)
    assert rep["hits"] > 5000
    assert rep["bitexact_frac"] >= 0.99, rep


def test_uneven_submap_counts(itm, tiny_submaps):
    """1, 2 and 3 submaps in every order give the oracle's maps."""
    w, subs = tiny_submaps
    T = w.frame(2).T_wc
    for idx in ([0], [2, 1], [1, 0, 2], [2, 0]):
        vg, ng, vo, no = combined_pair(itm, w, [subs[i] for i in idx], [POSES[i] for i in idx], T)
        compare_raycast(vg, ng, vo, no, T)


def test_disjoint_halves(itm):
    w = tiny_workload()
    Wd = w.intr.width
    left = np.zeros((w.intr.height, Wd), dtype=bool)
    left[:, :Wd // 2] = True
    subs = [fuse_pair(itm, w, range(w.n_frames), POSES[0], left),
            fuse_pair(itm, w, range(w.n_frames), POSES[1], ~left)]
    T = w.frame(4).T_wc
    vg, ng, vo, no = combined_pair(itm, w, subs, POSES[:2], T)
    rep = compare_raycast(vg, ng, vo, no, T)
    assert rep["hits"] > 5000


def test_maximum_submap_count_and_ragged_image(itm):
    """ITM_COMBINED_MAX submaps (the same four fused volumes repeated) and an
    image whose size is not a multiple of the 8x4 tile."""
    w = tiny_workload(n_frames=4)
    subs = [fuse_pair(itm, w, range(4), P) for P in POSES]
    n = itm.ITM_COMBINED_MAX
    idx = [i % 4 for i in range(n)]
    small = Intrinsics(101, 67, w.intr.fx, w.intr.fy, 50.3, 33.1)
    T = w.frame(1).T_wc
    vg, ng, vo, no = combined_pair(itm, w, [subs[i] for i in idx], [POSES[i] for i in idx], T, intr=small)
    compare_raycast(vg, ng, vo, no, T)


def test_empty_submaps_miss_everywhere(itm):
    import torch
    w = tiny_workload(n_frames=1)
    a, b = itm.Scene(**w.params), itm.Scene(**w.params)
    ci = intr_of(itm, w.intr)
    vtx = torch.full((w.intr.height, w.intr.width, 4), 7.0, dtype=torch.float32, device="cuda")
    nrm = torch.full_like(vtx, 7.0)
    itm.itm_raycast_combined([a.handle, b.handle], np.stack(POSES[:2]).astype(np.float32), ci, w.frame(0).T_wc,
                             vtx, nrm)
    torch.cuda.synchronize()
    assert not vtx.any().item() and not nrm.any().item()


def test_invalid_arguments(itm):
    import torch
    w = tiny_workload(n_frames=1)
    a = itm.Scene(**w.params)
    other = itm.Scene(**dict(w.params, voxel_size=0.02, mu=0.08))
    learned = itm.Scene(**dict(w.params, weight_mode=1))
    ci = intr_of(itm, w.intr)
    T = w.frame(0).T_wc
    vtx = torch.zeros((w.intr.height, w.intr.width, 4), dtype=torch.float32, device="cuda")
    nrm = torch.zeros_like(vtx)
    P1 = np.eye(4, dtype=np.float32)[None]
    bad = P1.copy()
    bad[0, 0, 3] = np.inf
    cases = [
        ([], np.zeros((0, 4, 4), np.float32)),
        ([a.handle] * 17, np.stack([np.eye(4, dtype=np.float32)] * 17)),
        ([a.handle, other.handle], np.stack([np.eye(4, dtype=np.float32)] * 2)),
        ([a.handle, learned.handle], np.stack([np.eye(4, dtype=np.float32)] * 2)),
        ([a.handle], bad),
        ([None], P1),
    ]
    for scenes, P in cases:
        with pytest.raises(itm.ItmError):
            itm.itm_raycast_combined(scenes, P, ci, T, vtx, nrm)
    with pytest.raises(itm.ItmError):
        itm.itm_raycast_combined([a.handle], P1, ci, T, vtx.view(-1)[1:], nrm)   # misaligned


@pytest.mark.slow
def test_kinect_scale_submaps(itm):
    """Three submaps of the room sequence at 640x480 (5 mm voxels), rendered
    from a pose between the submaps' trajectories."""
    w = kinect_workload(seed=3)
    p = dict(w.params, num_buckets=1 << 18, num_blocks=1 << 17, num_excess=1 << 16)
    subs = [fuse_pair(itm, w, range(k, k + 40, 4), P, params=p) for k, P in zip((0, 20, 40), POSES[:3])]
    T = w.frame(30).T_wc
    vg, ng, vo, no = combined_pair(itm, w, subs, POSES[:3], T)
    rep = compare_raycast(vg, ng, vo, no, T)
    assert rep["hits"] > 100000
