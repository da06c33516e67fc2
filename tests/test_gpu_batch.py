"""Batched per-frame core (submaps, many scenes) against the CPU oracle and the
single-scene path.

Every scene processed inside a batch is run through the oracle on the same
frames, crops and poses (a submap at its submap-relative pose), and its
allocated blocks, weights, voxels and raycast images must meet the parity bar
against the oracle's.  It must also end up bit-identical to the same scene
processed alone with itm_allocate / itm_integrate / itm_raycast -- with the
captured CUDA graph and without, for scenes of different resolutions, voxel
sizes and hash sizes in one batch, and for one frame fused into several
submaps at their relative poses (InfiniTAM v3 Sec. 7.2).
"""

import subprocess

import numpy as np
import pytest

import oracle
from synth import Intrinsics, batched, kinect_workload, tiny_workload
from tests.parity_util import compare_raycast, compare_volumes

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


def crop(frame_depth, intr, W, H):
    u0, v0 = (intr.width - W) // 2, (intr.height - H) // 2
    ci = Intrinsics(W, H, intr.fx, intr.fy, intr.cx - u0, intr.cy - v0)
    return np.ascontiguousarray(frame_depth[v0:v0 + H, u0:u0 + W]), ci


def small_room():
    """The first 80x60 room of the batched workload's 64 independent scenes
    (with its own voxel size, mu = 4 voxels)."""
    return next(w for w in batched.small_scenes() if w.intr.width == 80)


def scene_specs():
    """(workload, params, crop size) of scenes with uneven sizes."""
    tiny = tiny_workload()
    room = kinect_workload(seed=5)
    small = small_room()
    return [
        (tiny, dict(tiny.params), (160, 120)),
        (tiny, dict(tiny.params, num_buckets=1 << 8, num_excess=1 << 13), (96, 72)),
        (room, dict(room.params, num_buckets=1 << 16, num_blocks=1 << 17), (320, 240)),
        (room, dict(room.params, voxel_size=0.008, mu=0.032, num_buckets=1 << 18, num_blocks=1 << 17), (640, 480)),
        (small, dict(small.params), (80, 60)),
    ]


def oracle_scene(params):
    """The oracle for one scene: the OpenMP build where there is one (its
    results are byte-identical to the single-threaded build's)."""
    try:
        return oracle.Scene(**params, threaded=True)
    except (OSError, subprocess.CalledProcessError):
        return oracle.Scene(**params)


def as_intr(itm, c):
    return itm.make_intrinsics(c.width, c.height, c.fx, c.fy, c.cx, c.cy)


@pytest.mark.parametrize("use_graph,schedule", [(True, [1, 0, 0]), (False, [1, 0, 0]), (True, [4, 1, 1]),
                                                 (True, [2, 0, 1])])
def test_batch_equals_single_scene_path(itm, use_graph, schedule):
    """Also with the schedule knobs moved (blocks per integration CTA,
    scattered tile walks): results do not depend on them."""
    import torch
    specs = scene_specs()
    batch = itm.itm_batch_create(8)
    itm.itm_batch_set_graph(batch, use_graph)
    itm.itm_batch_set_schedule(batch, schedule)
    assert itm.itm_batch_get_schedule(batch) == schedule
    batched = [itm.Scene(**p) for _, p, _ in specs]
    alone = [itm.Scene(**p) for _, p, _ in specs]
    orcs = [oracle_scene(p) for _, p, _ in specs]
    stream = torch.cuda.Stream()
    for k in range(4):
        items, refs = [], []
        for (w, p, (W, H)), sb, sa, so in zip(specs, batched, alone, orcs):
            f = w.frame(k)
            d, ci = crop(f.depth, w.intr, W, H)
            D = dev(d)
            intr = as_intr(itm, ci)
            vb = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
            nb = torch.zeros_like(vb)
            va = torch.zeros_like(vb)
            na = torch.zeros_like(vb)
            items.append((sb.handle, D, intr, f.T_wc, vb, nb))
            refs.append((sa, so, d, ci, D, intr, f.T_wc, va, na, vb, nb))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            itm.itm_batch_run(batch, items, stream=stream)
        stream.synchronize()
        for sa, so, d, ci, D, intr, T, va, na, vb, nb in refs:
            sa.allocate(D, intr, T)
            sa.integrate(D, intr, T)
            sa.raycast(intr, T, va, na)
        torch.cuda.synchronize()
        for sa, so, d, ci, D, intr, T, va, na, vb, nb in refs:
            assert torch.equal(va, vb) and torch.equal(na, nb)
            # the batch against the oracle on the same crop and pose
            _, _, (vo, no) = so.process(d, ci.as_array(), T)
            assert so.status == 0
            compare_raycast(vb.cpu().numpy(), nb.cpu().numpy(), vo, no, T)
    for sb, sa, so in zip(batched, alone, orcs):
        assert sb.status() == 0 and sa.status() == 0
        rep = compare_volumes(sb.export(), sa.export())
        assert rep["sdf_bitexact_frac"] == 1.0
        compare_volumes(sb.export(), so.export())
        st_b, st_a = sb.stats(), sa.stats()
        assert st_b["updated_voxels"] == st_a["updated_voxels"] and st_b["frames"] == st_a["frames"] == 4
    itm.itm_batch_destroy(batch)


def submap_poses(n, seed=3):
    """World-from-submap rigid poses: rotations up to 15 degrees, offsets up to
    0.5 m."""
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


def test_one_frame_fused_into_submaps(itm):
    """One depth frame (one device buffer) fused into three submaps at their
    relative poses in one batch; each submap matches its own single-scene run
    and the oracle run at the submap-relative pose."""
    import torch
    w = kinect_workload(seed=9)
    p = dict(w.params, num_buckets=1 << 18, num_blocks=1 << 18)
    P = submap_poses(3)
    subs_b = [itm.Scene(**p) for _ in P]
    subs_a = [itm.Scene(**p) for _ in P]
    subs_o = [oracle_scene(p) for _ in P]
    batch = itm.itm_batch_create(4)
    stream = torch.cuda.Stream()
    ci = as_intr(itm, w.intr)
    H, W = w.intr.height, w.intr.width
    for k in (0, 10):
        f = w.frame(k)
        D = dev(f.depth)
        items, outs = [], []
        for Pi, sb in zip(P, subs_b):
            T = (np.linalg.inv(Pi) @ f.T_wc.astype(np.float64)).astype(np.float32)
            vb = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
            nb = torch.zeros_like(vb)
            items.append((sb.handle, D, ci, T, vb, nb))
            outs.append((T, vb, nb))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            itm.itm_batch_run(batch, items, stream=stream)
        stream.synchronize()
        for (T, vb, nb), sa, so in zip(outs, subs_a, subs_o):
            va = torch.zeros_like(vb)
            na = torch.zeros_like(vb)
            sa.process(D, ci, T, va, na)
            torch.cuda.synchronize()
            assert torch.equal(va, vb) and torch.equal(na, nb)
            _, _, (vo, no) = so.process(f.depth, w.intr.as_array(), T)
            assert so.status == 0
            compare_raycast(vb.cpu().numpy(), nb.cpu().numpy(), vo, no, T)
    for sb, sa, so in zip(subs_b, subs_a, subs_o):
        rep = compare_volumes(sb.export(), sa.export())
        assert rep["sdf_bitexact_frac"] == 1.0
        compare_volumes(sb.export(), so.export())
    itm.itm_batch_destroy(batch)


def test_batch_rejects_invalid_items(itm):
    import torch
    w = tiny_workload(n_frames=1)
    f = w.frame(0)
    D = dev(f.depth)
    ci = as_intr(itm, w.intr)
    a = itm.Scene(**w.params)
    learned = itm.Scene(**dict(w.params, weight_mode=1))
    batch = itm.itm_batch_create(2)
    with pytest.raises(itm.ItmError):
        itm.itm_batch_run(batch, [(a.handle, D, ci, f.T_wc, None, None)] * 2)   # same scene twice
    with pytest.raises(itm.ItmError):
        itm.itm_batch_run(batch, [(learned.handle, D, ci, f.T_wc, None, None)])
    b = itm.Scene(**w.params)
    c = itm.Scene(**w.params)
    with pytest.raises(itm.ItmError):
        itm.itm_batch_run(batch, [(s.handle, D, ci, f.T_wc, None, None) for s in (a, b, c)])  # over capacity
    for knobs in ([3, 0, 0], [1, 2, 0], [1, 0, -1], [1, 0]):
        with pytest.raises(itm.ItmError):
            if len(knobs) == 3:
                itm.itm_batch_set_schedule(batch, knobs)
            else:
                itm._check(itm._lib.itm_batch_set_schedule(batch, (itm.ctypes.c_int * 2)(*knobs), 2), "x")
    bad = f.T_wc.copy()
    bad[0, 0] = np.nan
    with pytest.raises(itm.ItmError):
        itm.itm_batch_run(batch, [(a.handle, D, ci, bad, None, None)])
    torch.cuda.synchronize()
    assert a.stats()["allocated_blocks"] == 0    # nothing ran
    itm.itm_batch_destroy(batch)
