"""The allocation-free block query against the scene path.

itm_frame_blocks_noalloc serves callers that cannot allocate device memory
once they are running (a real-time loop that must not wait on the
allocator, a framework that hands out device memory only from its own fixed
arenas).  It must return exactly the blocks that itm_allocate inserts into an
empty scene.  Consecutive calls share the library's fixed set, so the calls
below run back to back on overlapping frames: a set not cleared between
calls would hide blocks of the second frame.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _intr(itm, w):
    return itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)


def test_noalloc_block_set_equals_scene_allocation_on_consecutive_calls():
    import torch

    import paper_1708_00783_gb300 as itm
    from synth import kinect_workload, tiny_workload

    cap = 1 << 20
    coords = torch.empty((cap, 3), dtype=torch.int16, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    kinect = kinect_workload()
    calls = [(tiny_workload(n_frames=2), 1), (kinect, 5), (kinect, 6)]
    for w, k in calls:
        f = w.frame(k)
        d = _dev(f.depth)
        ci = _intr(itm, w)
        p = w.params
        itm.itm_frame_blocks_noalloc(d, ci, f.T_wc, p["voxel_size"], p["mu"], p["z_min"], p["z_max"],
                                     coords, cap, count)
        torch.cuda.synchronize()
        raw = int(count.item())
        assert raw & ~0x3FFFFFFF == 0, "flags set: %#x" % raw
        n = raw
        assert 0 < n <= cap
        got = coords[:n].cpu().numpy()
        got_set = {tuple(c) for c in got.tolist()}
        assert len(got_set) == n, "a block was reported twice"
        ref = itm.Scene(**p)
        ref.allocate(d, ci, f.T_wc)
        want = {tuple(c) for c in ref.export(with_voxels=False)[0].tolist()}
        assert ref.status() == 0
        assert got_set == want, (len(got_set - want), len(want - got_set))
        ref.close()


def test_noalloc_rejects_inputs_beyond_its_fixed_set():
    import torch

    import paper_1708_00783_gb300 as itm

    W, H = 4096, 4096
    depth = torch.ones((H, W), dtype=torch.float32, device="cuda")
    coords = torch.empty((16, 3), dtype=torch.int16, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    ci = itm.make_intrinsics(W, H, 500.0, 500.0, W / 2, H / 2)
    with pytest.raises(itm.ItmError) as e:
        itm.itm_frame_blocks_noalloc(depth, ci, np.eye(4), 0.005, 0.02, 0.4, 5.0, coords, 16, count)
    assert e.value.code == 8  # ITM_ERR_TOO_LARGE
    # a small cap is fine: the count still reports every block
    w = 64
    small = torch.ones((w, w), dtype=torch.float32, device="cuda")
    cs = itm.make_intrinsics(w, w, 60.0, 60.0, w / 2, w / 2)
    itm.itm_frame_blocks_noalloc(small, cs, np.eye(4), 0.005, 0.02, 0.4, 5.0, coords, 16, count)
    torch.cuda.synchronize()
    assert int(count.item()) > 16


def test_noalloc_flags_pixels_beyond_the_int16_block_range_and_refuses_non_rigid_poses():
    """A camera 5 km from the origin puts every segment outside the int16
    block coordinates: the pixels are dropped and the count carries
    ITM_NOALLOC_RANGE, as itm_allocate reports ITM_ST_RANGE for the same frame.
    A scaled pose (not rigid) is refused before any work."""
    import torch

    import paper_1708_00783_gb300 as itm
    from synth import tiny_workload

    w = tiny_workload(n_frames=1)
    f = w.frame(0)
    d = _dev(f.depth)
    ci = _intr(itm, w)
    p = w.params
    coords = torch.empty((1024, 3), dtype=torch.int16, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    far = f.T_wc.astype(np.float32).copy()
    far[0, 3] += 5000.0
    itm.itm_frame_blocks_noalloc(d, ci, far, p["voxel_size"], p["mu"], p["z_min"], p["z_max"], coords, 1024, count)
    torch.cuda.synchronize()
    raw = int(count.item())
    assert raw & itm.ITM_NOALLOC_RANGE
    assert raw & 0x3FFFFFFF == 0
    ref = itm.Scene(**p)
    ref.allocate(d, ci, far)
    assert ref.status() & 0x4  # ITM_ST_RANGE
    ref.close()
    scaled = f.T_wc.astype(np.float32).copy()
    scaled[:3, :3] *= 2.0
    with pytest.raises(itm.ItmError) as e:
        itm.itm_frame_blocks_noalloc(d, ci, scaled, p["voxel_size"], p["mu"], p["z_min"], p["z_max"],
                                     coords, 1024, count)
    assert e.value.code == itm.ITM_ERR_ARG
