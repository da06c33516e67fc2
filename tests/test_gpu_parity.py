"""CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs: allocated block sets and weights bit-exact, sdf within 1e-4, raycast
depth/normals within 0.5 mm / 0.5 degrees on >= 99.9% of pixels."""

import numpy as np
import pytest

import oracle
from synth import Intrinsics, kinect_workload, large_workload, tiny_workload
from tests.parity_util import compare_raycast, compare_volumes, key_of
from tests.test_oracle_pins import check_hash_invariants

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


def run_pair(itm, w, frames, params=None, raycast_frames=(), window=None):
    """Fuse `frames` of workload w on both sides; raycast after the frames in
    raycast_frames.  Returns (gpu scene, oracle scene, raycast reports)."""
    import torch
    p = dict(w.params if params is None else params)
    g = itm.Scene(**p)
    o = oracle.Scene(**p)
    ci = intr_of(itm, w.intr)
    ia = w.intr.as_array()
    H, W = w.intr.height, w.intr.width
    vtx = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    nrm = torch.zeros_like(vtx)
    reps = []
    for k in frames:
        f = w.frame(k)
        d = dev(f.depth)
        g.allocate(d, ci, f.T_wc)
        g.integrate(d, ci, f.T_wc)
        o.allocate(f.depth, ia, f.T_wc)
        o.integrate(f.depth, ia, f.T_wc)
        if k in raycast_frames:
            g.raycast(ci, f.T_wc, vtx, nrm)
            torch.cuda.synchronize()
            vo, no = o.raycast(W, H, ia, f.T_wc)
            reps.append(compare_raycast(vtx.cpu().numpy(), nrm.cpu().numpy(), vo, no, f.T_wc))
    return g, o, reps


def test_tiny_full_sequence(itm):
    w = tiny_workload()
    g, o, reps = run_pair(itm, w, range(w.n_frames), raycast_frames=set(range(w.n_frames)))
    assert g.status() == 0 and o.status == 0
    rep = compare_volumes(g.export(), o.export())
    st = g.stats()
    assert st["allocated_blocks"] == o.num_allocated
    assert st["frames"] == w.n_frames
    assert rep["sdf_bitexact_frac"] == 1.0  # the GPU follows the listing's float arithmetic exactly
    assert len(reps) == w.n_frames
    for r in reps:
        assert r["bitexact_frac"] >= 0.999, r


def test_tiny_updated_voxel_count_matches(itm):
    """The kernel's own update counter equals the oracle's count."""
    w = tiny_workload(n_frames=3)
    import torch
    g = itm.Scene(**w.params)
    o = oracle.Scene(**w.params)
    ci = intr_of(itm, w.intr)
    total = 0
    for k in range(3):
        f = w.frame(k)
        d = dev(f.depth)
        g.allocate(d, ci, f.T_wc)
        g.integrate(d, ci, f.T_wc)
        o.allocate(f.depth, w.intr.as_array(), f.T_wc)
        total += o.integrate(f.depth, w.intr.as_array(), f.T_wc)
    st = g.stats()
    assert st["updated_voxels"] == total
    assert 0 < st["visible_blocks"] <= st["allocated_blocks"]


def test_excess_chains_and_table_invariants(itm):
    """2^8 buckets force most blocks into excess chains and many intra-frame
    bucket collisions (resolved by the overflow pass)."""
    w = tiny_workload(n_frames=4)
    p = dict(w.params, num_buckets=1 << 8, num_excess=1 << 13)
    g, o, reps = run_pair(itm, w, range(4), params=p, raycast_frames={3})
    assert g.status() == 0
    compare_volumes(g.export(), o.export())
    st = g.stats()
    assert st["excess_used"] == o.excess_used
    coords = g.export(with_voxels=False)[0]
    check_hash_invariants(g.export_table(), coords, p["num_buckets"], p["num_excess"], p["num_blocks"],
                          st["allocated_blocks"], lambda x, y, z: itm.itm_hash_index(x, y, z, p["num_buckets"]))


@pytest.mark.parametrize("shape", [(37, 23), (33, 9), (160, 120)])
def test_ragged_image_sizes(itm, shape):
    """Image sizes that are not multiples of the 32x8 pixel tiles."""
    W, H = shape
    w = tiny_workload(n_frames=2)
    # a crop of the tiny frames with a shifted principal point describes the same rays
    u0, v0 = (160 - W) // 2, (120 - H) // 2
    intr = Intrinsics(W, H, w.intr.fx, w.intr.fy, w.intr.cx - u0, w.intr.cy - v0)
    import torch
    g = itm.Scene(**w.params)
    o = oracle.Scene(**w.params)
    ci = intr_of(itm, intr)
    vtx = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    nrm = torch.zeros_like(vtx)
    for k in range(2):
        f = w.frame(k)
        crop = np.ascontiguousarray(f.depth[v0:v0 + H, u0:u0 + W])
        g.allocate(dev(crop), ci, f.T_wc)
        g.integrate(dev(crop), ci, f.T_wc)
        o.allocate(crop, intr.as_array(), f.T_wc)
        o.integrate(crop, intr.as_array(), f.T_wc)
    g.raycast(ci, f.T_wc, vtx, nrm)
    vo, no = o.raycast(W, H, intr.as_array(), f.T_wc)
    compare_volumes(g.export(), o.export())
    compare_raycast(vtx.cpu().numpy(), nrm.cpu().numpy(), vo, no, f.T_wc)


def test_degenerate_inputs(itm):
    """Empty, negative and NaN depth allocate nothing; a camera facing away
    updates nothing; the volume is unchanged."""
    import torch
    w = tiny_workload(n_frames=1)
    f = w.frame(0)
    ci = intr_of(itm, w.intr)
    g = itm.Scene(**w.params)
    for bad in (np.zeros_like(f.depth), np.full_like(f.depth, -1.0), np.full_like(f.depth, np.nan)):
        g.allocate(dev(bad), ci, f.T_wc)
        g.integrate(dev(bad), ci, f.T_wc)
    st = g.stats()
    assert st["allocated_blocks"] == 0 and st["updated_voxels"] == 0 and st["status"] == 0
    g.allocate(dev(f.depth), ci, f.T_wc)
    g.integrate(dev(f.depth), ci, f.T_wc)
    before = g.export()
    away = f.T_wc.copy()
    away[:3, 0] *= -1
    away[:3, 2] *= -1
    n0 = g.stats()["updated_voxels"]
    g.integrate(dev(np.full_like(f.depth, 1.0)), ci, away)
    assert g.stats()["updated_voxels"] == n0
    after = g.export()
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    vtx = torch.ones((w.intr.height, w.intr.width, 4), dtype=torch.float32, device="cuda")
    nrm = torch.ones_like(vtx)
    empty = itm.Scene(**w.params)
    empty.raycast(ci, f.T_wc, vtx, nrm)
    assert not vtx.any().item() and not nrm.any().item()


def test_capacity_errors(itm):
    w = tiny_workload(n_frames=1)
    f = w.frame(0)
    ci = intr_of(itm, w.intr)
    g = itm.Scene(**dict(w.params, num_buckets=1 << 6, num_excess=16))
    g.allocate(dev(f.depth), ci, f.T_wc)
    assert g.status() == 3  # ITM_ERR_HASH_FULL
    assert g.stats()["excess_used"] == 16
    g = itm.Scene(**dict(w.params, num_blocks=100))
    g.allocate(dev(f.depth), ci, f.T_wc)
    assert g.status() == 4  # ITM_ERR_VBA_FULL
    assert g.stats()["allocated_blocks"] == 100


def test_invalid_arguments_are_rejected(itm):
    w = tiny_workload(n_frames=1)
    with pytest.raises(itm.ItmError):
        itm.Scene(**dict(w.params, num_buckets=1000))   # not a power of two
    with pytest.raises(itm.ItmError):
        itm.Scene(**dict(w.params, max_w=300))          # uint8 weights
    g = itm.Scene(**w.params)
    bad = itm.make_intrinsics(0, 0, 1, 1, 0, 0)
    with pytest.raises(itm.ItmError):
        g.allocate(dev(w.frame(0).depth), bad, w.frame(0).T_wc)
    with pytest.raises(itm.ItmError):
        itm.itm_allocate(g.handle, 0, intr_of(itm, w.intr), w.frame(0).T_wc)


def test_depth_u16_conversion_bit_exact(itm):
    import torch
    raw = np.concatenate([np.arange(65536), np.arange(7) * 9000]).astype(np.uint16)
    ref = oracle.depth_u16_to_f32(raw)
    r = dev(raw.view(np.int16))
    out = torch.empty(raw.size, dtype=torch.float32, device="cuda")
    itm.itm_depth_u16_to_f32(r, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    # unaligned start and ragged length take the scalar path
    out2 = torch.empty(raw.size, dtype=torch.float32, device="cuda")
    itm.itm_depth_u16_to_f32(r.data_ptr() + 2, out2.data_ptr() + 4, raw.size - 3)
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy()[1:raw.size - 2].view(np.uint32), ref[1:raw.size - 2].view(np.uint32))


def test_export_import_resume_is_bit_exact(itm):
    """Checkpoint / resume: export after 3 frames, import into a new scene,
    continue both for 2 frames: identical volumes."""
    w = tiny_workload(n_frames=5)
    ci = intr_of(itm, w.intr)
    a = itm.Scene(**w.params)
    for k in range(3):
        f = w.frame(k)
        a.process(dev(f.depth), ci, f.T_wc)
    c, F, Wt = a.export()
    b = itm.Scene(**w.params)
    b.import_blocks(c, F, Wt)
    cb, Fb, Wb = b.export()
    assert np.array_equal(cb, c) and np.array_equal(Fb, F) and np.array_equal(Wb, Wt)
    for k in range(3, 5):
        f = w.frame(k)
        a.process(dev(f.depth), ci, f.T_wc)
        b.process(dev(f.depth), ci, f.T_wc)
    compare_volumes(a.export(), b.export())


def test_uint16_frames_give_the_same_volume(itm):
    """The millimetre variant converted on the GPU fuses identically."""
    import torch
    w = tiny_workload(n_frames=2)
    ci = intr_of(itm, w.intr)
    a = itm.Scene(**w.params)
    b = itm.Scene(**w.params)
    for k in range(2):
        f = w.frame(k)
        a.process(dev(f.depth), ci, f.T_wc)
        d = torch.empty(f.depth.shape, dtype=torch.float32, device="cuda")
        itm.itm_depth_u16_to_f32(dev(f.depth_u16.view(np.int16)), d)
        b.process(d, ci, f.T_wc)
    compare_volumes(a.export(), b.export())


@pytest.mark.parametrize("which", ["tiny", "kinect"])
def test_fused_u16_allocation_equals_conversion_then_allocation(itm, which):
    """itm_process_frame_u16 (the frame converted inside the allocation) gives
    the float frame of itm_depth_u16_to_f32, the same volume and the same
    raycast maps, bit for bit, frame after frame (with holes and ragged
    edges in the Kinect frames)."""
    import torch
    w = tiny_workload(n_frames=4) if which == "tiny" else kinect_workload(seed=6)
    ci = intr_of(itm, w.intr)
    H, W = w.intr.height, w.intr.width
    a = itm.Scene(**w.params)
    b = itm.Scene(**w.params)
    maps = [torch.zeros((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(4)]
    for k in range(4):
        f = w.frame(k)
        raw = dev(f.depth_u16.view(np.int16))
        da = torch.empty((H, W), dtype=torch.float32, device="cuda")
        db = torch.full((H, W), np.nan, dtype=torch.float32, device="cuda")
        itm.itm_depth_u16_to_f32(raw, da)
        a.process(da, ci, f.T_wc, maps[0], maps[1])
        itm.itm_process_frame_u16(b.handle, raw, db, ci, f.T_wc, maps[2], maps[3])
        torch.cuda.synchronize()
        assert torch.equal(da, db)
        assert torch.equal(maps[0], maps[2]) and torch.equal(maps[1], maps[3])
    assert a.status() == 0 and b.status() == 0
    rep = compare_volumes(a.export(), b.export())
    assert rep["sdf_bitexact_frac"] == 1.0


@pytest.mark.slow
def test_kinect_scale_frames(itm):
    """Full 640x480, 5 mm voxels, 2^20 buckets: the configuration the
    benchmark times, through the same calls."""
    w = kinect_workload()
    frames = [0, 1, 2, 15, 30]
    g, o, reps = run_pair(itm, w, frames, raycast_frames={2, 30})
    assert g.status() == 0 and o.status == 0
    rep = compare_volumes(g.export(), o.export())
    assert rep["blocks"] > 5000
    for r in reps:
        assert r["hits"] > 250000


@pytest.mark.slow
def test_large_scale_frames(itm):
    """640x480 at 2 mm voxels with 2^22 buckets and 2^21 blocks, and again
    with 2^18 buckets so the excess list carries part of the table."""
    for nb in (1 << 22, 1 << 18):
        w = large_workload(num_buckets=nb)
        p = dict(w.params)
        g, o, _ = run_pair(itm, w, [0, 1], params=p)
        assert g.status() == 0 and o.status == 0
        compare_volumes(g.export(), o.export())
        if nb == 1 << 18:
            assert g.stats()["excess_used"] > 0


def _novel_pose(T, yaw_deg, back):
    """The pose turned about its own y axis and moved back along its view axis."""
    a = np.radians(yaw_deg)
    Ry = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    N = np.asarray(T, dtype=np.float64).copy()
    N[:3, :3] = N[:3, :3] @ Ry
    N[:3, 3] = N[:3, 3] - back * N[:3, 2]
    return N.astype(np.float32)


def test_raycast_range_bounds_hits_and_novel_views(itm):
    """Sec. 4.4 search range: each tile's [zmin, zmax] covers the depth of
    every hit in it (within mu: the two refinement steps may move the hit
    out of the block region that stopped the march), tiles with no block
    have no hit; raycasts from views that were never fused match the oracle."""
    import torch
    w = tiny_workload()
    g, o, _ = run_pair(itm, w, range(w.n_frames))
    ci = intr_of(itm, w.intr)
    H, W = w.intr.height, w.intr.width
    tx, ty = (W + 7) // 8, (H + 3) // 4
    mu = w.params["mu"]
    vtx = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    nrm = torch.zeros_like(vtx)
    zmin = torch.zeros(ty * tx, dtype=torch.float32, device="cuda")
    zmax = torch.zeros_like(zmin)
    base = w.frame(4).T_wc
    for yaw, back in ((0.0, 0.0), (12.0, 0.3), (-20.0, -0.5), (35.0, 0.8)):
        T = _novel_pose(base, yaw, back)
        itm.itm_raycast_range(g.handle, ci, T, zmin, zmax)
        g.raycast(ci, T, vtx, nrm)
        torch.cuda.synchronize()
        vo, no = o.raycast(W, H, w.intr.as_array(), T)
        rep = compare_raycast(vtx.cpu().numpy(), nrm.cpu().numpy(), vo, no, T)
        lo = zmin.cpu().numpy().reshape(ty, tx)
        hi = zmax.cpu().numpy().reshape(ty, tx)
        hit = vo[..., 3] > 0
        vv, uu = np.nonzero(hit)
        z = camera_depth_of(vo, T)[hit]
        tlo, thi = lo[vv // 4, uu // 8], hi[vv // 4, uu // 8]
        assert np.all(np.isfinite(tlo)), "a hit in a tile no block covers"
        assert np.all(z >= tlo - mu) and np.all(z <= thi + mu)
        assert np.isnan(lo).any() or rep["hits"] > 0


def camera_depth_of(vtx, T):
    from tests.parity_util import camera_depth
    return camera_depth(vtx, T)


def test_raycast_independent_of_tile_order(itm):
    """The raycast hands tiles out in the order of the previous raycast's
    per-tile costs (raster order when there is none for the image size).
    Each ray's result must not depend on that order: repeated raycasts from
    one pose, with a raycast of another image size in between (which makes
    the stored order unusable), give bit-identical maps, equal to the
    oracle's within the raycast tolerance."""
    import torch
    w = tiny_workload()
    g, o, _ = run_pair(itm, w, range(w.n_frames))
    ci = intr_of(itm, w.intr)
    H, W = w.intr.height, w.intr.width
    T = _novel_pose(w.frame(6).T_wc, 8.0, 0.2)
    small = Intrinsics(W - 24, H - 12, w.intr.fx, w.intr.fy, w.intr.cx - 12, w.intr.cy - 6)
    cs = intr_of(itm, small)
    outs = []
    for k in range(5):
        if k == 3:
            vs = torch.zeros((small.height, small.width, 4), dtype=torch.float32, device="cuda")
            g.raycast(cs, T, vs, torch.zeros_like(vs))
        v = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
        n = torch.zeros_like(v)
        g.raycast(ci, T, v, n)
        torch.cuda.synchronize()
        outs.append((v.cpu().numpy(), n.cpu().numpy()))
    for v, n in outs[1:]:
        assert np.array_equal(v, outs[0][0]) and np.array_equal(n, outs[0][1])
    vo, no = o.raycast(W, H, w.intr.as_array(), T)
    rep = compare_raycast(outs[0][0], outs[0][1], vo, no, T)
    assert rep["hits"] > 0


def _rot_y(deg):
    a = np.radians(deg)
    R = np.eye(4)
    R[0, 0] = R[2, 2] = np.cos(a)
    R[0, 2], R[2, 0] = np.sin(a), -np.sin(a)
    return R


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("change", ["pose", "intrinsics"])
def test_integration_at_another_pose_than_the_allocation(itm, change, weighted):
    """The visible list marks blocks whose voxels all project inside the image
    for the allocation's pose and intrinsics, and the integration then skips
    their bounds tests.  Integrating at another pose (10 degrees of yaw) or
    with other intrinsics (cx shifted by 40 px) must not use those marks:
    every block the GPU changes equals the oracle's integration of it at the
    new pose (the oracle integrates every allocated block, the GPU the
    allocation's visible list, so only the blocks the GPU changed compare).
    weighted: float weights, with a seeded per-pixel weight map in (0, 1]
    (zeros on a tenth of the pixels) on both sides."""
    w = kinect_workload(seed=3)
    ci = intr_of(itm, w.intr)
    ia = w.intr.as_array()
    rng = np.random.default_rng(11)

    def weight_map(shape):
        m = rng.uniform(0.05, 1.0, size=shape).astype(np.float32)
        m[rng.random(shape) < 0.1] = 0.0
        return m

    if weighted:
        p = dict(w.params, weight_mode=1)
        g, o = itm.Scene(**p), oracle.Scene(**p)
        for k in range(3):
            fk = w.frame(k)
            m = weight_map(fk.depth.shape)
            dk = dev(fk.depth)
            g.allocate(dk, ci, fk.T_wc)
            g.integrate(dk, ci, fk.T_wc, wpx=dev(m))
            o.allocate(fk.depth, ia, fk.T_wc)
            o.integrate(fk.depth, ia, fk.T_wc, m)
    else:
        g, o, _ = run_pair(itm, w, range(3))
    f = w.frame(3)
    d = dev(f.depth)
    g.allocate(d, ci, f.T_wc)
    o.allocate(f.depth, ia, f.T_wc)
    wpx = weight_map(f.depth.shape) if weighted else None
    T2, ci2, ia2 = f.T_wc, ci, ia
    if change == "pose":
        T2 = (np.asarray(f.T_wc, np.float64) @ _rot_y(10.0)).astype(np.float32)
    else:
        i2 = w.intr
        ci2 = itm.make_intrinsics(i2.width, i2.height, i2.fx, i2.fy, i2.cx + 40.0, i2.cy)
        ia2 = np.array([i2.fx, i2.fy, i2.cx + 40.0, i2.cy], dtype=np.float32)
    before = g.export()
    g.integrate(d, ci2, T2, wpx=None if wpx is None else dev(wpx))
    o.integrate(f.depth, ia2, T2, wpx)
    after = g.export()
    cg, Fg, Wg = after
    assert np.array_equal(before[0], cg)
    changed = np.any(Wg != before[2], axis=1)
    assert changed.sum() > 1000
    co, Fo, Wo = o.export()
    pos = {k: i for i, k in enumerate(key_of(co).tolist())}
    io = np.array([pos[k] for k in key_of(cg[changed]).tolist()])
    assert np.array_equal(Wg[changed], Wo[io])
    assert np.abs(Fg[changed] - Fo[io]).max() <= 1e-4


def test_raycast_wider_than_the_search_range_images(itm):
    """An image wider than the search-range tiles cover (4096 pixels) takes
    the raycast without a search range (one kernel, raster tiles): a
    4104 x 24 strip through the tiny scene's centre, a few pixels of it
    ragged against the warp tiles, equals the oracle's raycast within the
    raycast tolerance, twice in a row (the tile queues are not involved)."""
    import torch
    w = tiny_workload()
    g, o, _ = run_pair(itm, w, range(w.n_frames))
    T = w.frame(5).T_wc
    Wd, Hd = 4104, 24
    strip = Intrinsics(Wd, Hd, w.intr.fx, w.intr.fy, (Wd - 1) / 2.0, (Hd - 1) / 2.0)
    cs = intr_of(itm, strip)
    outs = []
    for _ in range(2):
        v = torch.zeros((Hd, Wd, 4), dtype=torch.float32, device="cuda")
        n = torch.zeros_like(v)
        g.raycast(cs, T, v, n)
        torch.cuda.synchronize()
        outs.append((v.cpu().numpy(), n.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    vo, no = o.raycast(Wd, Hd, strip.as_array(), T)
    rep = compare_raycast(outs[0][0], outs[0][1], vo, no, T)
    assert rep["hits"] > 1000


def test_fusion_of_an_image_wider_than_the_search_range_images(itm):
    """Allocation and integration of a frame wider than the search-range
    tiles cover (4104 x 24, rendered from the tiny scene without noise):
    the allocation then builds the visible list without a search range, and
    the volume after it equals the oracle's (block set and weights exact,
    sdf within 1e-4)."""
    w = tiny_workload()
    g, o, _ = run_pair(itm, w, range(3))
    T = w.frame(4).T_wc
    Wd, Hd = 4104, 24
    strip = Intrinsics(Wd, Hd, w.intr.fx, w.intr.fy, (Wd - 1) / 2.0, (Hd - 1) / 2.0)
    z = w.scene.render(strip, T)[0].astype(np.float32)
    z[(z < w.params["z_min"]) | (z > w.params["z_max"])] = 0.0
    assert np.count_nonzero(z) > 2000
    cs = intr_of(itm, strip)
    d = dev(z)
    g.allocate(d, cs, T)
    g.integrate(d, cs, T)
    o.allocate(z, strip.as_array(), T)
    o.integrate(z, strip.as_array(), T)
    assert g.status() == 0
    compare_volumes(g.export(), o.export())
