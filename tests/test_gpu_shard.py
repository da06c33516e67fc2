"""A scene split over parts by slabs of block columns, on the GPU against the
oracle's split (one GPU: the parts are separate scenes run one after the
other in one process; no kernel waits on another).

Each part's allocated blocks, weights and voxels and its raycast meet the
parity bar against the oracle part with the same split; the library's merge
of the parts' maps (itm_raycast_merge) meets it against the oracle's merge,
and the union of the parts' own blocks is the whole scene's block set.
"""

import numpy as np
import pytest

import oracle
from synth import kinect_workload, tiny_workload
from tests.parity_util import compare_raycast, compare_volumes, key_of

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


@pytest.mark.parametrize("which,parts,slab", [("tiny", 2, 4), ("tiny", 3, 2), ("kinect", 2, 8)])
def test_split_scene_matches_the_oracle_split(itm, which, parts, slab):
    import torch
    w = tiny_workload() if which == "tiny" else kinect_workload()
    frames = range(w.n_frames) if which == "tiny" else range(0, 6)
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    ia = w.intr.as_array()
    gs = [itm.Scene(**w.params) for _ in range(parts)]
    os_ = [oracle.Scene(**w.params) for _ in range(parts)]
    for i in range(parts):
        gs[i].set_shard(parts, i, slab)
        os_[i].set_shard(parts, i, slab)
    full = oracle.Scene(**w.params)
    H, W = w.intr.height, w.intr.width
    vparts = torch.zeros((parts, H, W, 4), dtype=torch.float32, device="cuda")
    nparts = torch.zeros_like(vparts)
    for k in frames:
        f = w.frame(k)
        D = dev(f.depth)
        for i in range(parts):
            gs[i].process(D, ci, f.T_wc, vparts[i], nparts[i])
            os_[i].allocate(f.depth, ia, f.T_wc)
            os_[i].integrate(f.depth, ia, f.T_wc)
        full.allocate(f.depth, ia, f.T_wc)
        full.integrate(f.depth, ia, f.T_wc)
    vm = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    nm = torch.zeros_like(vm)
    itm.itm_raycast_merge(vparts, nparts, parts, ci, f.T_wc, vm, nm)
    torch.cuda.synchronize()
    orc_maps = [o.raycast(W, H, ia, f.T_wc) for o in os_]
    owned = []
    for i in range(parts):
        assert gs[i].status() == 0
        compare_volumes(gs[i].export(), os_[i].export())
        compare_raycast(vparts[i].cpu().numpy(), nparts[i].cpu().numpy(), *orc_maps[i], f.T_wc)
        c = gs[i].export(with_voxels=False)[0]
        owned += [k for k, bx in zip(key_of(c).tolist(), c[:, 0]) if oracle.slab_owner(int(bx), parts, slab) == i]
    assert sorted(owned) == sorted(key_of(full.export(with_voxels=False)[0]).tolist())
    vo, no = oracle.merge_raycasts(np.stack([m[0] for m in orc_maps]), np.stack([m[1] for m in orc_maps]), f.T_wc)
    compare_raycast(vm.cpu().numpy(), nm.cpu().numpy(), vo, no, f.T_wc)


def test_merge_kernel_on_constructed_maps(itm):
    """The library's merge against the oracle's merge bit for bit on random
    maps with ties, misses and every part winning somewhere."""
    import torch
    rng = np.random.default_rng(5)
    parts, H, W = 3, 37, 23
    T = np.eye(4, dtype=np.float32)
    T[:3, 3] = [0.3, -0.1, 0.2]
    v = np.zeros((parts, H, W, 4), np.float32)
    n = rng.normal(size=(parts, H, W, 4)).astype(np.float32)
    hit = rng.uniform(size=(parts, H, W)) < 0.6
    z = rng.uniform(0.5, 3.0, size=(parts, H, W)).astype(np.float32)
    z[1, ::4] = z[0, ::4]                                   # ties between parts 0 and 1
    v[..., 0] = rng.uniform(-1, 1, size=(parts, H, W))
    v[..., 1] = rng.uniform(-1, 1, size=(parts, H, W))
    v[..., 2] = z + T[2, 3]
    v[..., 3] = hit
    vo, no = oracle.merge_raycasts(v, n, T)
    ci = itm.make_intrinsics(W, H, 30.0, 30.0, W / 2, H / 2)
    vm = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    nm = torch.zeros_like(vm)
    itm.itm_raycast_merge(dev(v), dev(n), parts, ci, T, vm, nm)
    torch.cuda.synchronize()
    assert np.array_equal(vm.cpu().numpy(), vo) and np.array_equal(nm.cpu().numpy(), no)
    with pytest.raises(itm.ItmError):
        itm.itm_raycast_merge(dev(v), dev(n), 0, ci, T, vm, nm)
