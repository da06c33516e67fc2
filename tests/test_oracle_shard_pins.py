"""Pins of the oracle's slab partition of one scene over several parts (the
multi-process form of the per-frame core; not in the paper).

Block column x belongs to part floor(x / w) mod n; part i keeps its own
columns and one column on either side; its raycast reports only hits in its
own columns; the parts' maps merge per pixel to the hit nearest the camera.
Checked here against the whole-scene oracle: each part's blocks are exactly
the whole scene's blocks in its kept columns, with bit-identical voxels, the
parts' own blocks cover the whole scene once, and the merged raycast meets
the parity bar against the whole scene's (on the tiny sequence) or comes
close to it (room: rays that graze a slab boundary may refine to a slightly
different point).  The merge rule is pinned on constructed maps.
"""

import numpy as np
import pytest

import oracle
from synth import kinect_workload, tiny_workload
from tests.parity_util import camera_depth, compare_raycast, key_of


def fuse_parts(w, n, width, frames):
    full = oracle.Scene(**w.params)
    parts = [oracle.Scene(**w.params) for _ in range(n)]
    for i, p in enumerate(parts):
        p.set_shard(n, i, width)
    ia = w.intr.as_array()
    for k in frames:
        f = w.frame(k)
        for sc in [full] + parts:
            sc.allocate(f.depth, ia, f.T_wc)
            sc.integrate(f.depth, ia, f.T_wc)
    return full, parts


def kept(bx, n, i, width):
    return any(oracle.slab_owner(bx + d, n, width) == i for d in (-1, 0, 1))


def test_slab_owner_is_floor_division_modulo():
    assert [oracle.slab_owner(x, 3, 4) for x in range(-9, 9)] == \
        [((x // 4) % 3) for x in range(-9, 9)]
    assert oracle.slab_owner(-1, 2, 8) == 1 and oracle.slab_owner(-8, 2, 8) == 1 and oracle.slab_owner(-9, 2, 8) == 0
    with pytest.raises(ValueError):
        oracle.Scene(**tiny_workload(n_frames=1).params).set_shard(2, 2, 8)
    with pytest.raises(ValueError):
        oracle.Scene(**tiny_workload(n_frames=1).params).set_shard(2, 0, 1)


@pytest.mark.parametrize("n,width", [(2, 4), (3, 2)])
def test_parts_hold_the_whole_scene_columns_bit_for_bit(n, width):
    w = tiny_workload()
    full, parts = fuse_parts(w, n, width, range(w.n_frames))
    cf, Ff, Wf = full.export()
    index = {k: j for j, k in enumerate(key_of(cf).tolist())}
    owned = []
    for i, p in enumerate(parts):
        c, F, Wt = p.export()
        keys = key_of(c).tolist()
        want = {k for k, bx in zip(key_of(cf).tolist(), cf[:, 0]) if kept(int(bx), n, i, width)}
        assert set(keys) == want
        for j, k in enumerate(keys):
            assert np.array_equal(F[j], Ff[index[k]]) and np.array_equal(Wt[j], Wf[index[k]])
        owned += [k for k, bx in zip(keys, c[:, 0]) if oracle.slab_owner(int(bx), n, width) == i]
    assert sorted(owned) == sorted(index)  # every block owned by exactly one part


def test_merged_raycast_meets_the_bar_on_the_tiny_sequence():
    w = tiny_workload()
    full, parts = fuse_parts(w, 2, 4, range(w.n_frames))
    f = w.frame(w.n_frames - 1)
    H, W = f.depth.shape
    ia = w.intr.as_array()
    vf, nf = full.raycast(W, H, ia, f.T_wc)
    maps = [p.raycast(W, H, ia, f.T_wc) for p in parts]
    vm, nm = oracle.merge_raycasts(np.stack([m[0] for m in maps]), np.stack([m[1] for m in maps]), f.T_wc)
    rep = compare_raycast(vm, nm, vf, nf, f.T_wc)
    assert rep["pass_frac"] >= 0.999 and rep["hit_agree"] == 1.0
    # each part reports only hits in its own columns
    inv_s = 1.0 / w.params["voxel_size"]
    for i, (v, _) in enumerate(maps):
        hit = v[..., 3] > 0
        bx = np.floor(v[hit][:, 0] * inv_s + 0.5).astype(np.int64) >> 3
        assert all(oracle.slab_owner(int(b), 2, 4) == i for b in bx)


def test_merged_raycast_close_to_the_whole_scene_in_the_room():
    """640x480 room, two parts of 8-block slabs: the merged map agrees with the
    whole scene's within the parity tolerance on >= 99.8% of pixels (the
    differences sit on rays that cross a slab boundary just before a grazing
    surface)."""
    w = kinect_workload()
    full, parts = fuse_parts(w, 2, 8, range(0, 6))
    f = w.frame(5)
    H, W = f.depth.shape
    ia = w.intr.as_array()
    vf, nf = full.raycast(W, H, ia, f.T_wc)
    maps = [p.raycast(W, H, ia, f.T_wc) for p in parts]
    vm, nm = oracle.merge_raycasts(np.stack([m[0] for m in maps]), np.stack([m[1] for m in maps]), f.T_wc)
    hf, hm = vf[..., 3] > 0, vm[..., 3] > 0
    assert np.mean(hf == hm) >= 0.999
    zf, zm = camera_depth(vf, f.T_wc), camera_depth(vm, f.T_wc)
    ok = (~hf & ~hm) | (hf & hm & (np.abs(zf - zm) <= 5e-4))
    assert np.mean(ok) >= 0.998


def test_merge_takes_the_nearest_hit_and_the_lower_part_on_ties():
    T = np.eye(4, dtype=np.float32)
    T[:3, 3] = [0.1, -0.2, 0.3]
    H, W = 2, 3
    v = np.zeros((3, H, W, 4), np.float32)
    n = np.zeros((3, H, W, 4), np.float32)

    def put(k, y, x, z):
        v[k, y, x] = [0.1 + 0.01 * x, -0.2 + 0.01 * y, 0.3 + z, 1.0]  # camera depth z
        n[k, y, x] = [0.0, 0.0, -1.0, 1.0 + k]  # w tags the part

    put(0, 0, 0, 2.0); put(1, 0, 0, 1.5); put(2, 0, 0, 3.0)   # part 1 nearest
    put(2, 0, 1, 0.7)                                          # only part 2
    put(0, 1, 0, 1.25); put(1, 1, 0, 1.25)                     # tie: part 0
    put(1, 1, 2, 4.0); put(2, 1, 2, 0.5)                       # part 2 nearest
    vm, nm = oracle.merge_raycasts(v, n, T)
    assert nm[0, 0, 3] == 2.0 and nm[0, 1, 3] == 3.0 and nm[1, 0, 3] == 1.0 and nm[1, 2, 3] == 3.0
    assert np.array_equal(vm[0, 0], v[1, 0, 0]) and np.array_equal(vm[1, 2], v[2, 1, 2])
    assert not vm[0, 2].any() and not nm[1, 1].any()          # no part hits: zeros
