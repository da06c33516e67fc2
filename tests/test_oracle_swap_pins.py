"""Pins of the oracle's swapping (Sec. 5).

The paper keeps the active part of the map in device memory and the rest in
a host block store with one slot per hash entry; a swapped-out block keeps its
entry (marked as not in device memory), transfers go through buffers of fixed
size, and data the device integrated while a block's host data was away is
fused with that data afterwards (the secondary integration).  Readings
(recorded with the others in the design notes): the fusion is the weighted
mean of the two voxels with the clamped weight sum, a side that has not
observed the voxel (weight 0) contributing nothing; at most K blocks move per
call, taken bucket by bucket and, within a chain, in ascending key order;
blocks leave the device once no allocation segment has met them for `idle`
allocations.  Each test checks the oracle against something other than
itself: fusions with exact closed-form results, a brute-force ordering of the
exported hash table, a run without swapping, and the table's own invariants.
"""

import numpy as np
import pytest

import oracle
from synth import tiny_workload
from synth.scenes import Intrinsics
from tests.test_oracle_pins import scene_params


def _keys(coords):
    return {tuple(int(v) for v in c) for c in coords}


def _by_key(coords, *arrays):
    return {tuple(int(v) for v in c): tuple(a[i] for a in arrays) for i, c in enumerate(coords)}


def _packed(x, y, z):
    return (x & 0xFFFF) | ((y & 0xFFFF) << 16) | ((z & 0xFFFF) << 32)


def _to_host_then_back(sc, b, sdf_h, w_h, sdf_d, w_d):
    """Block b holds (sdf_h, w_h) when it is swapped out; it is met again and
    its new device block is set to (sdf_d, w_d) before the fusion."""
    sc.set_block(b, sdf_h, w_h)
    sc.swap_enable(64, idle_frames=0)
    assert sc.swap_out() == 1
    assert sc.swap_counters()["swapped_out"] == 1
    sc.set_block(b, sdf_d, w_d)  # meets the swapped-out key: new device block, host data waiting
    assert sc.swap_counters()["waiting"] == 1
    assert sc.swap_in() == 1
    c, F, W = sc.export()
    assert _keys(c) == {tuple(b)}
    return F[0], W[0]


def test_fusion_closed_forms():
    """(W_d F_d + W_h F_h) / (W_d + W_h) with weight min(W_d + W_h, max_w), on
    values whose results are exact; one-sided voxels keep that side's value."""
    sdf_h = np.zeros(512, np.float32)
    w_h = np.zeros(512, np.float32)
    sdf_d = np.zeros(512, np.float32)
    w_d = np.zeros(512, np.float32)
    # voxel 0: both observed, exact mean
    sdf_d[0], w_d[0], sdf_h[0], w_h[0] = 0.5, 1, -0.25, 3
    # voxel 1: weight sum above max_w = 100 is clamped; the mean is exact
    sdf_d[1], w_d[1], sdf_h[1], w_h[1] = 0.5, 96, -0.5, 32
    # voxel 2: host never observed it: device value kept bit for bit
    sdf_d[2], w_d[2], sdf_h[2], w_h[2] = 0.1, 3, 0.7, 0
    # voxel 3: device has not observed it yet: host value taken bit for bit
    sdf_d[3], w_d[3], sdf_h[3], w_h[3] = 1.0, 0, 0.1, 7
    # voxel 4: neither observed it
    sdf_d[4], w_d[4], sdf_h[4], w_h[4] = 1.0, 0, 1.0, 0
    # voxel 5: a third-value mean that is exact in binary: (2*0.75 + 6*0.25)/8
    sdf_d[5], w_d[5], sdf_h[5], w_h[5] = 0.75, 2, 0.25, 6
    sc = oracle.Scene(**scene_params())
    F, W = _to_host_then_back(sc, (1, 2, 3), sdf_h, w_h, sdf_d, w_d)
    assert F[0] == -0.0625 and W[0] == 4
    assert F[1] == 0.25 and W[1] == 100
    assert F[2] == np.float32(0.1) and W[2] == 3
    assert F[3] == np.float32(0.1) and W[3] == 7
    assert F[4] == 1.0 and W[4] == 0
    assert F[5] == 0.375 and W[5] == 8
    assert sc.swap_counters() == dict(host_data=0, swapped_out=0, waiting=0, moved_in=1, moved_out=1)


def test_block_waiting_for_its_host_data_stays_on_the_device():
    """A block met again while its host data waits for the secondary fusion
    is no swap-out candidate, however idle (its device copy would overwrite
    the waiting data): swap_out moves nothing until swap_in has fused it, and
    the fusion then gives the closed-form mean of both."""
    sc = oracle.Scene(**scene_params())
    b = (1, 2, 3)
    sc.set_block(b, np.full(512, -0.25, np.float32), np.full(512, 3.0, np.float32))
    sc.swap_enable(64, idle_frames=0)
    assert sc.swap_out() == 1
    sc.set_block(b, np.full(512, 0.5, np.float32), np.full(512, 1.0, np.float32))
    assert sc.swap_counters()["waiting"] == 1
    assert sc.swap_out() == 0
    assert sc.swap_counters()["waiting"] == 1
    assert sc.swap_in() == 1
    c, F, W = sc.export()
    assert _keys(c) == {b}
    assert np.all(F[0] == -0.0625) and np.all(W[0] == 4)   # (1 * 0.5 + 3 * -0.25) / 4
    assert sc.swap_out() == 1                              # fused: a candidate again


def test_round_trip_restores_the_block():
    """Out to the host, met again, fused into an empty device block: the
    block comes back bit for bit (every device weight is 0)."""
    rng = np.random.default_rng(5)
    sdf = rng.uniform(-1, 1, 512).astype(np.float32)
    w = rng.integers(0, 100, 512).astype(np.float32)
    sc = oracle.Scene(**scene_params())
    F, W = _to_host_then_back(sc, (-4, 0, 7), sdf, w, np.ones(512, np.float32), np.zeros(512, np.float32))
    assert np.array_equal(F[w > 0], sdf[w > 0]) and np.array_equal(W, w)
    assert np.all(F[w == 0] == 1.0)


def test_transfers_are_bounded_and_taken_in_bucket_then_key_order():
    """With idle 0 every block in device memory is a candidate; each call moves
    exactly min(K, candidates) blocks, the first K of the brute-force order
    (bucket, packed key) over the exported table.  A small table makes long
    chains."""
    p = scene_params(num_buckets=1 << 4, num_excess=1 << 10)
    sc = oracle.Scene(**p)
    rng = np.random.default_rng(11)
    keys = set()
    while len(keys) < 300:
        keys.add(tuple(int(v) for v in rng.integers(-40, 40, 3)))
    for b in sorted(keys):
        sc.set_block(b, 0.5, 1.0)
    K = 37
    sc.swap_enable(K, idle_frames=0)
    moved = set()
    while True:
        E = sc.entries()
        resident = [tuple(int(v) for v in e[:3]) for e in E if e[4] >= 0]
        order = sorted(resident, key=lambda k: (oracle.hash_index(*k, p["num_buckets"]), _packed(*k)))
        n = sc.swap_out()
        assert n == min(K, len(resident))
        if n == 0:
            break
        c, _, _, _ = sc.swap_export_host()
        now = _keys(c)
        assert now - moved == set(order[:n])
        moved = now
    assert moved == keys
    assert sc.num_allocated == 0
    assert sc.swap_counters()["swapped_out"] == len(keys)


def test_met_key_reuses_its_entry():
    """A swapped-out key met again is not inserted a second time: same entry
    index, no excess slot used, the key once in the table."""
    p = scene_params(num_buckets=1 << 3, num_excess=1 << 8)
    sc = oracle.Scene(**p)
    keys = [(i, -i, 2 * i) for i in range(40)]
    for b in keys:
        sc.set_block(b, 0.25, 2.0)
    E0 = sc.entries()
    used0 = sc.excess_used
    sc.swap_enable(1000, idle_frames=0)
    assert sc.swap_out() == len(keys)
    assert np.all(sc.entries()[:, 4] < 0)
    for b in keys[::3]:
        sc.set_block(b, 0.25, 2.0)
    E1 = sc.entries()
    assert sc.excess_used == used0
    assert np.array_equal(E1[:, :4], E0[:, :4])
    seen = [tuple(e[:3]) for e in E1 if e[4] >= -1]
    assert len(seen) == len(set(seen)) == len(keys)
    assert sc.swap_counters()["waiting"] == len(keys[::3])


def _plane_frames(intr):
    """Two fixed views: the identity pose facing the plane z = +1, and the
    pose turned by 180 degrees about y facing z = -1 (each plane is behind the
    camera in the other view, so neither view updates the other's blocks)."""
    d = np.full((intr.height, intr.width), 1.0, np.float32)
    T1 = np.eye(4, dtype=np.float32)
    T2 = np.diag([-1.0, 1.0, -1.0, 1.0]).astype(np.float32)
    return [(d, T1), (d, T2)]


@pytest.mark.parametrize("K", [1 << 20, 4096])
def test_swapping_is_transparent_when_nothing_it_holds_is_observed(K):
    """Alternating the two views, with unbounded or large K and idle 1: each
    view's blocks leave the device when the other view is fused and come back
    (and are fused with their host data before integration) when it returns.
    Device plus host store equal a run without swapping, bit for bit, and the
    device holds exactly the current view's blocks."""
    intr = Intrinsics(64, 48, 60.0, 60.0, 31.5, 23.5)
    ia = intr.as_array()
    p = scene_params()
    a, b = oracle.Scene(**p), oracle.Scene(**p)
    b.swap_enable(K, idle_frames=1)
    frames = _plane_frames(intr)
    view_keys = []
    for k in range(6):
        d, T = frames[k % 2]
        a.allocate(d, ia, T)
        a.integrate(d, ia, T)
        b.allocate(d, ia, T)
        b.swap_in()
        b.integrate(d, ia, T)
        b.swap_out()
        ca, Fa, Wa = a.export()
        cb, Fb, Wb = b.export()
        ch, Fh, Wh, st = b.swap_export_host()
        if k < 2:
            view_keys.append(_keys(cb))
        assert _keys(cb) == view_keys[k % 2]
        assert not (_keys(cb) & _keys(ch)) and _keys(cb) | _keys(ch) == _keys(ca)
        assert np.all(st == oracle.Scene.SW_HOST)
        ref = _by_key(ca, Fa, Wa)
        for key, (F, W) in list(_by_key(cb, Fb, Wb).items()) + list(_by_key(ch, Fh, Wh).items()):
            assert np.array_equal(F, ref[key][0]) and np.array_equal(W, ref[key][1])
    assert view_keys[0] and view_keys[1] and not (view_keys[0] & view_keys[1])


def test_bounded_swap_in_defers_the_fusion():
    """With K smaller than the blocks waiting, the rest keep waiting (their
    device blocks go on integrating) and are fused by later calls; the key
    sets of device and host stay disjoint and together equal a run without
    swapping."""
    w = tiny_workload(n_frames=8)
    p = dict(w.params)
    ia = w.intr.as_array()
    a, b = oracle.Scene(**p), oracle.Scene(**p)
    K = 16
    b.swap_enable(K, idle_frames=1)
    waited = 0
    for k in list(range(8)) + list(range(0, 8, 2)):  # the revisit meets many swapped-out blocks at once
        f = w.frame(k)
        a.allocate(f.depth, ia, f.T_wc)
        a.integrate(f.depth, ia, f.T_wc)
        b.allocate(f.depth, ia, f.T_wc)
        before = b.swap_counters()["waiting"]
        n_in = b.swap_in()
        assert n_in == min(K, before)
        waited = max(waited, before - n_in)
        b.integrate(f.depth, ia, f.T_wc)
        assert b.swap_out() <= K
        cb = _keys(b.export()[0])
        ch, _, _, st = b.swap_export_host()
        # waiting blocks have both a device block and host data
        both = _keys(ch[st == oracle.Scene.SW_MERGE])
        assert both <= cb
        assert not (cb & _keys(ch[st == oracle.Scene.SW_HOST]))
        assert cb | _keys(ch) == _keys(a.export()[0])
    assert waited > 0  # the bound was reached at least once


def test_swapped_out_blocks_return_to_the_free_list():
    """A full block array swapped out is free again: as many new keys fit,
    and the swapped-out ones come back into the freed blocks too."""
    p = scene_params(num_blocks=64)
    sc = oracle.Scene(**p)
    first = [(i, 0, 0) for i in range(64)]
    for b in first:
        sc.set_block(b, 0.5, 1.0)
    assert sc.num_allocated == 64 and sc.status == 0
    sc.swap_enable(1000, idle_frames=0)
    assert sc.swap_out() == 64 and sc.num_allocated == 0
    for i in range(64):
        sc.set_block((i, 1, 0), 0.25, 2.0)
    assert sc.num_allocated == 64 and sc.status == 0
    assert sc.swap_out() == 64
    for b in first:
        sc.set_block(b, 0.75, 3.0)  # met again: fresh blocks, host data waiting
    assert sc.num_allocated == 64 and sc.status == 0 and sc.swap_counters()["waiting"] == 64
