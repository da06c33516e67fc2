"""Swapping (Sec. 5) on the GPU against the oracle.

Both sides run the paper's swapping pipeline per frame (allocation, swap-in,
integration, raycast, swap-out) with the same transfer bound and idle rule.
The selection order (bucket, then key) depends only on the set of keys, and
the fusion is written with the same rounded operations on both sides, so the
device volume, the host store and the per-entry swap states must agree bit
for bit, compared by block coordinates (block indices and excess slots come
from atomics).  Cases: the tiny sequence with a revisit and a tight bound
(fusions deferred), a small hash table with long chains, learned (float)
weights, a Kinect-scale run, a round trip against a run without swapping, a
reset, a block array too small even with swapping, and argument errors.
"""

import numpy as np
import pytest

import oracle
from synth import kinect_workload, large_workload, tiny_workload
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


def _by_key(coords, *arrays):
    return {tuple(int(v) for v in c): tuple(a[i] for a in arrays) for i, c in enumerate(coords)}


def compare_host(g, o):
    """Host stores and swap states of GPU scene g and oracle scene o."""
    cg, Fg, Wg, Sg = g.swap_export_host()
    co, Fo, Wo, So = o.swap_export_host()
    a, b = _by_key(cg, Fg, Wg, Sg), _by_key(co, Fo, Wo, So)
    assert set(a) == set(b), "host key sets differ: %d only on GPU, %d only in oracle" % (
        len(set(a) - set(b)), len(set(b) - set(a)))
    for k, (F, W, S) in a.items():
        Fo_, Wo_, So_ = b[k]
        assert S == So_, k
        assert np.array_equal(F, Fo_) and np.array_equal(W, Wo_), k
    return len(a)


def compare_counters(g, o):
    cg, co = g.swap_counters(), o.swap_counters()
    for k in ("host_data", "swapped_out", "waiting", "moved_in", "moved_out"):
        assert cg[k] == co[k], (k, cg, co)
    return cg


def run(itm, w, frames, K, idle, params=None, wpx=None, raycast_every=0):
    import torch
    p = dict(params or w.params)
    g, o = itm.Scene(**p), oracle.Scene(**p)
    g.swap_enable(K, idle)
    o.swap_enable(K, idle)
    ia = w.intr.as_array()
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    V = torch.zeros((w.intr.height, w.intr.width, 4), dtype=torch.float32, device="cuda")
    N = torch.zeros_like(V)
    deferred = 0
    for step, k in enumerate(frames):
        f = w.frame(k)
        D = dev(f.depth)
        g.allocate(D, ci, f.T_wc)
        o.allocate(f.depth, ia, f.T_wc)
        waiting = o.swap_counters()["waiting"]
        g.swap_in()
        deferred = max(deferred, waiting - o.swap_in())
        if wpx is None:
            g.integrate(D, ci, f.T_wc)
            o.integrate(f.depth, ia, f.T_wc)
        else:
            W = wpx(k, f.depth.shape)
            g.integrate(D, ci, f.T_wc, wpx=dev(W))
            o.integrate(f.depth, ia, f.T_wc, W)
        if raycast_every and step % raycast_every == 0:
            g.raycast(ci, f.T_wc, V, N)
            vo, no = o.raycast(w.intr.width, w.intr.height, ia, f.T_wc)
            compare_raycast(V.cpu().numpy(), N.cpu().numpy(), vo, no, f.T_wc)
        g.swap_out()
        o.swap_out()
        assert g.status() == 0
        compare_volumes(g.export(), o.export())
        compare_counters(g, o)
    n_host = compare_host(g, o)
    return g, o, deferred, n_host


def test_tiny_sequence_with_revisit_and_tight_bound(itm):
    w = tiny_workload(n_frames=8)
    frames = list(range(8)) + list(range(0, 8, 2))
    g, o, deferred, n_host = run(itm, w, frames, K=16, idle=1, raycast_every=3)
    c = g.swap_counters()
    assert deferred > 0 and c["moved_out"] > 100 and c["moved_in"] > 0 and n_host > 0


def test_long_chains_and_idle_two(itm):
    w = tiny_workload(n_frames=8)
    p = dict(w.params, num_buckets=1 << 8, num_excess=1 << 13)
    frames = list(range(8)) + [1, 3, 5]
    g, o, _, n_host = run(itm, w, frames, K=40, idle=2, params=p)
    assert g.swap_counters()["moved_out"] > 40 and n_host > 0


def test_learned_weights(itm):
    w = tiny_workload(n_frames=6)
    rng = np.random.default_rng(9)

    def wpx(k, shape):
        W = rng.uniform(0.05, 1.0, size=shape).astype(np.float32)
        W[rng.uniform(size=shape) < 0.1] = 0.0
        return W

    p = dict(w.params, weight_mode=1)
    g, o, _, n_host = run(itm, w, list(range(6)) + [0, 2], K=24, idle=1, params=p, wpx=wpx)
    assert g.swap_counters()["moved_in"] > 0


def test_kinect_scale(itm):
    w = kinect_workload(seed=4)
    frames = list(range(0, 40, 4)) + [0, 4]
    g, o, _, n_host = run(itm, w, frames, K=2048, idle=1, raycast_every=5)
    c = g.swap_counters()
    assert c["moved_out"] > 2048 and c["moved_in"] > 0


def test_large_corridor_window(itm):
    """The corridor at 2 mm with 2^22 buckets (the large configuration's
    table) and a device block array of 2^18 blocks: frames 40 apart, so
    every frame brings ~80k new blocks and the blocks left behind move out."""
    w = large_workload()
    p = dict(w.params, num_blocks=1 << 18)
    g, o, _, n_host = run(itm, w, [0, 40, 80], K=1 << 16, idle=1, params=p, raycast_every=2)
    c = g.swap_counters()
    assert c["moved_out"] > 10000 and n_host > 10000


def test_round_trip_equals_run_without_swapping(itm):
    """Everything out (idle 0), then the same frame again: every block comes
    back through reactivation and fusion into empty device blocks, so the
    volume equals a run that never swapped, bit for bit."""
    import torch
    w = tiny_workload(n_frames=3)
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    a, b = itm.Scene(**w.params), itm.Scene(**w.params)
    b.swap_enable(1 << 16, idle_frames=0)
    for k in range(3):
        f = w.frame(k)
        D = dev(f.depth)
        for sc in (a, b):
            sc.allocate(D, ci, f.T_wc)
            sc.integrate(D, ci, f.T_wc)
    b.swap_out()
    assert b.export()[0].shape[0] == 0
    n_host = b.swap_counters()["swapped_out"]
    f = w.frame(2)
    D = dev(f.depth)
    b.allocate(D, ci, f.T_wc)
    b.swap_in()
    ca = a.export()
    cb = b.export()
    touched = set(map(tuple, cb[0].tolist()))
    ref = _by_key(ca[0], ca[1], ca[2])
    got = _by_key(cb[0], cb[1], cb[2])
    for key in touched:
        assert np.array_equal(got[key][0], ref[key][0]) and np.array_equal(got[key][1], ref[key][1])
    c = b.swap_counters()
    assert c["moved_in"] == len(touched) and c["swapped_out"] == n_host - len(touched)
    torch.cuda.synchronize()


def test_invalid_arguments(itm):
    w = tiny_workload(n_frames=1)
    g = itm.Scene(**w.params)
    with pytest.raises(itm.ItmError):
        g.swap_in()
    with pytest.raises(itm.ItmError):
        g.swap_out()
    with pytest.raises(itm.ItmError):
        g.swap_enable(0, 1)
    with pytest.raises(itm.ItmError):
        g.swap_enable(16, -1)
    g.swap_enable(16, 1)
    with pytest.raises(itm.ItmError):
        g.swap_enable(16, 1)
    assert g.swap_counters() == dict(host_data=0, swapped_out=0, waiting=0, moved_in=0, moved_out=0)
    c, F, W, S = g.swap_export_host()
    assert len(c) == 0


def test_reset_clears_swapping_and_the_run_starts_over(itm):
    """itm_scene_reset with swapping on: every entry back to "in device
    memory" with nothing on the host, counters at 0; the same frames then
    give what a fresh oracle gives."""
    w = tiny_workload(n_frames=5)
    g, o, _, _ = run(itm, w, list(range(5)), K=16, idle=1)
    assert g.swap_counters()["swapped_out"] > 0
    g.reset()
    c = g.swap_counters()
    assert c["host_data"] == 0 and c["waiting"] == 0 and c["moved_in"] == 0 and c["moved_out"] == 0
    assert g.export()[0].shape[0] == 0 and len(g.swap_export_host()[0]) == 0
    o2 = oracle.Scene(**w.params)
    o2.swap_enable(16, 1)
    ia = w.intr.as_array()
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    for k in range(5):
        f = w.frame(k)
        D = dev(f.depth)
        g.allocate(D, ci, f.T_wc)
        g.swap_in()
        g.integrate(D, ci, f.T_wc)
        g.swap_out()
        o2.allocate(f.depth, ia, f.T_wc)
        o2.swap_in()
        o2.integrate(f.depth, ia, f.T_wc)
        o2.swap_out()
    assert g.status() == 0
    compare_volumes(g.export(), o2.export())
    compare_host(g, o2)
    compare_counters(g, o2)


def test_block_array_too_small_even_with_swapping_is_reported(itm):
    """A frame that meets more blocks than the device array holds fills it
    whatever swapping moves out: the status says so (which blocks made it in
    is then up to the order of the atomics, so only the status is compared)."""
    w = tiny_workload(n_frames=2)
    p = dict(w.params, num_blocks=256)
    g, o = itm.Scene(**p), oracle.Scene(**p)
    g.swap_enable(64, 1)
    o.swap_enable(64, 1)
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    f = w.frame(0)
    g.allocate(dev(f.depth), ci, f.T_wc)
    g.swap_in()
    g.swap_out()
    o.allocate(f.depth, w.intr.as_array(), f.T_wc)
    assert itm.ERRORS.get(g.status()) == "ITM_ERR_VBA_FULL"
    assert o.status & oracle.ST_VBA_FULL
    assert g.stats()["allocated_blocks"] <= 256
