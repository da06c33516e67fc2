"""The OpenMP build of the oracle gives the single-threaded results (CPU).

The multi-threaded CPU baseline is the same C source compiled with -fopenmp:
integration in parallel over blocks, raycasts over image rows, allocation's
segment walks over rows with the insertions kept in row-major order.  Its
hash table, voxels, counts, maps, colour and swap state must be identical
byte for byte to the plain build's on the same inputs.
"""

import numpy as np
import pytest

import oracle
from synth import kinect_workload, tiny_workload


@pytest.fixture(scope="module")
def mt():
    try:
        oracle.build_threaded()
    except Exception as e:  # pragma: no cover - no OpenMP in this compiler
        pytest.skip("no OpenMP build: %s" % e)
    return oracle


def _same(a, b):
    assert a.status == b.status and a.num_allocated == b.num_allocated
    assert np.array_equal(a.entries(), b.entries())
    ca, sa, wa = a.export()
    cb, sb, wb = b.export()
    assert np.array_equal(ca, cb)
    assert np.array_equal(sa.view(np.uint32), sb.view(np.uint32)) and np.array_equal(wa, wb)


def _run(w, frames, threaded, colour=False, swap=None):
    sc = oracle.Scene(**w.params, threaded=threaded)
    if colour:
        sc.colour_enable()
    if swap:
        sc.swap_enable(*swap)
    ia = w.intr.as_array()
    rng = np.random.default_rng(5)
    out = []
    for k in frames:
        f = w.frame(k)
        sc.allocate(f.depth, ia, f.T_wc)
        if colour:
            rgb = rng.integers(0, 256, size=(w.intr.height, w.intr.width, 3), dtype=np.uint8)
            n = sc.integrate_colour(f.depth, ia, f.T_wc, rgb, ia)
        else:
            n = sc.integrate(f.depth, ia, f.T_wc)
        if swap:
            out.append((sc.swap_out(), sc.swap_in()))
        V, N = sc.raycast(w.intr.width, w.intr.height, ia, f.T_wc)
        out.append((n, V.tobytes(), N.tobytes()))
    return sc, out


def test_threads_reported(mt):
    assert mt.threads() >= 1


def test_tiny_sequence_identical(mt):
    w = tiny_workload()
    a, oa = _run(w, range(w.n_frames), False)
    b, ob = _run(w, range(w.n_frames), True)
    assert oa == ob
    _same(a, b)


def test_kinect_frames_identical_with_colour(mt):
    w = kinect_workload(seed=2, width=320, height=240)
    a, oa = _run(w, [0, 5, 10], False, colour=True)
    b, ob = _run(w, [0, 5, 10], True, colour=True)
    assert oa == ob
    _same(a, b)
    assert np.array_equal(a.export_colour()[1], b.export_colour()[1])


def test_swapping_and_overflow_identical(mt):
    """Swapping state and the status bits of a volume that runs out of blocks
    come out the same: the insertions happen in the same order."""
    w = kinect_workload(seed=3, width=320, height=240, n_frames=60)
    frames = list(range(0, 60, 6))
    a, oa = _run(w, frames, False, swap=(512, 1))
    b, ob = _run(w, frames, True, swap=(512, 1))
    assert oa == ob
    _same(a, b)
    assert a.swap_counters() == b.swap_counters()
    for x, y in zip(a.swap_export_host(), b.swap_export_host()):
        assert np.array_equal(x, y)
    small = dict(w.params, num_blocks=3000)
    wa, wb = oracle.Scene(**small), oracle.Scene(**small, threaded=True)
    f = w.frame(0)
    sa = wa.allocate(f.depth, w.intr.as_array(), f.T_wc)
    sb = wb.allocate(f.depth, w.intr.as_array(), f.T_wc)
    assert sa == sb and sa & oracle.ST_VBA_FULL
    _same(wa, wb)


def test_combined_raycast_identical(mt):
    w = tiny_workload(n_frames=4)
    ia = w.intr.as_array()
    scenes = []
    for threaded in (False, True):
        sc = oracle.Scene(**w.params, threaded=threaded)
        for k in range(4):
            f = w.frame(k)
            sc.allocate(f.depth, ia, f.T_wc)
            sc.integrate(f.depth, ia, f.T_wc)
        scenes.append(sc)
    P = np.eye(4, dtype=np.float32)[None]
    f = w.frame(2)
    Va, Na = oracle.raycast_combined([scenes[0]], P, w.intr.width, w.intr.height, ia, f.T_wc)
    Vb, Nb = oracle.raycast_combined([scenes[1]], P, w.intr.width, w.intr.height, ia, f.T_wc)
    assert np.array_equal(Va, Vb) and np.array_equal(Na, Nb)
