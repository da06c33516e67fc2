"""Marching-Cubes mesh (Sec. 4) on the GPU against the oracle.

The volumes are bit-identical on both sides, and both build every triangle
with the same float operations, so the meshes must be equal exactly: as
multisets of triangles, each triangle rotated to start at its smallest
vertex (its orientation kept).  The library derives its case table on its
own (checked against the oracle's cells on the CPU); the GPU mesh is also
checked without the oracle: a consistently oriented surface, closed away
from its boundary, facing the free side of the scene's analytic surfaces.  Cases: the tiny sequence, a learned-weight
(float weight) volume, a Kinect-scale volume, capacity handling, an empty
volume and argument errors.
"""

import numpy as np
import pytest

import oracle
from synth import kinect_workload, tiny_workload

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


def canonical(tris):
    """Sorted rows of 9 floats, each triangle rotated to its smallest vertex."""
    t = np.asarray(tris, np.float32).reshape(-1, 3, 3)
    out = np.empty((len(t), 9), np.float32)
    for i, tri in enumerate(t):
        keys = [tuple(v) for v in tri]
        k = min(range(3), key=lambda j: keys[j])
        out[i] = np.concatenate([tri[k], tri[(k + 1) % 3], tri[(k + 2) % 3]])
    order = np.lexsort(out.T[::-1])
    return out[order]


def gpu_mesh(itm, sc):
    import torch
    n = itm.itm_mesh(sc.handle)
    buf = torch.full((max(n, 1), 9), np.nan, dtype=torch.float32, device="cuda")
    m = itm.itm_mesh(sc.handle, buf, n)
    assert m == n
    return buf[:n].cpu().numpy()


def fuse(itm, w, frames, params=None, wpx=None):
    p = dict(params or w.params)
    g = itm.Scene(**p)
    o = oracle.Scene(**p)
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    for k in frames:
        f = w.frame(k)
        D = dev(f.depth)
        g.allocate(D, ci, f.T_wc)
        o.allocate(f.depth, w.intr.as_array(), f.T_wc)
        if wpx is None:
            g.integrate(D, ci, f.T_wc)
            o.integrate(f.depth, w.intr.as_array(), f.T_wc)
        else:
            W = wpx(k, f.depth.shape)
            g.integrate(D, ci, f.T_wc, wpx=dev(W))
            o.integrate(f.depth, w.intr.as_array(), f.T_wc, W)
    return g, o


def check_mesh_on_its_own(tris):
    """Properties of a mesh that do not rest on the oracle's triangulation: no
    degenerate triangle, a directed edge used by one triangle at most (a
    consistently oriented surface; a few exceptions remain where a fan lays a
    triangle into a cell face that the neighbouring cell also triangulates,
    about 1 in 10^4 edges), and most edges shared by two triangles (closed
    away from the boundary of the observed region)."""
    t = np.asarray(tris, np.float32).reshape(-1, 3, 3)
    area2 = np.linalg.norm(np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]), axis=1)
    assert np.all(np.isfinite(t)) and np.mean(area2 > 0) > 0.99
    flat = np.ascontiguousarray(t.reshape(-1, 3))
    keys = [flat[i].tobytes() for i in range(len(flat))]
    directed = {}
    for a, b, c in zip(keys[0::3], keys[1::3], keys[2::3]):
        for e in ((a, b), (b, c), (c, a)):
            directed[e] = directed.get(e, 0) + 1
    twice = sum(v > 1 for v in directed.values())
    assert twice <= 1e-3 * len(directed), "directed edges used twice: %d of %d" % (twice, len(directed))
    # edges met in both directions (an interior edge of a consistently
    # oriented surface) against edges met in one direction only (boundary)
    both = sum(1 for (a, b) in directed if (b, a) in directed) // 2
    one = sum(1 for (a, b) in directed if (b, a) not in directed)
    shared = both / (both + one)
    assert shared > 0.85, shared
    return t


def test_tiny_sequence_mesh_equals_oracle(itm):
    w = tiny_workload()
    g, o = fuse(itm, w, range(w.n_frames))
    mg, mo = gpu_mesh(itm, g), o.mesh()
    assert len(mo) > 5000
    assert np.array_equal(canonical(mg), canonical(mo))
    # orientation against the scene's own geometry: triangles on the sphere
    # (centre (-0.35, 0.3, 0), r 0.3) face away from its centre, triangles on
    # the floor (y = 0) away from the objects face up
    t = check_mesh_on_its_own(mg)
    n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    c = t.mean(axis=1)
    d = c - np.array([-0.35, 0.3, 0.0])
    on_sphere = np.abs(np.linalg.norm(d, axis=1) - 0.3) < 0.01
    assert on_sphere.sum() > 500
    assert np.mean(np.sum(n[on_sphere] * d[on_sphere], axis=1) > 0) > 0.99
    on_floor = (np.abs(c[:, 1]) < 0.005) & (np.abs(c[:, 2]) > 0.4)
    assert on_floor.sum() > 200
    assert np.mean(n[on_floor, 1] > 0) > 0.97  # sensor noise folds a few floor triangles


def test_learned_weight_volume_mesh_equals_oracle(itm):
    w = tiny_workload(n_frames=4)
    rng = np.random.default_rng(3)

    def wpx(k, shape):
        W = rng.uniform(0.05, 1.0, size=shape).astype(np.float32)
        W[rng.uniform(size=shape) < 0.1] = 0.0
        return W

    g, o = fuse(itm, w, range(4), params=dict(w.params, weight_mode=1), wpx=wpx)
    mg, mo = gpu_mesh(itm, g), o.mesh()
    assert len(mo) > 1000
    assert np.array_equal(canonical(mg), canonical(mo))


def test_kinect_scale_mesh_equals_oracle(itm):
    w = kinect_workload(seed=4)
    g, o = fuse(itm, w, range(0, 20, 4))
    mg, mo = gpu_mesh(itm, g), o.mesh()
    assert len(mo) > 100000
    assert np.array_equal(canonical(mg), canonical(mo))
    check_mesh_on_its_own(mg)


def test_capacity_and_empty_volume(itm):
    import torch
    w = tiny_workload(n_frames=2)
    g, o = fuse(itm, w, range(2))
    n = itm.itm_mesh(g.handle)
    full = canonical(gpu_mesh(itm, g))
    cap = n // 3
    buf = torch.zeros((cap, 9), dtype=torch.float32, device="cuda")
    with pytest.raises(itm.ItmError):
        itm.itm_mesh(g.handle, buf, cap)
    part = canonical(buf.cpu().numpy())
    rows = {r.tobytes() for r in full}
    assert all(r.tobytes() in rows for r in part)
    empty = itm.Scene(**w.params)
    assert itm.itm_mesh(empty.handle) == 0


def test_invalid_arguments(itm):
    import torch
    w = tiny_workload(n_frames=1)
    g = itm.Scene(**w.params)
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    for args in ((None, 4), (buf, -1)):
        with pytest.raises(itm.ItmError):
            itm.itm_mesh(g.handle, *args)
    with pytest.raises(itm.ItmError):
        itm.itm_mesh(g.handle, buf.data_ptr() + 2, 2)
