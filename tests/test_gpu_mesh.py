"""Marching-Cubes mesh (Sec. 4) on the GPU against the oracle.

The volumes are bit-identical on both sides, and both build every triangle
with the same float operations, so the meshes must be equal exactly: as
multisets of triangles, each triangle rotated to start at its smallest
vertex (its orientation kept).  Cases: the tiny sequence, a learned-weight
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


def test_tiny_sequence_mesh_equals_oracle(itm):
    w = tiny_workload()
    g, o = fuse(itm, w, range(w.n_frames))
    mg, mo = gpu_mesh(itm, g), o.mesh()
    assert len(mo) > 5000
    assert np.array_equal(canonical(mg), canonical(mo))


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
