"""Colour voxels (Sec. 3.1) on the GPU against the oracle.

Both sides fuse the same seeded RGB frames, seen by a colour camera with its
own resolution, intrinsics and a rigid offset from the depth camera, with the
same rounded operations, so the colour voxels must agree bit for bit
(compared by block coordinates), as must the depth volume and the colour of
the raycast's hits.  Cases: the tiny sequence, three Kinect-scale frames,
argument errors.
"""

import numpy as np
import pytest

import oracle
from synth import kinect_workload, tiny_workload
from tests.parity_util import compare_volumes

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


def _d2c():
    """A colour camera 2 cm to the side, slightly turned (about 1 degree)."""
    c, s = np.cos(np.radians(1.0)), np.sin(np.radians(1.0))
    T = np.eye(4)
    T[:3, :3] = [[c, 0, s], [0, 1, 0], [-s, 0, c]]
    T[:3, 3] = [0.02, -0.01, 0.005]
    return T.astype(np.float32)


def _compare_colour(g, o):
    cg, Cg = g.export_colour()
    co, Co = o.export_colour()
    a = {tuple(int(x) for x in k): Cg[i] for i, k in enumerate(cg)}
    b = {tuple(int(x) for x in k): Co[i] for i, k in enumerate(co)}
    assert set(a) == set(b)
    bad = [k for k in a if not np.array_equal(a[k], b[k])]
    assert not bad, (len(bad), bad[:3])
    return sum(int((v[:, 3] > 0).sum()) for v in a.values())


def _run(itm, w, frames, colour_size, seed):
    import torch
    Wc, Hc = colour_size
    fxc = w.intr.fx * Wc / w.intr.width
    cc = itm.make_intrinsics(Wc, Hc, fxc, fxc, (Wc - 1) / 2.0, (Hc - 1) / 2.0)
    cca = np.array([fxc, fxc, (Wc - 1) / 2.0, (Hc - 1) / 2.0], np.float32)
    T = _d2c()
    g, o = itm.Scene(**w.params), oracle.Scene(**w.params)
    g.colour_enable()
    o.colour_enable()
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    ia = w.intr.as_array()
    rng = np.random.default_rng(seed)
    for k in frames:
        f = w.frame(k)
        rgb = rng.integers(0, 256, size=(Hc, Wc, 3), dtype=np.uint8)
        D = dev(f.depth)
        g.allocate(D, ci, f.T_wc)
        g.integrate_colour(D, ci, f.T_wc, dev(rgb), cc, T)
        o.allocate(f.depth, ia, f.T_wc)
        o.integrate_colour(f.depth, ia, f.T_wc, rgb, cca, T)
    assert g.status() == 0
    compare_volumes(g.export(), o.export())
    coloured = _compare_colour(g, o)
    # colour of the raycast's hits, from the GPU's own vertex map on both sides
    V = torch.zeros((w.intr.height, w.intr.width, 4), dtype=torch.float32, device="cuda")
    N = torch.zeros_like(V)
    g.raycast(ci, f.T_wc, V, N)
    out = torch.zeros((w.intr.height, w.intr.width, 4), dtype=torch.uint8, device="cuda")
    g.colour_at(V, out)
    torch.cuda.synchronize()
    vh = V.cpu().numpy()
    want = o.colour_at(vh)
    assert np.array_equal(out.cpu().numpy(), want)
    hits = vh[..., 3] > 0
    return coloured, float(np.mean(want[hits][:, 3] > 0)) if hits.any() else 0.0


def test_tiny_sequence_colour_equals_oracle(itm):
    w = tiny_workload()
    coloured, hit_coloured = _run(itm, w, range(w.n_frames), (200, 150), seed=11)
    assert coloured > 10000 and hit_coloured > 0.9


def test_kinect_scale_colour_equals_oracle(itm):
    w = kinect_workload(seed=4)
    coloured, hit_coloured = _run(itm, w, [0, 3, 6], (640, 480), seed=12)
    assert coloured > 100000 and hit_coloured > 0.9


def test_colour_arguments(itm):
    import torch
    w = tiny_workload(n_frames=1)
    g = itm.Scene(**w.params)
    ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
    D = torch.zeros((w.intr.height, w.intr.width), dtype=torch.float32, device="cuda")
    rgb = torch.zeros((w.intr.height, w.intr.width, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(itm.ItmError):  # colour off
        g.integrate_colour(D, ci, np.eye(4), rgb, ci)
    g.colour_enable()
    with pytest.raises(itm.ItmError):  # twice
        g.colour_enable()
    with pytest.raises(itm.ItmError):  # colour and swapping exclude each other
        g.swap_enable(16, 1)
    learned = itm.Scene(**dict(w.params, weight_mode=1))
    with pytest.raises(itm.ItmError):
        learned.colour_enable()
    sw = itm.Scene(**w.params)
    sw.swap_enable(16, 1)
    with pytest.raises(itm.ItmError):
        sw.colour_enable()
    bad = np.eye(4)
    bad[0, 0] = np.nan
    with pytest.raises(itm.ItmError):
        g.integrate_colour(D, ci, np.eye(4), rgb, ci, bad)
