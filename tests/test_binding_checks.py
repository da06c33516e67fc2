"""The Scene wrapper checks every buffer before it calls the library (CPU).

A host tensor, a numpy array, the wrong dtype, a strided view or a buffer
smaller than the intrinsics ask for raises ItmError(ITM_ERR_ARG) in Python,
so no such pointer reaches a kernel; valid buffers pass through unchanged.
The library calls are replaced by stubs here, and a tensor subclass stands in
for a CUDA tensor (this host has no GPU).
"""

import numpy as np
import pytest
import torch

import paper_1708_00783_gb300 as itm


class FakeCuda(torch.Tensor):
    @property
    def is_cuda(self):
        return True


def cuda_like(*shape, dtype=torch.float32):
    return torch.zeros(*shape, dtype=dtype).as_subclass(FakeCuda)


CALLS = ("itm_allocate", "itm_integrate", "itm_integrate_weighted", "itm_raycast", "itm_process_frame",
         "itm_integrate_colour", "itm_colour_at")


@pytest.fixture()
def scene(monkeypatch):
    reached = []
    for name in CALLS:
        monkeypatch.setattr(itm, name, lambda *a, _n=name, **k: reached.append(_n))
    sc = object.__new__(itm.Scene)
    sc.handle = 1
    sc.params = {}
    sc.reached = reached
    yield sc
    sc.handle = None


H, W = 12, 16
INTR = itm.make_intrinsics(W, H, 20.0, 20.0, 7.5, 5.5)
T = np.eye(4)


def test_valid_buffers_reach_the_library(scene):
    d = cuda_like(H, W)
    v, n = cuda_like(H, W, 4), cuda_like(H, W, 4)
    scene.allocate(d, INTR, T)
    scene.integrate(d, INTR, T)
    scene.integrate(d, INTR, T, wpx=cuda_like(H, W))
    scene.raycast(INTR, T, v, n)
    scene.process(d, INTR, T)
    scene.process(d, INTR, T, v, n)
    scene.integrate_colour(d, INTR, T, cuda_like(H, W, 3, dtype=torch.uint8), INTR)
    scene.colour_at(v, cuda_like(H, W, 4, dtype=torch.uint8))
    scene.allocate(123456, INTR, T)  # a raw device address passes as is
    assert scene.reached == ["itm_allocate", "itm_integrate", "itm_integrate_weighted", "itm_raycast",
                             "itm_process_frame", "itm_process_frame", "itm_integrate_colour", "itm_colour_at",
                             "itm_allocate"]


@pytest.mark.parametrize("bad, why", [
    (torch.zeros(H, W), "not on a CUDA device"),
    (np.zeros((H, W), np.float32), "CUDA tensor is needed"),
    (cuda_like(H, W, dtype=torch.float64), "dtype"),
    (cuda_like(W, 2 * H)[:, ::2], "not contiguous"),
    (cuda_like(H, W - 1), "at least"),
])
def test_bad_depth_refused_before_the_library(scene, bad, why):
    for call in (lambda: scene.allocate(bad, INTR, T), lambda: scene.integrate(bad, INTR, T),
                 lambda: scene.process(bad, INTR, T)):
        with pytest.raises(itm.ItmError, match=why) as e:
            call()
        assert e.value.code == itm.ITM_ERR_ARG
    assert scene.reached == []


def test_bad_maps_and_colour_buffers_refused(scene):
    d, v = cuda_like(H, W), cuda_like(H, W, 4)
    cases = [
        lambda: scene.raycast(INTR, T, cuda_like(H, W, 3), v),               # vertex map too small
        lambda: scene.raycast(INTR, T, v, torch.zeros(H, W, 4)),             # normal map on the host
        lambda: scene.process(d, INTR, T, v, cuda_like(H, W, 4, dtype=torch.float16)),
        lambda: scene.integrate(d, INTR, T, wpx=cuda_like(H, W, dtype=torch.uint8)),
        lambda: scene.integrate_colour(d, INTR, T, cuda_like(H, W, 3), INTR),  # float RGB
        lambda: scene.integrate_colour(d, INTR, T, cuda_like(H, W, 2, dtype=torch.uint8), INTR),
        lambda: scene.colour_at(cuda_like(5, 3), cuda_like(5, 4, dtype=torch.uint8)),  # 15 floats: no whole point
        lambda: scene.colour_at(v, cuda_like(H, W, 2, dtype=torch.uint8)),
    ]
    for c in cases:
        with pytest.raises(itm.ItmError) as e:
            c()
        assert e.value.code == itm.ITM_ERR_ARG
    assert scene.reached == []


def test_batch_items_checked():
    """make_batch_items (and so itm_batch_run given tuples) checks each
    item's depth and map buffers the same way."""
    d, v = cuda_like(H, W), cuda_like(H, W, 4)
    arr = itm.make_batch_items([(1, d, INTR, T, v, cuda_like(H, W, 4)), (2, d, INTR, T, None, None)])
    assert len(arr) == 2 and arr[1].vertex_dev is None
    for bad in [(1, torch.zeros(H, W), INTR, T, v, v), (1, d, INTR, T, cuda_like(H, W), v),
                (1, d, INTR, T, v, cuda_like(H, W, 4, dtype=torch.float64))]:
        with pytest.raises(itm.ItmError) as e:
            itm.make_batch_items([(2, d, INTR, T, None, None), bad])
        assert e.value.code == itm.ITM_ERR_ARG and "batch item 1" in str(e.value)


def test_noalloc_call_checks_its_buffers(monkeypatch):
    """itm_frame_blocks_noalloc checks depth, coords and count like the Scene
    calls do: a host or numpy buffer, the wrong dtype or too small a buffer
    never reaches the library."""
    reached = []

    class Lib:
        def itm_frame_blocks_noalloc(self, *a):
            reached.append(a)
            return 0

    monkeypatch.setattr(itm, "_lib", Lib())
    d, coords, count = cuda_like(H, W), cuda_like(8, 3, dtype=torch.int16), cuda_like(1, dtype=torch.int32)
    itm.itm_frame_blocks_noalloc(d, INTR, T, 0.01, 0.04, 0.2, 5.0, coords, 8, count, stream=0)
    assert len(reached) == 1
    bad_calls = [
        (torch.zeros(H, W), coords, 8, count),                    # host depth
        (np.zeros((H, W), np.float32), coords, 8, count),         # numpy depth
        (cuda_like(H, W, dtype=torch.float64), coords, 8, count),  # wrong dtype
        (cuda_like(H, W - 1), coords, 8, count),                  # smaller than the image
        (d, cuda_like(8, 3, dtype=torch.int32), 8, count),        # coords dtype
        (d, coords, 9, count),                                    # cap beyond coords
        (d, coords, 8, cuda_like(1, dtype=torch.int64)),          # count dtype
        (d, coords, 8, torch.zeros(1, dtype=torch.int32)),        # host count
    ]
    for depth, c, cap, n in bad_calls:
        with pytest.raises(itm.ItmError) as e:
            itm.itm_frame_blocks_noalloc(depth, INTR, T, 0.01, 0.04, 0.2, 5.0, c, cap, n, stream=0)
        assert e.value.code == itm.ITM_ERR_ARG
    assert len(reached) == 1
