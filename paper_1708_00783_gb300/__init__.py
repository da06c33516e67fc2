"""GB300-native hashed-TSDF reconstruction core (InfiniTAM v3, Sec. 3-4).

Python binding of ``libitm.so``: the functions below carry the names of the
C ABI declared in ``include/itm.h`` and only marshal arguments (device
pointers of torch tensors, host structs, the current CUDA stream).  Every
step of the per-frame path runs in the library's CUDA kernels; there is no
CPU fallback: importing this package fails when the library is missing.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

_HERE = os.path.dirname(os.path.abspath(__file__))
# ITM_CHECK_BOUNDS=1 selects the bounds-checked debug build (built by
# build.build(checked=True)); the default is the release library
LIB_PATH = _build_mod.LIB_CHECKED if os.environ.get("ITM_CHECK_BOUNDS") == "1" else _build_mod.LIB

ITM_OK = 0
ERRORS = {1: "ITM_ERR_ARG", 2: "ITM_ERR_CUDA", 3: "ITM_ERR_HASH_FULL", 4: "ITM_ERR_VBA_FULL",
          5: "ITM_ERR_RANGE", 6: "ITM_ERR_TIMEOUT", 7: "ITM_ERR_OVERFLOW", 8: "ITM_ERR_TOO_LARGE",
          9: "ITM_ERR_SINGULAR", 10: "ITM_ERR_BOUNDS"}
(ITM_ERR_ARG, ITM_ERR_CUDA, ITM_ERR_HASH_FULL, ITM_ERR_VBA_FULL, ITM_ERR_RANGE, ITM_ERR_TIMEOUT, ITM_ERR_OVERFLOW,
 ITM_ERR_TOO_LARGE, ITM_ERR_SINGULAR, ITM_ERR_BOUNDS) = range(1, 11)
ITM_NOALLOC_MAX_BLOCKS = 1 << 21
ITM_NOALLOC_RANGE = 1 << 30      # count bit: a pixel left the int16 block range
ITM_NOALLOC_OVERFLOW = -(1 << 31)  # count bit 31 (a negative count): the fixed set overflowed
ITM_MLP_FEATURES, ITM_MLP_HIDDEN, ITM_MLP_PARAMS = 52, 64, 7617
ITM_MLP_PACKED_BYTES, ITM_MLP_SCRATCH_PER_SAMPLE = 17168, 257
ITM_BATCH_STAGES = 6
ITM_BATCH_KNOBS = 3
ITM_COMBINED_MAX = 16
ITM_ICP_SUMS = 29
ITM_ICP_WORK_DOUBLES = ITM_ICP_SUMS * 1025
ITM_TRACK_MAX_LEVELS = 8
ST_HASH_FULL, ST_VBA_FULL, ST_RANGE, ST_TIMEOUT, ST_OVERFLOW = 0x1, 0x2, 0x4, 0x8, 0x10


class ItmError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__("%s failed: %s (%d)" % (what, ERRORS.get(code, "?"), code))
        self.code = code


class itm_intrinsics(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class itm_scene_params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("mu", ctypes.c_float), ("max_w", ctypes.c_int),
                ("num_buckets", ctypes.c_int), ("num_excess", ctypes.c_int), ("num_blocks", ctypes.c_int),
                ("z_min", ctypes.c_float), ("z_max", ctypes.c_float), ("weight_mode", ctypes.c_int)]


class itm_batch_item(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("depth_dev", ctypes.c_void_p), ("intr", itm_intrinsics),
                ("T_wc", ctypes.c_float * 16), ("vertex_dev", ctypes.c_void_p), ("normal_dev", ctypes.c_void_p)]


class itm_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("allocated_blocks", ctypes.c_int32),
                ("excess_used", ctypes.c_int32), ("visible_blocks", ctypes.c_int32),
                ("last_requests", ctypes.c_int32), ("last_overflow", ctypes.c_int32),
                ("updated_voxels", ctypes.c_uint64), ("visited_voxels", ctypes.c_uint64),
                ("frames", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class itm_swap_counters(ctypes.Structure):
    _fields_ = [("host_data", ctypes.c_int64), ("swapped_out", ctypes.c_int64), ("waiting", ctypes.c_int64),
                ("moved_in", ctypes.c_int64), ("moved_out", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = [
    "itm_scene_create", "itm_scene_destroy", "itm_scene_reset", "itm_allocate", "itm_integrate",
    "itm_integrate_weighted", "itm_raycast", "itm_process_frame", "itm_depth_u16_to_f32",
    "itm_scene_stats", "itm_scene_status", "itm_scene_export", "itm_scene_export_table",
    "itm_scene_import", "itm_hash_index", "itm_version", "itm_frame_blocks_noalloc", "itm_raycast_range",
    "itm_mlp_pack", "itm_conf_weights", "itm_conf_features", "itm_mlp_loss_grad", "itm_mlp_adam",
    "itm_batch_create", "itm_batch_destroy", "itm_batch_run", "itm_batch_set_tuning", "itm_batch_get_tuning",
    "itm_batch_set_schedule", "itm_batch_get_schedule",
    "itm_batch_set_graph", "itm_swap_enable", "itm_swap_in", "itm_swap_out", "itm_swap_get_counters",
    "itm_swap_export_host", "itm_colour_enable", "itm_integrate_colour", "itm_colour_at", "itm_scene_export_colour",
]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libitm.so is not built (%s); run paper_1708_00783_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    fp16 = ctypes.POINTER(ctypes.c_float)
    sp = ctypes.POINTER(itm_scene_params)
    ip = ctypes.POINTER(itm_intrinsics)
    sig = {
        "itm_scene_create": (I, [sp, ctypes.POINTER(P)]),
        "itm_scene_destroy": (I, [P]),
        "itm_scene_reset": (I, [P, P]),
        "itm_allocate": (I, [P, P, ip, fp16, P]),
        "itm_integrate": (I, [P, P, ip, fp16, P]),
        "itm_integrate_weighted": (I, [P, P, P, ip, fp16, P]),
        "itm_raycast": (I, [P, ip, fp16, P, P, P]),
        "itm_process_frame": (I, [P, P, ip, fp16, P, P, P]),
        "itm_allocate_u16": (I, [P, P, P, ip, fp16, P]),
        "itm_process_frame_u16": (I, [P, P, P, ip, fp16, P, P, P]),
        "itm_depth_u16_to_f32": (I, [P, P, ctypes.c_int64, P]),
        "itm_scene_stats": (I, [P, ctypes.POINTER(itm_stats)]),
        "itm_scene_status": (I, [P]),
        "itm_scene_export": (I, [P, P, P, P, I, ctypes.POINTER(I)]),
        "itm_scene_export_table": (I, [P, P]),
        "itm_scene_import": (I, [P, P, P, P, I]),
        "itm_hash_index": (ctypes.c_uint32, [I, I, I, I]),
        "itm_version": (ctypes.c_char_p, []),
        "itm_frame_blocks_noalloc": (I, [P, ip, fp16, F, F, F, F, P, I, P, P]),
        "itm_raycast_range": (I, [P, ip, fp16, P, P, P]),
        "itm_raycast_combined": (I, [ctypes.POINTER(P), fp16, I, ip, fp16, P, P, P]),
        "itm_depth_halve": (I, [P, I, I, P, P]),
        "itm_mesh": (I, [P, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), P]),
        "itm_mesh_case_table": (I, [P, P]),
        "itm_scene_set_shard": (I, [P, I, I, I]),
        "itm_raycast_merge": (I, [P, P, I, ip, fp16, P, P, P]),
        "itm_icp_reduce": (I, [P, ip, fp16, P, P, ip, fp16, F, P, P]),
        "itm_icp_step": (I, [ctypes.POINTER(ctypes.c_double), fp16, ctypes.POINTER(ctypes.c_double)]),
        "itm_track_scratch_bytes": (ctypes.c_size_t, [I, I, I]),
        "itm_track_depth": (I, [P, ip, I, ctypes.POINTER(I), fp16, P, P, ip, fp16, fp16, ctypes.POINTER(I), P, P]),
        "itm_mlp_pack": (I, [P, P, P]),
        "itm_conf_weights": (I, [P, ip, F, P, P, P]),
        "itm_process_frame_weighted": (I, [P, P, P, P, ip, fp16, P, P, P]),
        "itm_conf_features": (I, [P, ip, F, P, I, P, P]),
        "itm_mlp_loss_grad": (I, [P, P, P, I, P, P, P, P]),
        "itm_mlp_adam": (I, [P, P, P, P, I, F, P]),
        "itm_batch_create": (I, [I, ctypes.POINTER(P)]),
        "itm_batch_destroy": (I, [P]),
        "itm_batch_run": (I, [P, ctypes.POINTER(itm_batch_item), I, P]),
        "itm_batch_set_tuning": (I, [P, ctypes.POINTER(I), I]),
        "itm_batch_get_tuning": (I, [P, ctypes.POINTER(I), I]),
        "itm_batch_set_schedule": (I, [P, ctypes.POINTER(I), I]),
        "itm_batch_get_schedule": (I, [P, ctypes.POINTER(I), I]),
        "itm_batch_set_graph": (I, [P, I]),
        "itm_swap_enable": (I, [P, I, I]),
        "itm_swap_in": (I, [P, P]),
        "itm_swap_out": (I, [P, P]),
        "itm_swap_get_counters": (I, [P, ctypes.POINTER(itm_swap_counters)]),
        "itm_swap_export_host": (I, [P, P, P, P, P, I, ctypes.POINTER(I)]),
        "itm_colour_enable": (I, [P]),
        "itm_integrate_colour": (I, [P, P, ip, fp16, P, ip, fp16, P]),
        "itm_colour_at": (I, [P, P, ctypes.c_int64, P, P]),
        "itm_scene_export_colour": (I, [P, P, P, I, ctypes.POINTER(I)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    return lib


_lib = _load()


def lib():
    return _lib


# ------------------------------------------------------------ marshalling

def _ptr(x):
    """Device (or host) address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _pose(T):
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float32).reshape(16))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _buffer(x, dtype, count, what):
    """A buffer on its way to the device: a contiguous CUDA tensor of `dtype`
    with at least `count` elements (None, or a raw device address given as an
    int, passes as is).  Anything else raises ItmError(ITM_ERR_ARG) before a
    pointer reaches a kernel."""
    if x is None or isinstance(x, int):
        return x
    import torch
    why = None
    if not isinstance(x, torch.Tensor):
        why = "a CUDA tensor is needed, not %s" % type(x).__name__
    elif not x.is_cuda:
        why = "the tensor is on %s, not on a CUDA device" % x.device
    elif x.dtype != dtype:
        why = "dtype %s, expected %s" % (x.dtype, dtype)
    elif not x.is_contiguous():
        why = "the tensor is not contiguous"
    elif x.numel() < count:
        why = "%d elements, at least %d needed" % (x.numel(), count)
    if why:
        raise ItmError(ITM_ERR_ARG, "%s (%s)" % (what, why))
    return x


def _f32_t():
    import torch
    return torch.float32


def _u8_t():
    import torch
    return torch.uint8


def _pixels(intr):
    return max(0, int(getattr(intr, "width", 0))) * max(0, int(getattr(intr, "height", 0)))


def make_intrinsics(width, height, fx, fy, cx, cy) -> itm_intrinsics:
    return itm_intrinsics(int(width), int(height), float(fx), float(fy), float(cx), float(cy))


def make_params(voxel_size, mu, max_w, num_buckets, num_excess, num_blocks, z_min, z_max,
                weight_mode=0, **_ignored) -> itm_scene_params:
    return itm_scene_params(float(voxel_size), float(mu), int(max_w), int(num_buckets), int(num_excess),
                            int(num_blocks), float(z_min), float(z_max), int(weight_mode))


CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")


def load_config(name_or_path):
    """A scene configuration from JSON: {"scene": the itm_scene_params fields,
    "intrinsics": the itm_intrinsics fields, ...}.  name_or_path is one of
    the files in configs/ by name ("tiny", "kinect", "large") or a path.
    Returns (a dict of scene parameters for Scene(**params), itm_intrinsics).
    Unknown or missing fields raise ValueError."""
    import json
    path = name_or_path
    if not os.path.exists(path):
        path = os.path.join(CONFIG_DIR, "%s.json" % name_or_path)
    with open(path) as f:
        cfg = json.load(f)
    scene, intr = dict(cfg.get("scene", {})), dict(cfg.get("intrinsics", {}))
    want_s = {n for n, _ in itm_scene_params._fields_}
    want_i = {n for n, _ in itm_intrinsics._fields_}
    scene.setdefault("weight_mode", 0)
    if set(scene) != want_s or set(intr) != want_i:
        raise ValueError("%s: scene fields %s and intrinsics fields %s expected" % (path, sorted(want_s),
                                                                                    sorted(want_i)))
    return scene, make_intrinsics(**intr)


def _check(code, what):
    if code != ITM_OK:
        raise ItmError(code, what)


# ------------------------------------------------------------ the C ABI

def itm_scene_create(params: itm_scene_params) -> int:
    h = ctypes.c_void_p()
    _check(_lib.itm_scene_create(ctypes.byref(params), ctypes.byref(h)), "itm_scene_create")
    return h.value


def itm_scene_destroy(scene):
    _check(_lib.itm_scene_destroy(scene), "itm_scene_destroy")


def itm_scene_reset(scene, stream=None):
    _check(_lib.itm_scene_reset(scene, _stream(stream)), "itm_scene_reset")


def itm_allocate(scene, depth, intr, T_wc, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_allocate(scene, _ptr(depth), ctypes.byref(intr), p, _stream(stream)), "itm_allocate")


def itm_integrate(scene, depth, intr, T_wc, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_integrate(scene, _ptr(depth), ctypes.byref(intr), p, _stream(stream)), "itm_integrate")


def itm_integrate_weighted(scene, depth, wpx, intr, T_wc, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_integrate_weighted(scene, _ptr(depth), _ptr(wpx), ctypes.byref(intr), p, _stream(stream)),
           "itm_integrate_weighted")


def itm_raycast(scene, intr, T_wc, vertex, normal, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_raycast(scene, ctypes.byref(intr), p, _ptr(vertex), _ptr(normal), _stream(stream)),
           "itm_raycast")


def itm_raycast_range(scene, intr, T_wc, zmin, zmax, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_raycast_range(scene, ctypes.byref(intr), p, _ptr(zmin), _ptr(zmax), _stream(stream)),
           "itm_raycast_range")


def itm_raycast_combined(scenes, submap_from_world, intr, T_wc, vertex, normal, stream=None):
    """Raycast of the combined map of posed submaps (scene handles and their
    submap-from-world poses, n x 4 x 4)."""
    n = len(scenes)
    arr = (ctypes.c_void_p * max(1, n))(*scenes)
    P = np.ascontiguousarray(np.asarray(submap_from_world, dtype=np.float32).reshape(-1))
    if P.size != 16 * n:
        raise ValueError("submap_from_world must hold one 4x4 pose per scene")
    a, p = _pose(T_wc)
    _check(_lib.itm_raycast_combined(arr, P.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n, ctypes.byref(intr), p,
                                     _ptr(vertex), _ptr(normal), _stream(stream)), "itm_raycast_combined")


def itm_mesh(scene, triangles=None, capacity=0, stream=None):
    """Marching-Cubes mesh into triangles (device float [capacity, 9]);
    returns the mesh's triangle count (raises ItmError(ITM_ERR_TOO_LARGE)
    when it exceeds capacity; use capacity 0 to count)."""
    n = ctypes.c_int64(0)
    r = _lib.itm_mesh(scene, _ptr(triangles), int(capacity), ctypes.byref(n), _stream(stream))
    if r == ITM_ERR_TOO_LARGE and capacity == 0:
        return n.value
    _check(r, "itm_mesh")
    return n.value


def itm_scene_set_shard(scene, parts, index, slab_blocks):
    """Make the scene part `index` of `parts` of a scene split by slabs of
    `slab_blocks` block columns (parts = 1: the whole scene)."""
    _check(_lib.itm_scene_set_shard(scene, int(parts), int(index), int(slab_blocks)), "itm_scene_set_shard")


def itm_raycast_merge(vertex_parts, normal_parts, parts, intr, T_wc, vertex, normal, stream=None):
    """Per pixel, the parts' hit nearest to the camera (device float4 maps:
    parts x height x width in, height x width out)."""
    n = _pixels(intr)
    _buffer(vertex_parts, _f32_t(), 4 * n * int(parts), "itm_raycast_merge: vertex_parts")
    _buffer(normal_parts, _f32_t(), 4 * n * int(parts), "itm_raycast_merge: normal_parts")
    _buffer(vertex, _f32_t(), 4 * n, "itm_raycast_merge: vertex")
    _buffer(normal, _f32_t(), 4 * n, "itm_raycast_merge: normal")
    a, p = _pose(T_wc)
    _check(_lib.itm_raycast_merge(_ptr(vertex_parts), _ptr(normal_parts), int(parts), ctypes.byref(intr), p,
                                  _ptr(vertex), _ptr(normal), _stream(stream)), "itm_raycast_merge")


def itm_mesh_case_table():
    """The Marching-Cubes case table of itm_mesh (host call): triangle counts
    uint8[256] and edge indices uint8[256, 5, 3]."""
    count = np.zeros(256, dtype=np.uint8)
    edges = np.zeros((256, 5, 3), dtype=np.uint8)
    _check(_lib.itm_mesh_case_table(count.ctypes.data, edges.ctypes.data), "itm_mesh_case_table")
    return count, edges


def itm_depth_halve(depth_in, width, height, depth_out, stream=None):
    _check(_lib.itm_depth_halve(_ptr(depth_in), int(width), int(height), _ptr(depth_out), _stream(stream)),
           "itm_depth_halve")


def itm_icp_reduce(depth, intr, T_g, vertex, normal, ref_intr, T_ref, dist_thresh, work, stream=None):
    a, p = _pose(T_g)
    b, q = _pose(T_ref)
    _check(_lib.itm_icp_reduce(_ptr(depth), ctypes.byref(intr), p, _ptr(vertex), _ptr(normal), ctypes.byref(ref_intr),
                               q, float(dist_thresh), _ptr(work), _stream(stream)), "itm_icp_reduce")


def itm_icp_step(sums, T):
    """Host Gauss-Newton step: (new T, step (6)); raises ItmError when the
    system has no unique solution."""
    s = np.ascontiguousarray(np.asarray(sums, dtype=np.float64).reshape(ITM_ICP_SUMS))
    a, p = _pose(T)
    a = a.copy()
    x = np.zeros(6)
    _check(_lib.itm_icp_step(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "itm_icp_step")
    return a.reshape(4, 4), x


def itm_track_scratch_bytes(width, height, levels):
    return int(_lib.itm_track_scratch_bytes(int(width), int(height), int(levels)))


def itm_track_depth(depth, intr, iters, dist_thresh, vertex, normal, ref_intr, T_ref, T_init, scratch, stream=None):
    """Coarse-to-fine depth tracking; iters[l], dist_thresh[l] per pyramid
    level (0 = input resolution).  Returns (T, steps)."""
    L = len(iters)
    it = (ctypes.c_int * L)(*[int(x) for x in iters])
    th = np.ascontiguousarray(np.asarray(dist_thresh, dtype=np.float32).reshape(L))
    b, q = _pose(T_ref)
    T = np.ascontiguousarray(np.asarray(T_init, dtype=np.float32).reshape(16)).copy()
    steps = ctypes.c_int(0)
    _check(_lib.itm_track_depth(_ptr(depth), ctypes.byref(intr), L, it, th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                _ptr(vertex), _ptr(normal), ctypes.byref(ref_intr), q,
                                T.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(steps), _ptr(scratch),
                                _stream(stream)), "itm_track_depth")
    return T.reshape(4, 4), steps.value


def itm_allocate_u16(scene, raw, depth, intr, T_wc, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_allocate_u16(scene, _ptr(raw), _ptr(depth), ctypes.byref(intr), p, _stream(stream)),
           "itm_allocate_u16")


def itm_process_frame_u16(scene, raw, depth, intr, T_wc, vertex=None, normal=None, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_process_frame_u16(scene, _ptr(raw), _ptr(depth), ctypes.byref(intr), p, _ptr(vertex),
                                      _ptr(normal), _stream(stream)), "itm_process_frame_u16")


def itm_process_frame(scene, depth, intr, T_wc, vertex=None, normal=None, stream=None):
    a, p = _pose(T_wc)
    _check(_lib.itm_process_frame(scene, _ptr(depth), ctypes.byref(intr), p, _ptr(vertex), _ptr(normal),
                                  _stream(stream)), "itm_process_frame")


def itm_depth_u16_to_f32(raw, out, n=None, stream=None):
    n = raw.numel() if n is None else n
    _check(_lib.itm_depth_u16_to_f32(_ptr(raw), _ptr(out), int(n), _stream(stream)), "itm_depth_u16_to_f32")


def itm_scene_stats(scene) -> dict:
    st = itm_stats()
    _check(_lib.itm_scene_stats(scene, ctypes.byref(st)), "itm_scene_stats")
    return st.as_dict()


def itm_scene_status(scene) -> int:
    return _lib.itm_scene_status(scene)


def itm_scene_export(scene, with_voxels=True):
    """(coords int16 [n,3], sdf float32 [n,512], w float32 [n,512]) in block
    array order (host numpy arrays)."""
    n = ctypes.c_int(0)
    _check(_lib.itm_scene_export(scene, None, None, None, 0, ctypes.byref(n)), "itm_scene_export")
    cnt = n.value
    coords = np.zeros((max(cnt, 1), 3), dtype=np.int16)
    sdf = np.zeros((max(cnt, 1), 512), dtype=np.float32) if with_voxels else None
    w = np.zeros((max(cnt, 1), 512), dtype=np.float32) if with_voxels else None
    _check(_lib.itm_scene_export(scene, coords.ctypes.data, sdf.ctypes.data if with_voxels else None,
                                 w.ctypes.data if with_voxels else None, cnt, ctypes.byref(n)), "itm_scene_export")
    if with_voxels:
        return coords[:cnt], sdf[:cnt], w[:cnt]
    return coords[:cnt], None, None


def itm_scene_export_table(scene, num_buckets, num_excess) -> np.ndarray:
    out = np.zeros((num_buckets + num_excess, 5), dtype=np.int32)
    _check(_lib.itm_scene_export_table(scene, out.ctypes.data), "itm_scene_export_table")
    return out


def itm_scene_import(scene, coords, sdf, w):
    coords = np.ascontiguousarray(coords, dtype=np.int16)
    sdf = np.ascontiguousarray(sdf, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    n = coords.shape[0]
    _check(_lib.itm_scene_import(scene, coords.ctypes.data, sdf.ctypes.data, w.ctypes.data, n), "itm_scene_import")


def itm_hash_index(x, y, z, num_buckets) -> int:
    return int(_lib.itm_hash_index(int(x), int(y), int(z), int(num_buckets)))


def itm_version() -> str:
    return _lib.itm_version().decode()


def itm_frame_blocks_noalloc(depth, intr, T_wc, voxel_size, mu, z_min, z_max, coords, cap, count, stream=None):
    """Blocks one depth frame touches, into caller buffers (coords: device
    int16 [cap, 3]; count: device int32 [1], the block count in its low 30
    bits with the ITM_NOALLOC_RANGE / ITM_NOALLOC_OVERFLOW flags); the library
    allocates nothing.  Every buffer is checked (device, dtype, contiguity,
    size) before the call."""
    import torch
    _buffer(depth, _f32_t(), _pixels(intr), "itm_frame_blocks_noalloc: depth")
    _buffer(coords, torch.int16, 3 * max(0, int(cap)), "itm_frame_blocks_noalloc: coords")
    _buffer(count, torch.int32, 1, "itm_frame_blocks_noalloc: count")
    a, p = _pose(T_wc)
    _check(_lib.itm_frame_blocks_noalloc(_ptr(depth), ctypes.byref(intr), p, float(voxel_size), float(mu),
                                         float(z_min), float(z_max), _ptr(coords), int(cap), _ptr(count),
                                         _stream(stream)), "itm_frame_blocks_noalloc")


def itm_mlp_pack(params, packed, stream=None):
    _check(_lib.itm_mlp_pack(_ptr(params), _ptr(packed), _stream(stream)), "itm_mlp_pack")


def itm_conf_weights(depth, intr, mu, packed, wpx, stream=None):
    _check(_lib.itm_conf_weights(_ptr(depth), ctypes.byref(intr), float(mu), _ptr(packed), _ptr(wpx),
                                 _stream(stream)), "itm_conf_weights")


def itm_process_frame_weighted(scene, depth, packed, wpx, intr, T_wc, vertex=None, normal=None, stream=None):
    """One learned-weight frame: the per-pixel weights beside the allocation,
    then the weighted integration and (with vertex) the raycast."""
    a, p = _pose(T_wc)
    _check(_lib.itm_process_frame_weighted(scene, _ptr(depth), _ptr(packed), _ptr(wpx), ctypes.byref(intr), p,
                                           _ptr(vertex), _ptr(normal), _stream(stream)), "itm_process_frame_weighted")


def itm_conf_features(depth, intr, mu, pixels, n, feat, stream=None):
    _check(_lib.itm_conf_features(_ptr(depth), ctypes.byref(intr), float(mu), _ptr(pixels), int(n), _ptr(feat),
                                  _stream(stream)), "itm_conf_features")


def itm_mlp_loss_grad(params, feat, labels, n, scratch, grad, loss, stream=None):
    _check(_lib.itm_mlp_loss_grad(_ptr(params), _ptr(feat), _ptr(labels), int(n), _ptr(scratch), _ptr(grad),
                                  _ptr(loss), _stream(stream)), "itm_mlp_loss_grad")


def itm_mlp_adam(params, grad, m, v, step, lr, stream=None):
    _check(_lib.itm_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), _stream(stream)),
           "itm_mlp_adam")


def itm_batch_create(max_items) -> int:
    h = ctypes.c_void_p()
    _check(_lib.itm_batch_create(int(max_items), ctypes.byref(h)), "itm_batch_create")
    return h.value


def itm_batch_destroy(batch):
    _check(_lib.itm_batch_destroy(batch), "itm_batch_destroy")


def make_batch_items(items):
    """items: iterable of (scene handle, depth tensor/pointer, itm_intrinsics,
    T_wc 4x4, vertex or None, normal or None)."""
    items = list(items)
    arr = (itm_batch_item * len(items))()
    for k, (scene, depth, intr, T, vtx, nrm) in enumerate(items):
        n = _pixels(intr)
        _buffer(depth, _f32_t(), n, "batch item %d: depth" % k)
        _buffer(vtx, _f32_t(), 4 * n, "batch item %d: vertex" % k)
        _buffer(nrm, _f32_t(), 4 * n, "batch item %d: normal" % k)
        arr[k].scene = scene
        arr[k].depth_dev = _ptr(depth)
        arr[k].intr = intr
        arr[k].T_wc[:] = [float(x) for x in np.asarray(T, dtype=np.float32).reshape(16)]
        arr[k].vertex_dev = _ptr(vtx)
        arr[k].normal_dev = _ptr(nrm)
    return arr


def itm_batch_run(batch, items, stream=None):
    """items: a ctypes array from make_batch_items, or the tuples it takes."""
    arr = items if isinstance(items, ctypes.Array) else make_batch_items(items)
    _check(_lib.itm_batch_run(batch, arr, len(arr), _stream(stream)), "itm_batch_run")


def itm_batch_set_tuning(batch, ctas_per_sm):
    a = (ctypes.c_int * ITM_BATCH_STAGES)(*[int(x) for x in ctas_per_sm])
    _check(_lib.itm_batch_set_tuning(batch, a, ITM_BATCH_STAGES), "itm_batch_set_tuning")


def itm_batch_set_schedule(batch, knobs):
    """[blocks per integration CTA (1, 2, 4), scattered enumeration walk (0/1),
    scattered raycast walk (0/1)]."""
    a = (ctypes.c_int * ITM_BATCH_KNOBS)(*[int(x) for x in knobs])
    _check(_lib.itm_batch_set_schedule(batch, a, ITM_BATCH_KNOBS), "itm_batch_set_schedule")


def itm_batch_get_schedule(batch):
    a = (ctypes.c_int * ITM_BATCH_KNOBS)()
    _check(_lib.itm_batch_get_schedule(batch, a, ITM_BATCH_KNOBS), "itm_batch_get_schedule")
    return list(a)


def itm_batch_get_tuning(batch):
    a = (ctypes.c_int * ITM_BATCH_STAGES)()
    _check(_lib.itm_batch_get_tuning(batch, a, ITM_BATCH_STAGES), "itm_batch_get_tuning")
    return list(a)


def itm_batch_set_graph(batch, use_graph):
    _check(_lib.itm_batch_set_graph(batch, int(bool(use_graph))), "itm_batch_set_graph")


# ------------------------------------------------------------ convenience

# ------------------------------------------------------ Sec. 3.1 colour voxels

def itm_colour_enable(scene):
    _check(_lib.itm_colour_enable(scene), "itm_colour_enable")


def itm_integrate_colour(scene, depth, intr, T_wc, rgb, intr_colour, T_d2c=None, stream=None):
    """rgb: device uint8 tensor [Hc, Wc, 3]; intr_colour: itm_intrinsics of
    the colour camera; T_d2c: depth-to-colour rigid map (identity if None)."""
    a, p = _pose(T_wc)
    b, q = _pose(np.eye(4, dtype=np.float32) if T_d2c is None else T_d2c)
    _check(_lib.itm_integrate_colour(scene, _ptr(depth), ctypes.byref(intr), p, _ptr(rgb), ctypes.byref(intr_colour),
                                     q, _stream(stream)), "itm_integrate_colour")


def itm_colour_at(scene, points, out, stream=None):
    """points: device float32 [..., 4]; out: device uint8 [..., 4]."""
    n = points.numel() // 4
    _check(_lib.itm_colour_at(scene, _ptr(points), int(n), _ptr(out), _stream(stream)), "itm_colour_at")


def itm_scene_export_colour(scene):
    """(coords int16 [n,3], rgbw uint8 [n,512,4]) in the order of itm_scene_export."""
    n = ctypes.c_int(0)
    _check(_lib.itm_scene_export_colour(scene, None, None, 0, ctypes.byref(n)), "itm_scene_export_colour")
    cnt = n.value
    coords = np.zeros((max(cnt, 1), 3), dtype=np.int16)
    rgbw = np.zeros((max(cnt, 1), 512, 4), dtype=np.uint8)
    _check(_lib.itm_scene_export_colour(scene, coords.ctypes.data, rgbw.ctypes.data, cnt, ctypes.byref(n)),
           "itm_scene_export_colour")
    return coords[:cnt], rgbw[:cnt]


# ------------------------------------------------------------ Sec. 5 swapping

SW_HOST, SW_MERGE = 1, 2


def itm_swap_enable(scene, transfer_blocks, idle_frames=1):
    _check(_lib.itm_swap_enable(scene, int(transfer_blocks), int(idle_frames)), "itm_swap_enable")


def itm_swap_in(scene, stream=None):
    _check(_lib.itm_swap_in(scene, _stream(stream)), "itm_swap_in")


def itm_swap_out(scene, stream=None):
    _check(_lib.itm_swap_out(scene, _stream(stream)), "itm_swap_out")


def itm_swap_get_counters(scene) -> dict:
    c = itm_swap_counters()
    _check(_lib.itm_swap_get_counters(scene, ctypes.byref(c)), "itm_swap_get_counters")
    return c.as_dict()


def itm_swap_export_host(scene, weight_mode=0):
    """(coords int16 [n,3], sdf float32 [n,512], w float32 [n,512], state
    int32 [n]) of the host slots of the entries with host data."""
    n = ctypes.c_int(0)
    _check(_lib.itm_swap_export_host(scene, None, None, None, None, 0, ctypes.byref(n)), "itm_swap_export_host")
    cnt = n.value
    coords = np.zeros((max(cnt, 1), 3), dtype=np.int16)
    sdf = np.zeros((max(cnt, 1), 512), dtype=np.float32)
    w = np.zeros((max(cnt, 1), 512), dtype=np.uint8 if weight_mode == 0 else np.float32)
    st = np.zeros(max(cnt, 1), dtype=np.int32)
    _check(_lib.itm_swap_export_host(scene, coords.ctypes.data, sdf.ctypes.data, w.ctypes.data, st.ctypes.data,
                                     cnt, ctypes.byref(n)), "itm_swap_export_host")
    return coords[:cnt], sdf[:cnt], w[:cnt].astype(np.float32), st[:cnt]


class Scene:
    """Owning wrapper of an itm_scene handle.  Its methods take torch CUDA
    tensors (float32 depth [H, W] and maps [H, W, 4], uint8 RGB [Hc, Wc, 3])
    and check device, dtype, contiguity and size against the intrinsics
    before calling the library."""

    def __init__(self, voxel_size, mu, max_w, num_buckets, num_excess, num_blocks, z_min, z_max,
                 weight_mode=0, **_ignored):
        self.params = dict(voxel_size=voxel_size, mu=mu, max_w=max_w, num_buckets=num_buckets,
                           num_excess=num_excess, num_blocks=num_blocks, z_min=z_min, z_max=z_max,
                           weight_mode=weight_mode)
        self.handle = itm_scene_create(make_params(**self.params))

    @classmethod
    def from_config(cls, name_or_path):
        """(Scene, itm_intrinsics) of a JSON configuration (load_config)."""
        params, intr = load_config(name_or_path)
        return cls(**params), intr

    def close(self):
        if getattr(self, "handle", None):
            itm_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_shard(self, parts, index, slab_blocks):
        """Make this scene part `index` of `parts` (see itm_scene_set_shard)."""
        itm_scene_set_shard(self.handle, parts, index, slab_blocks)

    def reset(self, stream=None):
        itm_scene_reset(self.handle, stream)

    def allocate(self, depth, intr, T_wc, stream=None):
        _buffer(depth, _f32_t(), _pixels(intr), "Scene.allocate: depth")
        itm_allocate(self.handle, depth, intr, T_wc, stream)

    def integrate(self, depth, intr, T_wc, stream=None, wpx=None):
        _buffer(depth, _f32_t(), _pixels(intr), "Scene.integrate: depth")
        _buffer(wpx, _f32_t(), _pixels(intr), "Scene.integrate: wpx")
        if wpx is None:
            itm_integrate(self.handle, depth, intr, T_wc, stream)
        else:
            itm_integrate_weighted(self.handle, depth, wpx, intr, T_wc, stream)

    def raycast(self, intr, T_wc, vertex, normal, stream=None):
        _buffer(vertex, _f32_t(), 4 * _pixels(intr), "Scene.raycast: vertex")
        _buffer(normal, _f32_t(), 4 * _pixels(intr), "Scene.raycast: normal")
        itm_raycast(self.handle, intr, T_wc, vertex, normal, stream)

    def process_weighted(self, depth, packed, wpx, intr, T_wc, vertex=None, normal=None, stream=None):
        """One learned-weight frame (weight_mode 1): see itm_process_frame_weighted."""
        import torch
        _buffer(depth, _f32_t(), _pixels(intr), "Scene.process_weighted: depth")
        _buffer(packed, torch.uint8, ITM_MLP_PACKED_BYTES, "Scene.process_weighted: packed")
        _buffer(wpx, _f32_t(), _pixels(intr), "Scene.process_weighted: wpx")
        _buffer(vertex, _f32_t(), 4 * _pixels(intr), "Scene.process_weighted: vertex")
        _buffer(normal, _f32_t(), 4 * _pixels(intr), "Scene.process_weighted: normal")
        itm_process_frame_weighted(self.handle, depth, packed, wpx, intr, T_wc, vertex, normal, stream)

    def process(self, depth, intr, T_wc, vertex=None, normal=None, stream=None):
        _buffer(depth, _f32_t(), _pixels(intr), "Scene.process: depth")
        _buffer(vertex, _f32_t(), 4 * _pixels(intr), "Scene.process: vertex")
        _buffer(normal, _f32_t(), 4 * _pixels(intr), "Scene.process: normal")
        itm_process_frame(self.handle, depth, intr, T_wc, vertex, normal, stream)

    def stats(self) -> dict:
        return itm_scene_stats(self.handle)

    def status(self) -> int:
        return itm_scene_status(self.handle)

    def export(self, with_voxels=True):
        return itm_scene_export(self.handle, with_voxels)

    def colour_enable(self):
        itm_colour_enable(self.handle)

    def integrate_colour(self, depth, intr, T_wc, rgb, intr_colour, T_d2c=None, stream=None):
        _buffer(depth, _f32_t(), _pixels(intr), "Scene.integrate_colour: depth")
        _buffer(rgb, _u8_t(), 3 * _pixels(intr_colour), "Scene.integrate_colour: rgb")
        itm_integrate_colour(self.handle, depth, intr, T_wc, rgb, intr_colour, T_d2c, stream)

    def colour_at(self, points, out, stream=None):
        _buffer(points, _f32_t(), 0, "Scene.colour_at: points")
        n = points.numel() if hasattr(points, "numel") else 0
        if n % 4:
            raise ItmError(ITM_ERR_ARG, "Scene.colour_at: points (not a multiple of 4 floats)")
        _buffer(out, _u8_t(), n, "Scene.colour_at: out")
        itm_colour_at(self.handle, points, out, stream)

    def export_colour(self):
        return itm_scene_export_colour(self.handle)

    def swap_enable(self, transfer_blocks, idle_frames=1):
        itm_swap_enable(self.handle, transfer_blocks, idle_frames)

    def swap_in(self, stream=None):
        itm_swap_in(self.handle, stream)

    def swap_out(self, stream=None):
        itm_swap_out(self.handle, stream)

    def swap_counters(self) -> dict:
        return itm_swap_get_counters(self.handle)

    def swap_export_host(self):
        return itm_swap_export_host(self.handle, self.params["weight_mode"])

    def export_table(self):
        return itm_scene_export_table(self.handle, self.params["num_buckets"], self.params["num_excess"])

    def import_blocks(self, coords, sdf, w):
        itm_scene_import(self.handle, coords, sdf, w)
