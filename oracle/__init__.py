"""CPU oracle for the hashed-TSDF per-frame core (allocation, integration,
raycast) of InfiniTAM v3, Sec. 3-4.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg are the only callers.  The product path never
imports this package.  The arithmetic lives in ``itm_oracle.c`` (plain C,
single-threaded, fp32 with every operation rounded separately, as the paper's
listings are written in float); this module only marshals numpy arrays.
``Scene(..., threaded=True)`` runs the same source built with OpenMP (the
multi-threaded CPU baseline), whose results are identical.

Every function here is pinned by tests in ``tests/test_oracle_pins.py``,
``tests/test_oracle_conf_pins.py``, ``tests/test_oracle_combined_pins.py``,
``tests/test_oracle_swap_pins.py`` and ``tests/test_oracle_colour_pins.py``
against closed forms, brute force and analytic geometry; see the docstrings
there for which pin covers which step.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "itm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_LIB_MT = os.path.join(_LIB_DIR, "liboracle_omp.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

ST_HASH_FULL = 1
ST_VBA_FULL = 2
ST_RANGE = 4


def _compile(out: str, extra, force: bool) -> str:
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build."""
    return _compile(_LIB, [], force)


def build_threaded(force: bool = False) -> str:
    """The same source with OpenMP (liboracle_omp.so)."""
    return _compile(_LIB_MT, ["-fopenmp"], force)


_lib = None
_lib_mt = None


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _load_threaded():
    global _lib_mt
    if _lib_mt is None:
        _lib_mt = _bind(ctypes.CDLL(build_threaded()))
    return _lib_mt


def threads() -> int:
    """Threads the OpenMP build runs its parallel loops with."""
    return int(_load_threaded().orc_threads())


def _bind(lib):
    P = ctypes.c_void_p
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i16p = np.ctypeslib.ndpointer(np.int16, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
    lib.orc_hash_index.restype = ctypes.c_uint32
    lib.orc_hash_index.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32]
    lib.orc_scene_new.restype = P
    lib.orc_scene_new.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float]
    lib.orc_scene_free.argtypes = [P]
    lib.orc_allocate.restype = ctypes.c_int
    lib.orc_allocate.argtypes = [P, f32p, ctypes.c_int, ctypes.c_int, f32p, f32p]
    lib.orc_integrate.restype = ctypes.c_longlong
    lib.orc_integrate.argtypes = [P, f32p, ctypes.c_int, ctypes.c_int, f32p, f32p, P]
    lib.orc_raycast.restype = ctypes.c_int
    lib.orc_raycast.argtypes = [P, ctypes.c_int, ctypes.c_int, f32p, f32p, f32p, f32p]
    lib.orc_status.restype = ctypes.c_int
    lib.orc_status.argtypes = [P]
    lib.orc_num_allocated.restype = ctypes.c_int
    lib.orc_num_allocated.argtypes = [P]
    lib.orc_excess_used.restype = ctypes.c_int
    lib.orc_excess_used.argtypes = [P]
    lib.orc_export.restype = ctypes.c_int
    lib.orc_export.argtypes = [P, i16p, P, P, ctypes.c_int]
    lib.orc_entries.argtypes = [P, i32p]
    lib.orc_depth_u16_to_f32.argtypes = [u16p, f32p, ctypes.c_longlong]
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    lib.orc_bf16.restype = ctypes.c_float
    lib.orc_bf16.argtypes = [ctypes.c_float]
    lib.orc_conf_features.restype = ctypes.c_int
    lib.orc_conf_features.argtypes = [f32p, ctypes.c_int, ctypes.c_int, f32p, ctypes.c_float, ctypes.c_int,
                                      ctypes.c_int, f64p]
    lib.orc_mlp_forward.restype = ctypes.c_double
    lib.orc_mlp_forward.argtypes = [f32p, f64p, ctypes.c_int, P, P]
    lib.orc_mlp_loss_grad.restype = ctypes.c_double
    lib.orc_mlp_loss_grad.argtypes = [f32p, f64p, f32p, ctypes.c_int, ctypes.c_int, f64p]
    lib.orc_conf_weights.argtypes = [f32p, ctypes.c_int, ctypes.c_int, f32p, ctypes.c_float, f32p, f32p]
    lib.orc_set_block.restype = ctypes.c_int
    lib.orc_set_block.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, f32p, f32p]
    lib.orc_combined_value.restype = ctypes.c_float
    lib.orc_combined_value.argtypes = [P, f32p, ctypes.c_int, f32p, P]
    lib.orc_raycast_combined.restype = ctypes.c_int
    lib.orc_raycast_combined.argtypes = [P, f32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, f32p, f32p, f32p, f32p]
    I = ctypes.c_int
    lib.orc_depth_halve.argtypes = [f32p, I, I, f32p]
    lib.orc_icp_reduce.argtypes = [f32p, I, I, f32p, f32p, f32p, f32p, I, I, f32p, f32p, ctypes.c_float, f64p, P]
    lib.orc_icp_update.restype = I
    lib.orc_icp_update.argtypes = [f64p, f32p, P]
    i32p_ = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    lib.orc_mesh.restype = ctypes.c_longlong
    lib.orc_mesh.argtypes = [P, P, ctypes.c_longlong]
    lib.orc_cell_triangles.restype = I
    lib.orc_cell_triangles.argtypes = [f32p, i32p_]
    lib.orc_track.restype = I
    lib.orc_track.argtypes = [f32p, I, I, f32p, I, i32p_, f32p, f32p, f32p, I, I, f32p, f32p, f32p]
    lib.orc_swap_enable.restype = I
    lib.orc_swap_enable.argtypes = [P, I, I]
    lib.orc_swap_in.restype = I
    lib.orc_swap_in.argtypes = [P]
    lib.orc_swap_out.restype = I
    lib.orc_swap_out.argtypes = [P]
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    lib.orc_swap_counters.argtypes = [P, i64p]
    lib.orc_swap_export_host.restype = I
    lib.orc_swap_export_host.argtypes = [P, P, P, P, P, I]
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    lib.orc_colour_enable.restype = I
    lib.orc_colour_enable.argtypes = [P]
    lib.orc_integrate_colour.restype = ctypes.c_longlong
    lib.orc_integrate_colour.argtypes = [P, f32p, I, I, f32p, f32p, u8p, I, I, f32p, f32p]
    lib.orc_colour_at.argtypes = [P, f32p, ctypes.c_longlong, u8p]
    lib.orc_export_colour.restype = I
    lib.orc_export_colour.argtypes = [P, i16p, u8p, I]
    lib.orc_threads.restype = I
    lib.orc_threads.argtypes = []
    lib.orc_scene_set_shard.restype = I
    lib.orc_scene_set_shard.argtypes = [P, I, I, I]
    lib.orc_merge_raycasts.argtypes = [I, f32p, f32p, I, I, f32p, f32p, f32p]
    return lib


def hash_index(x: int, y: int, z: int, num_buckets: int) -> int:
    return int(_load().orc_hash_index(int(x), int(y), int(z), num_buckets - 1))


def depth_u16_to_f32(raw: np.ndarray) -> np.ndarray:
    raw = np.ascontiguousarray(raw, dtype=np.uint16)
    out = np.empty(raw.shape, dtype=np.float32)
    _load().orc_depth_u16_to_f32(raw.ravel(), out.ravel(), raw.size)
    return out


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


class Scene:
    """One hashed TSDF volume held by the oracle."""

    def __init__(self, voxel_size, mu, max_w, num_buckets, num_excess, num_blocks,
                 z_min, z_max, threaded=False, **_ignored):
        lib = self._lib = _load_threaded() if threaded else _load()
        self.p = lib.orc_scene_new(voxel_size, mu, int(max_w), int(num_buckets), int(num_excess),
                                   int(num_blocks), z_min, z_max)
        if not self.p:
            raise ValueError("invalid scene parameters")
        self.params = dict(voxel_size=voxel_size, mu=mu, max_w=max_w, num_buckets=num_buckets,
                           num_excess=num_excess, num_blocks=num_blocks, z_min=z_min, z_max=z_max)

    def __del__(self):
        if getattr(self, "p", None):
            self._lib.orc_scene_free(self.p)
            self.p = None

    def allocate(self, depth, intr, T_wc) -> int:
        d = _f32(depth)
        H, W = d.shape
        return self._lib.orc_allocate(self.p, d, W, H, _f32(intr), _f32(T_wc).ravel())

    def integrate(self, depth, intr, T_wc, wpx=None) -> int:
        d = _f32(depth)
        H, W = d.shape
        wp = None
        if wpx is not None:
            wpx = _f32(wpx)
            assert wpx.shape == d.shape
            wp = wpx.ctypes.data
        return int(self._lib.orc_integrate(self.p, d, W, H, _f32(intr), _f32(T_wc).ravel(), wp))

    def raycast(self, W, H, intr, T_wc):
        vtx = np.zeros((H, W, 4), dtype=np.float32)
        nrm = np.zeros((H, W, 4), dtype=np.float32)
        self._lib.orc_raycast(self.p, W, H, _f32(intr), _f32(T_wc).ravel(), vtx, nrm)
        return vtx, nrm

    def process(self, depth, intr, T_wc, raycast=True, wpx=None):
        """One frame of the per-frame core: allocate, integrate, raycast."""
        st = self.allocate(depth, intr, T_wc)
        n = self.integrate(depth, intr, T_wc, wpx)
        out = self.raycast(depth.shape[1], depth.shape[0], intr, T_wc) if raycast else None
        return st, n, out

    @property
    def status(self) -> int:
        return self._lib.orc_status(self.p)

    @property
    def num_allocated(self) -> int:
        return self._lib.orc_num_allocated(self.p)

    @property
    def excess_used(self) -> int:
        return self._lib.orc_excess_used(self.p)

    def set_shard(self, n, i, w):
        """Make this scene part i of n: block column x belongs to part
        floor(x / w) mod n; the part keeps its own columns and their x
        neighbours, and its raycast reports only hits in its own columns."""
        if self._lib.orc_scene_set_shard(self.p, int(n), int(i), int(w)) != 0:
            raise ValueError("invalid shard")

    def export(self, with_voxels=True):
        """(coords int16 [n,3], sdf float32 [n,512], w float32 [n,512]) in
        allocation order."""
        n = self.num_allocated
        coords = np.zeros((n, 3), dtype=np.int16)
        sdf = np.zeros((n, 512), dtype=np.float32) if with_voxels else None
        w = np.zeros((n, 512), dtype=np.float32) if with_voxels else None
        self._lib.orc_export(self.p, coords, sdf.ctypes.data if with_voxels else None,
                           w.ctypes.data if with_voxels else None, n)
        return coords, sdf, w

    def entries(self) -> np.ndarray:
        nb, ne = self.params["num_buckets"], self.params["num_excess"]
        out = np.zeros((nb + ne, 5), dtype=np.int32)
        self._lib.orc_entries(self.p, out)
        return out

    def mesh(self):
        """Marching-Cubes triangles of the zero level set: float32 [n, 3, 3]
        (three world-space vertices each, counter-clockwise seen from F > 0)."""
        n = int(self._lib.orc_mesh(self.p, None, 0))
        out = np.zeros((max(n, 1), 3, 3), dtype=np.float32)
        self._lib.orc_mesh(self.p, out.ctypes.data, n)
        return out[:n]

    # Sec. 3.1 colour voxels (readings in itm_oracle.c at colour_update)
    def colour_enable(self):
        if self._lib.orc_colour_enable(self.p) != 0:
            raise ValueError("colour already on")

    def integrate_colour(self, depth, intr, T_wc, rgb, intr_c, T_d2c=None) -> int:
        """Depth integration plus the colour of rgb (uint8 [Hc, Wc, 3]) seen
        by a camera with intrinsics intr_c (fx, fy, cx, cy) at T_d2c from the
        depth camera (identity when None)."""
        d = _f32(depth)
        H, W = d.shape
        rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
        Hc, Wc = rgb.shape[:2]
        T = np.eye(4, dtype=np.float32) if T_d2c is None else _f32(T_d2c)
        n = self._lib.orc_integrate_colour(self.p, d, W, H, _f32(intr), _f32(T_wc).ravel(), rgb.ravel(), Wc, Hc,
                                         _f32(intr_c), _f32(T).ravel())
        if n < 0:
            raise ValueError("colour is off")
        return int(n)

    def colour_at(self, pts):
        """r, g, b, colour weight (uint8 [..., 4]) of the voxel nearest each
        point (x, y, z, valid) of pts (float32 [..., 4])."""
        p = _f32(pts)
        out = np.zeros(p.shape[:-1] + (4,), dtype=np.uint8)
        self._lib.orc_colour_at(self.p, p.reshape(-1), p.size // 4, out.reshape(-1))
        return out

    def export_colour(self):
        """(coords int16 [n,3], rgbw uint8 [n,512,4]) in allocation order."""
        n = self.num_allocated
        coords = np.zeros((max(n, 1), 3), dtype=np.int16)
        rgbw = np.zeros((max(n, 1), 512, 4), dtype=np.uint8)
        self._lib.orc_export_colour(self.p, coords, rgbw.reshape(-1), n)
        return coords[:n], rgbw[:n]

    # Sec. 5 swapping (readings in itm_oracle.c above orc_swap_enable)
    SW_HOST, SW_MERGE = 1, 2

    def swap_enable(self, transfer_blocks, idle_frames=1):
        if self._lib.orc_swap_enable(self.p, int(transfer_blocks), int(idle_frames)) != 0:
            raise ValueError("swapping already on or invalid arguments")

    def swap_in(self) -> int:
        return int(self._lib.orc_swap_in(self.p))

    def swap_out(self) -> int:
        return int(self._lib.orc_swap_out(self.p))

    def swap_counters(self) -> dict:
        out = np.zeros(5, dtype=np.int64)
        self._lib.orc_swap_counters(self.p, out)
        return dict(host_data=int(out[0]), swapped_out=int(out[1]), waiting=int(out[2]),
                    moved_in=int(out[3]), moved_out=int(out[4]))

    def swap_export_host(self):
        """(coords int16 [n,3], sdf float32 [n,512], w float32 [n,512], state
        int32 [n]) of the blocks with host data, in entry order."""
        lib = self._lib
        n = int(lib.orc_swap_export_host(self.p, None, None, None, None, 0))
        coords = np.zeros((max(n, 1), 3), dtype=np.int16)
        sdf = np.zeros((max(n, 1), 512), dtype=np.float32)
        w = np.zeros((max(n, 1), 512), dtype=np.float32)
        st = np.zeros(max(n, 1), dtype=np.int32)
        lib.orc_swap_export_host(self.p, coords.ctypes.data, sdf.ctypes.data, w.ctypes.data, st.ctypes.data, n)
        return coords[:n], sdf[:n], w[:n], st[:n]

    def set_block(self, b, sdf, w):
        """Allocate block b (if missing) and set its 512 voxels (x + 8y + 64z)."""
        sdf = _f32(np.broadcast_to(np.asarray(sdf, dtype=np.float32), (512,)))
        w = _f32(np.broadcast_to(np.asarray(w, dtype=np.float32), (512,)))
        if self._lib.orc_set_block(self.p, int(b[0]), int(b[1]), int(b[2]), sdf, w) != 0:
            raise RuntimeError("block could not be allocated")


# ------------------------------------------------------------- combined map

def _lib_of(scenes):
    return scenes[0]._lib if scenes else _load()


def _scene_array(scenes):
    arr = (ctypes.c_void_p * max(1, len(scenes)))(*[sc.p for sc in scenes])
    return arr


def _poses(P, n):
    P = _f32(P).reshape(n, 4, 4)
    return np.ascontiguousarray(P.reshape(-1))


def combined_value(scenes, P, X):
    """Sec. 7.2 combined TSDF at world point X over submaps with
    submap-from-world poses P (n x 4 x 4): (value, weight sum)."""
    n = len(scenes)
    den = ctypes.c_float(0.0)
    v = _lib_of(scenes).orc_combined_value(_scene_array(scenes), _poses(P, n), n, _f32(X), ctypes.byref(den))
    return float(v), float(den.value)


def raycast_combined(scenes, P, W, H, intr, T_wc):
    """Raycast of the combined map of posed submaps: (vertex, normal) maps."""
    n = len(scenes)
    vtx = np.zeros((H, W, 4), dtype=np.float32)
    nrm = np.zeros((H, W, 4), dtype=np.float32)
    _lib_of(scenes).orc_raycast_combined(_scene_array(scenes), _poses(P, n) if n else np.zeros(16, np.float32),
                                         n, W, H, _f32(intr), _f32(T_wc).ravel(), vtx, nrm)
    return vtx, nrm


# ------------------------------------------------------- learned confidence

N_FEATURES = 52
N_HIDDEN = 64
N_PARAMS = N_HIDDEN * N_FEATURES + N_HIDDEN + N_HIDDEN * N_HIDDEN + N_HIDDEN + N_HIDDEN + 1


def bf16(x) -> np.ndarray:
    lib = _load()
    a = np.asarray(x, dtype=np.float32)
    return np.vectorize(lambda v: lib.orc_bf16(float(v)), otypes=[np.float32])(a)


def conf_features(depth, intr, mu, u, v):
    """52 features of pixel (u, v) (fp64) and whether the pixel has depth."""
    d = _f32(depth)
    H, W = d.shape
    x = np.zeros(N_FEATURES, dtype=np.float64)
    ok = _load().orc_conf_features(d, W, H, _f32(intr), mu, int(u), int(v), x)
    return x, bool(ok)


def mlp_forward(params, x, round_bf16=True):
    """(logit, h1, h2) of one feature vector."""
    h1 = np.zeros(N_HIDDEN, dtype=np.float64)
    h2 = np.zeros(N_HIDDEN, dtype=np.float64)
    o = _load().orc_mlp_forward(_f32(params), np.ascontiguousarray(x, dtype=np.float64), int(round_bf16),
                                h1.ctypes.data, h2.ctypes.data)
    return o, h1, h2


def mlp_loss_grad(params, X, y, round_bf16=True):
    """Mean BCE loss and its gradient (fp64, length N_PARAMS)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    g = np.zeros(N_PARAMS, dtype=np.float64)
    loss = _load().orc_mlp_loss_grad(_f32(params), X, _f32(y), X.shape[0], int(round_bf16), g)
    return loss, g


def conf_weights(depth, intr, mu, params):
    d = _f32(depth)
    H, W = d.shape
    out = np.zeros((H, W), dtype=np.float32)
    _load().orc_conf_weights(d, W, H, _f32(intr), mu, _f32(params), out)
    return out


# ------------------------------------------------------------------ tracking

def depth_halve(depth):
    """One pyramid level: means of the valid depths of 2x2 pixel blocks."""
    d = _f32(depth)
    H, W = d.shape
    out = np.zeros((H // 2, W // 2), dtype=np.float32)
    _load().orc_depth_halve(d, W, H, out)
    return out


def icp_reduce(depth, intr, T_g, V, N, intr_r, T_ref, dist_thresh):
    """Sec. 4.1.1 point-to-plane sums: (sums[29], abs_sums[28]); see
    orc_icp_reduce for the layout."""
    d = _f32(depth)
    H, W = d.shape
    V, N = _f32(V), _f32(N)
    Hr, Wr = V.shape[:2]
    sums = np.zeros(29)
    abs_sums = np.zeros(28)
    _load().orc_icp_reduce(d, W, H, _f32(intr), _f32(T_g).ravel(), V.ravel(), N.ravel(), Wr, Hr, _f32(intr_r),
                           _f32(T_ref).ravel(), float(dist_thresh), sums, abs_sums.ctypes.data)
    return sums, abs_sums


def icp_update(sums, T):
    """Gauss-Newton step: (new T, step x (6), ok)."""
    Tn = _f32(T).copy().ravel()
    x = np.zeros(6)
    ok = _load().orc_icp_update(np.ascontiguousarray(sums, dtype=np.float64), Tn, x.ctypes.data) == 0
    return Tn.reshape(4, 4), x, ok


def track(depth, intr, iters, thresh, V, N, intr_r, T_ref, T_init):
    """Coarse-to-fine tracking; iters[l], thresh[l] for pyramid level l
    (0 = input resolution).  Returns (T, steps)."""
    d = _f32(depth)
    H, W = d.shape
    V, N = _f32(V), _f32(N)
    Hr, Wr = V.shape[:2]
    T = _f32(T_init).copy().ravel()
    it = np.ascontiguousarray(iters, dtype=np.int32)
    steps = _load().orc_track(d, W, H, _f32(intr), len(it), it, _f32(thresh), V.ravel(), N.ravel(), Wr, Hr,
                              _f32(intr_r), _f32(T_ref).ravel(), T)
    return T.reshape(4, 4), int(steps)


def slab_owner(bx, n, w):
    """Part that owns block column bx: floor(bx / w) mod n."""
    return (int(bx) // int(w)) % int(n)


def merge_raycasts(vtx, nrm, T_wc):
    """The parts' raycasts (vtx, nrm: float32 [n, H, W, 4]) merged per pixel:
    the hit nearest to the camera (camera depth from float(T_wc^-1)), equal
    depths to the lower part."""
    vtx = _f32(vtx)
    nrm = _f32(nrm)
    n, H, W = vtx.shape[:3]
    vo = np.zeros((H, W, 4), dtype=np.float32)
    no = np.zeros((H, W, 4), dtype=np.float32)
    _load().orc_merge_raycasts(n, vtx.ravel(), nrm.ravel(), W, H, _f32(T_wc).ravel(), vo, no)
    return vo, no


def cell_triangles(F):
    """Marching-Cubes triangles of one cell with corner values F[8] (corner
    k at (k & 1, (k >> 1) & 1, k >> 2)), as edge indices [n, 3]."""
    tri = np.zeros(36, dtype=np.int32)
    n = _load().orc_cell_triangles(_f32(F), tri)
    return tri[:3 * n].reshape(n, 3)
