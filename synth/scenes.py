"""Analytic scenes, seeded camera paths and a Kinect-style depth sensor model.

Conventions used everywhere in this repository:

* world frame: metres, +y up;
* camera frame: +x right, +y down, +z forward (pinhole, u = fx*X/Z + cx,
  v = fy*Y/Z + cy, pixel (u, v) = (column, row));
* a pose is camera-to-world, a rigid 4x4 matrix, row-major.

Depth frames are z-depth in metres (float32), 0 = no measurement.  The
renderer intersects each pixel's ray with every primitive in fp64 and keeps
the nearest hit; the sensor model then adds axial Gaussian noise
sigma(z) = 0.0012 + 0.0019 (z - 0.4)^2 (Nguyen, Izadi and Lovell, 2012) and,
for the room scenes, replaces a share of the pixels on depth edges by
"flying pixels" interpolated between foreground and background.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np


# ----------------------------------------------------------------------------
# camera model
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Intrinsics:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def as_array(self) -> np.ndarray:
        return np.array([self.fx, self.fy, self.cx, self.cy], dtype=np.float32)


def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Camera-to-world pose (fp64) of a camera at `eye` looking at `target`."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, dtype=np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = x, y, f, eye
    return T


def pose_from_yaw_pitch(eye, yaw, pitch) -> np.ndarray:
    fwd = np.array([math.cos(pitch) * math.sin(yaw), math.sin(pitch),
                    math.cos(pitch) * math.cos(yaw)])
    return look_at(eye, np.asarray(eye) + fwd)


def pixel_rays(intr: Intrinsics, T_wc: np.ndarray):
    """Origin and per-pixel world directions (fp64) whose camera z is 1, so the
    ray parameter of a hit is its z-depth."""
    u = np.arange(intr.width, dtype=np.float64)
    v = np.arange(intr.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - intr.cx) / intr.fx, (vv - intr.cy) / intr.fy,
                   np.ones_like(uu)], axis=-1).reshape(-1, 3)
    D = dc @ np.asarray(T_wc, dtype=np.float64)[:3, :3].T
    return np.asarray(T_wc, dtype=np.float64)[:3, 3].copy(), D


# ----------------------------------------------------------------------------
# primitives: exact fp64 ray intersection and signed distance
# ----------------------------------------------------------------------------

_INF = np.inf


class Primitive:
    def intersect(self, o: np.ndarray, D: np.ndarray) -> np.ndarray:  # pragma: no cover
        raise NotImplementedError

    def bound(self):
        """Bounding sphere (centre, radius), or None for unbounded primitives."""
        return None

    def sdf(self, p: np.ndarray) -> np.ndarray:  # pragma: no cover
        raise NotImplementedError


class FloorPlane(Primitive):
    """Solid half-space y <= 0."""

    def intersect(self, o, D):
        with np.errstate(divide="ignore", invalid="ignore"):
            t = -o[1] / D[:, 1]
        t = np.where((D[:, 1] < 0) & (t > 0), t, _INF)
        return t

    def sdf(self, p):
        return p[..., 1]


class Sphere(Primitive):
    def __init__(self, c, r):
        self.c = np.asarray(c, dtype=np.float64)
        self.r = float(r)

    def bound(self):
        return self.c, self.r

    def intersect(self, o, D):
        oc = o - self.c
        a = np.einsum("ij,ij->i", D, D)
        b = D @ oc
        cc = oc @ oc - self.r * self.r
        if cc <= 0:
            return np.full(D.shape[0], _INF)
        disc = b * b - a * cc
        with np.errstate(invalid="ignore"):
            t = (-b - np.sqrt(disc)) / a
        return np.where((disc >= 0) & (t > 0), t, _INF)

    def sdf(self, p):
        return np.linalg.norm(p - self.c, axis=-1) - self.r


class Box(Primitive):
    """Solid axis-aligned box."""

    def __init__(self, lo, hi):
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)

    def bound(self):
        return 0.5 * (self.lo + self.hi), 0.5 * float(np.linalg.norm(self.hi - self.lo))

    def intersect(self, o, D):
        if np.all(o > self.lo) and np.all(o < self.hi):
            return np.full(D.shape[0], _INF)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / D
            t1 = (self.lo - o) * inv
            t2 = (self.hi - o) * inv
        t1 = np.nan_to_num(t1, nan=-_INF)
        t2 = np.nan_to_num(t2, nan=_INF)
        tn = np.max(np.minimum(t1, t2), axis=1)
        tf = np.min(np.maximum(t1, t2), axis=1)
        return np.where((tn <= tf) & (tn > 0), tn, _INF)

    def sdf(self, p):
        c = 0.5 * (self.lo + self.hi)
        h = 0.5 * (self.hi - self.lo)
        q = np.abs(p - c) - h
        outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
        inside = np.minimum(np.max(q, axis=-1), 0.0)
        return outside + inside


class Cylinder(Primitive):
    """Solid capped cylinder with a vertical (y) axis."""

    def __init__(self, cx, cz, r, y0, y1):
        self.cx, self.cz, self.r, self.y0, self.y1 = map(float, (cx, cz, r, y0, y1))

    def bound(self):
        hh = 0.5 * (self.y1 - self.y0)
        return np.array([self.cx, 0.5 * (self.y0 + self.y1), self.cz]), math.hypot(self.r, hh)

    def intersect(self, o, D):
        ox, oz = o[0] - self.cx, o[2] - self.cz
        if ox * ox + oz * oz < self.r * self.r and self.y0 < o[1] < self.y1:
            return np.full(D.shape[0], _INF)
        a = D[:, 0] ** 2 + D[:, 2] ** 2
        b = D[:, 0] * ox + D[:, 2] * oz
        cc = ox * ox + oz * oz - self.r * self.r
        disc = b * b - a * cc
        with np.errstate(invalid="ignore", divide="ignore"):
            ts = (-b - np.sqrt(disc)) / a
        ys = o[1] + ts * D[:, 1]
        side = np.where((disc >= 0) & (a > 0) & (ts > 0) & (ys >= self.y0) & (ys <= self.y1), ts, _INF)
        best = side
        for yc in (self.y0, self.y1):
            with np.errstate(invalid="ignore", divide="ignore"):
                tc = (yc - o[1]) / D[:, 1]
            px = ox + tc * D[:, 0]
            pz = oz + tc * D[:, 2]
            ok = (tc > 0) & (px * px + pz * pz <= self.r * self.r)
            best = np.minimum(best, np.where(ok, tc, _INF))
        return best

    def sdf(self, p):
        dr = np.hypot(p[..., 0] - self.cx, p[..., 2] - self.cz) - self.r
        hh = 0.5 * (self.y1 - self.y0)
        dy = np.abs(p[..., 1] - 0.5 * (self.y0 + self.y1)) - hh
        d = np.stack([dr, dy], axis=-1)
        return np.minimum(np.max(d, axis=-1), 0.0) + np.linalg.norm(np.maximum(d, 0.0), axis=-1)


class RoomInside(Primitive):
    """The inside faces of an axis-aligned room; everything outside is solid."""

    def __init__(self, lo, hi):
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)

    def intersect(self, o, D):
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(D > 0, (self.hi - o) / D, np.where(D < 0, (self.lo - o) / D, _INF))
        t = np.min(t, axis=1)
        return np.where(t > 0, t, _INF)

    def sdf(self, p):
        return np.min(np.minimum(p - self.lo, self.hi - p), axis=-1)


def _cull_rect(bound, intr: Intrinsics, T: np.ndarray):
    """Inclusive pixel rectangle (v0, v1, u0, u1) that contains the projection
    of a bounding sphere, or None when no finite rectangle is known."""
    if bound is None:
        return None
    c, R = bound
    R = R * 1.001 + 1e-6
    cc = T[:3, :3].T @ (np.asarray(c) - T[:3, 3])
    if cc[2] - R <= 1e-3:
        if cc[2] + R <= 0:
            return (1, 0, 1, 0)
        return None
    xs = np.array([cc[0] - R, cc[0] + R])
    ys = np.array([cc[1] - R, cc[1] + R])
    zs = np.array([cc[2] - R, cc[2] + R])
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    u = intr.fx * X / Z + intr.cx
    v = intr.fy * Y / Z + intr.cy
    u0 = max(int(math.floor(u.min())) - 1, 0)
    u1 = min(int(math.ceil(u.max())) + 1, intr.width - 1)
    v0 = max(int(math.floor(v.min())) - 1, 0)
    v1 = min(int(math.ceil(v.max())) + 1, intr.height - 1)
    return (v0, v1, u0, u1)


class AnalyticScene:
    def __init__(self, prims: List[Primitive]):
        self.prims = prims

    def render(self, intr: Intrinsics, T_wc: np.ndarray):
        """Exact z-depth (fp64, [H, W]; 0 where nothing is hit) and primitive id.

        Each bounded primitive is only intersected with the rays inside a
        conservative pixel rectangle around its projected bounding sphere."""
        T = np.asarray(T_wc, dtype=np.float64)
        o, D = pixel_rays(intr, T)
        H, W = intr.height, intr.width
        best = np.full(D.shape[0], _INF)
        pid = np.full(D.shape[0], -1, dtype=np.int32)
        for i, pr in enumerate(self.prims):
            rows = _cull_rect(pr.bound(), intr, T)
            if rows is None:
                sel = slice(None)
            else:
                v0, v1, u0, u1 = rows
                if v0 > v1 or u0 > u1:
                    continue
                vv, uu = np.meshgrid(np.arange(v0, v1 + 1), np.arange(u0, u1 + 1), indexing="ij")
                sel = (vv * W + uu).ravel()
            t = pr.intersect(o, D[sel])
            m = t < best[sel]
            best[sel] = np.where(m, t, best[sel])
            pid[sel] = np.where(m, i, pid[sel])
        z = np.where(np.isfinite(best), best, 0.0)
        return z.reshape(H, W), pid.reshape(H, W)

    def sdf(self, p: np.ndarray) -> np.ndarray:
        """Signed distance to the nearest solid (positive in free space), fp64."""
        d = None
        for pr in self.prims:
            s = pr.sdf(p)
            d = s if d is None else np.minimum(d, s)
        return d


# ----------------------------------------------------------------------------
# sensor model
# ----------------------------------------------------------------------------

def sensor_sigma(z):
    """Axial noise standard deviation (m) of a structured-light depth sensor."""
    z = np.asarray(z, dtype=np.float64)
    return 0.0012 + 0.0019 * (z - 0.4) ** 2


def depth_edges(z: np.ndarray, jump: float = 0.1) -> np.ndarray:
    """Pixels with a valid 4-neighbour whose depth differs by more than `jump`."""
    H, W = z.shape
    e = np.zeros((H, W), dtype=bool)
    valid = z > 0
    for dy, dx in ((0, 1), (1, 0)):
        a = z[: H - dy, : W - dx]
        b = z[dy:, dx:]
        va = valid[: H - dy, : W - dx] & valid[dy:, dx:]
        j = va & (np.abs(a - b) > jump)
        e[: H - dy, : W - dx] |= j
        e[dy:, dx:] |= j
    return e


def apply_sensor(z_true: np.ndarray, rng: np.random.Generator, flying_frac: float,
                 z_range=(0.0, np.inf), noise_scale: float = 1.0):
    """Noisy measured depth (fp64) and the mask of flying pixels."""
    H, W = z_true.shape
    valid = z_true > 0
    z = z_true + noise_scale * sensor_sigma(z_true) * rng.standard_normal((H, W))
    z = np.where(valid, z, 0.0)
    flying = np.zeros((H, W), dtype=bool)
    if flying_frac > 0:
        edges = depth_edges(z_true)
        idx = np.flatnonzero(edges)
        n = min(int(round(flying_frac * np.count_nonzero(valid))), idx.size)
        if n > 0:
            pick = rng.choice(idx, size=n, replace=False)
            pad = np.pad(np.where(valid, z_true, np.nan), 1, constant_values=np.nan)
            r, c = np.unravel_index(pick, (H, W))
            neigh = np.stack([pad[r + 1, c + 1], pad[r, c + 1], pad[r + 2, c + 1],
                              pad[r + 1, c], pad[r + 1, c + 2]], axis=0)
            fg = np.nanmin(neigh, axis=0)
            bg = np.nanmax(neigh, axis=0)
            a = rng.uniform(0.0, 1.0, size=n)
            z.flat[pick] = fg + a * (bg - fg)
            flying.flat[pick] = True
    lo, hi = z_range
    keep = (z >= lo) & (z <= hi) & (z > 0)
    return np.where(keep, z, 0.0), flying & keep


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Frame:
    index: int
    depth: np.ndarray          # float32 [H, W], metres, 0 = invalid
    depth_u16: np.ndarray      # uint16 [H, W], millimetres, 0 = invalid
    T_wc: np.ndarray           # float32 [4, 4], camera-to-world, row-major
    depth_true: np.ndarray     # float64 [H, W], exact depth before noise
    flying: np.ndarray         # bool [H, W]


@dataclasses.dataclass
class Workload:
    name: str
    intr: Intrinsics
    params: dict               # scene parameters (voxel_size, mu, max_w, ...)
    n_frames: int
    scene: AnalyticScene
    pose_fn: Callable[[int], np.ndarray]
    seed: int
    flying_frac: float
    z_range: tuple
    noise_scale: float = 1.0
    _cache: dict = dataclasses.field(default_factory=dict, repr=False)

    def pose(self, k: int) -> np.ndarray:
        return self.pose_fn(k)

    def frame(self, k: int) -> Frame:
        if k in self._cache:
            return self._cache[k]
        T = self.pose_fn(k)
        T32 = T.astype(np.float32)
        z_true, _ = self.scene.render(self.intr, T32.astype(np.float64))
        rng = np.random.default_rng([self.seed, 7919, k])
        z, flying = apply_sensor(z_true, rng, self.flying_frac, self.z_range, self.noise_scale)
        # the float frame is the millimetre frame divided by 1000, so the two
        # variants describe the same measurement
        mm = np.clip(np.rint(z * 1000.0), 0, 65535).astype(np.uint16)
        depth = (mm.astype(np.float64) / 1000.0).astype(np.float32)
        f = Frame(k, depth, mm, T32, z_true, flying)
        if len(self._cache) < 64:
            self._cache[k] = f
        return f


def _smooth_path(rng, n_frames, fps, lo, hi, v_max, w_max_deg, yaw0, yaw_amp, pitch_amp):
    """Seeded smooth trajectory: each coordinate a sum of three sinusoids,
    rescaled so the speed stays <= v_max and the turn rate <= w_max_deg."""
    t = np.arange(n_frames) / fps
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    fr = rng.uniform(0.03, 0.25, size=(5, 3))
    ph = rng.uniform(0, 2 * np.pi, size=(5, 3))
    am = rng.uniform(0.3, 1.0, size=(5, 3))
    am /= am.sum(axis=1, keepdims=True)

    def comp(i, tt):
        return np.sum(am[i] * np.sin(2 * np.pi * fr[i] * tt[:, None] + ph[i]), axis=1)

    tt = np.linspace(0, t[-1] if n_frames > 1 else 1.0, 4 * max(n_frames, 2))
    pos = np.stack([comp(i, tt) for i in range(3)], axis=1)          # in [-1, 1]
    dt = tt[1] - tt[0] if tt.size > 1 else 1.0
    speed = np.max(np.linalg.norm(np.diff(pos * half, axis=0), axis=1) / dt) if tt.size > 1 else 0
    sp = 1.0 if speed <= v_max else v_max / speed
    yaw = comp(3, tt)
    pitch = comp(4, tt)
    ang = np.max(np.hypot(np.diff(yaw * yaw_amp), np.diff(pitch * pitch_amp)) / dt) if tt.size > 1 else 0
    sa = 1.0 if ang <= math.radians(w_max_deg) else math.radians(w_max_deg) / ang

    def pose(k):
        tk = np.array([k / fps])
        p = mid + sp * half * np.array([comp(i, tk)[0] for i in range(3)])
        return pose_from_yaw_pitch(p, yaw0 + sa * yaw_amp * comp(3, tk)[0],
                                   sa * pitch_amp * comp(4, tk)[0])

    return pose


def _room_primitives(rng, lo, hi, n, size_lo=0.1, size_hi=0.6):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    prims: List[Primitive] = []
    for _ in range(n):
        kind = rng.integers(0, 3)
        size = rng.uniform(size_lo, size_hi)
        h = 0.5 * size
        on_floor = rng.uniform() < 0.5
        if on_floor:
            x = rng.uniform(lo[0] + h, hi[0] - h)
            z = rng.uniform(lo[2] + h, hi[2] - h)
            y = lo[1] + h
        else:
            wall = rng.integers(0, 4)
            y = rng.uniform(lo[1] + h, hi[1] - h)
            if wall == 0:
                x, z = lo[0] + h, rng.uniform(lo[2] + h, hi[2] - h)
            elif wall == 1:
                x, z = hi[0] - h, rng.uniform(lo[2] + h, hi[2] - h)
            elif wall == 2:
                x, z = rng.uniform(lo[0] + h, hi[0] - h), lo[2] + h
            else:
                x, z = rng.uniform(lo[0] + h, hi[0] - h), hi[2] - h
        if kind == 0:
            prims.append(Sphere((x, y, z), h))
        elif kind == 1:
            e = h * rng.uniform(0.6, 1.0, size=3)
            e[np.argmax(e)] = h
            prims.append(Box((x - e[0], y - e[1], z - e[2]), (x + e[0], y + e[1], z + e[2])))
        else:
            r = h * rng.uniform(0.5, 1.0)
            prims.append(Cylinder(x, z, r, y - h, y + h))
    return prims


def _params(voxel_size, mu, max_w, nb, ne, nv, z_min, z_max):
    return dict(voxel_size=voxel_size, mu=mu, max_w=max_w, num_buckets=nb,
                num_excess=ne, num_blocks=nv, z_min=z_min, z_max=z_max)


def tiny_workload(seed: int = 0, n_frames: int = 10, noise_scale: float = 1.0) -> Workload:
    """160x120 view of a sphere and a box on a floor from a 10-degree arc."""
    intr = Intrinsics(160, 120, 140.0, 140.0, 80.0, 60.0)
    scene = AnalyticScene([FloorPlane(), Sphere((-0.35, 0.3, 0.0), 0.3),
                           Box((0.15, 0.0, -0.2), (0.55, 0.4, 0.2))])
    centre = np.array([0.0, 0.2, 0.0])

    def pose(k):
        a = math.radians(-5.0 + 10.0 * k / max(n_frames - 1, 1))
        eye = np.array([1.5 * math.sin(a), 0.6, 1.5 * math.cos(a)])
        return look_at(eye, centre)

    return Workload("tiny", intr, _params(0.01, 0.04, 100, 1 << 16, 1 << 14, 1 << 16, 0.2, 5.0),
                    n_frames, scene, pose, seed, 0.0, (0.0, 5.0), noise_scale)


def kinect_workload(seed: int = 0, n_frames: int = 300, width: int = 640, height: int = 480,
                    params: Optional[dict] = None) -> Workload:
    """640x480 Kinect-like sequence in a 4x3x2.5 m room with 20 primitives
    (other image sizes keep the field of view: focal length scaled with the
    width)."""
    sc = width / 640.0
    intr = Intrinsics(width, height, 525.0 * sc, 525.0 * sc, (width - 1) / 2.0, (height - 1) / 2.0)
    rng = np.random.default_rng([seed, 1])
    lo, hi = (-2.0, 0.0, -1.5), (2.0, 2.5, 1.5)
    prims: List[Primitive] = [RoomInside(lo, hi)] + _room_primitives(rng, lo, hi, 20)
    pose = _smooth_path(np.random.default_rng([seed, 2]), n_frames, 30.0,
                        (-1.5, 0.5, -1.0), (1.5, 2.0, 1.0), 0.5, 30.0,
                        yaw0=rng.uniform(0, 2 * np.pi), yaw_amp=2.0, pitch_amp=0.3)
    p = _params(0.005, 0.02, 100, 1 << 20, 1 << 17, 1 << 19, 0.4, 5.0)
    if params:
        p.update(params)
    return Workload("kinect", intr, p, n_frames, AnalyticScene(prims), pose, seed, 0.01, (0.4, 5.0))


def large_workload(seed: int = 0, n_frames: int = 1000, num_buckets: int = 1 << 22) -> Workload:
    """640x480 walk along a 20x10x3 m corridor with 200 primitives, 2 mm voxels."""
    intr = Intrinsics(640, 480, 525.0, 525.0, 319.5, 239.5)
    rng = np.random.default_rng([seed, 3])
    lo, hi = (-10.0, 0.0, -5.0), (10.0, 3.0, 5.0)
    prims: List[Primitive] = [RoomInside(lo, hi)] + _room_primitives(rng, lo, hi, 200)
    sway = np.random.default_rng([seed, 4]).uniform(0, 2 * np.pi, size=3)

    def pose(k):
        s = k / max(n_frames - 1, 1)
        eye = np.array([-9.0 + 18.0 * s, 1.5 + 0.2 * math.sin(6.0 * s + sway[0]),
                        1.5 * math.sin(3.0 * s + sway[1])])
        yaw = math.pi / 2 + 0.35 * math.sin(5.0 * s + sway[2])
        return pose_from_yaw_pitch(eye, yaw, -0.1)

    return Workload("large", intr, _params(0.002, 0.01, 100, num_buckets, 1 << 18, 1 << 21, 0.4, 5.0),
                    n_frames, AnalyticScene(prims), pose, seed, 0.01, (0.4, 5.0))


def workload_by_name(name: str, **kw) -> Workload:
    return {"tiny": tiny_workload, "kinect": kinect_workload, "large": large_workload}[name](**kw)
