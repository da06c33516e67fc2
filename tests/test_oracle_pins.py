"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form of the truncated signed distance of a plane, a brute-force sweep of the
block grid, analytic ray/primitive geometry, modular arithmetic of the printed
hash function, or the exact rational value of a unit conversion.  A plausible
mistake in the oracle (a dropped term, a wrong sign, a transposed pose, a
capped weight used as the divisor, a missing chain link) fails at least one.
"""

import math
import os

import numpy as np
import pytest

import oracle
from synth import Intrinsics, tiny_workload
from synth.scenes import look_at

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v) if "." in v else int(v)
    return vals


def random_pose(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = rng.uniform(-1.0, 1.0, 3)
    return T.astype(np.float32)


SMALL = Intrinsics(40, 30, 35.0, 35.0, 19.5, 14.5)


def scene_params(**kw):
    p = dict(voxel_size=0.01, mu=0.04, max_w=100, num_buckets=1 << 12, num_excess=1 << 12,
             num_blocks=1 << 14, z_min=0.1, z_max=10.0)
    p.update(kw)
    return p


def voxel_camera_coords(coords, s, T_wc):
    """fp64 camera coordinates of every voxel of the exported blocks: voxel g
    at world g*s, mapped by the rigid inverse of the (float) pose."""
    T = T_wc.astype(np.float64)
    R, t = T[:3, :3], T[:3, 3]
    l = np.arange(512)
    local = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    g = coords.astype(np.int64)[:, None, :] * 8 + local[None]
    p = g.astype(np.float64) * float(np.float32(s))
    return (p - t) @ R                       # row vectors: R^T (p - t)


def projection_margin_ok(pc, intr, margin=1e-3):
    with np.errstate(divide="ignore", invalid="ignore"):
        u = intr.fx * pc[..., 0] / pc[..., 2] + intr.cx
        v = intr.fy * pc[..., 1] / pc[..., 2] + intr.cy
    inside = (pc[..., 2] > 0) & (u >= 1 + margin) & (u <= intr.width - 2 - margin) & \
             (v >= 1 + margin) & (v <= intr.height - 2 - margin)
    outside = (pc[..., 2] <= 0) | (u < 1 - margin) | (u > intr.width - 2 + margin) | \
              (v < 1 - margin) | (v > intr.height - 2 + margin)
    return inside, outside


def fuse_planes(depths, T, params, intr=SMALL):
    sc = oracle.Scene(**params)
    for D in depths:
        depth = np.full((intr.height, intr.width), D, dtype=np.float32)
        sc.allocate(depth, intr.as_array(), T)
        sc.integrate(depth, intr.as_array(), T)
    return sc


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_frame_plane_closed_form(seed):
    """Sec. 4.3: one frame of a fronto-parallel plane at depth D gives every
    voxel in front of or within mu behind it F = clamp((D - z)/mu, -1, 1),
    W = 1, and leaves voxels further behind at their defaults (Sec. 3.1)."""
    rng = np.random.default_rng(seed)
    T = random_pose(rng) if seed else np.eye(4, dtype=np.float32)
    D, p = 1.0 + 0.3 * seed, scene_params()
    sc = fuse_planes([D], T, p)
    coords, F, Wt = sc.export()
    assert coords.shape[0] > 50
    dflt = golden("voxel_defaults.txt")
    pc = voxel_camera_coords(coords, p["voxel_size"], T)
    inside, outside = projection_margin_ok(pc, SMALL)
    eta = D - pc[..., 2]
    upd = inside & (eta >= -p["mu"] + 1e-6)
    behind = inside & (eta < -p["mu"] - 1e-6)
    expect = np.clip(eta / p["mu"], -1.0, 1.0)
    assert upd.sum() > 1000
    np.testing.assert_allclose(F[upd], expect[upd], atol=1e-5, rtol=0)
    assert np.all(Wt[upd] == 1)
    assert np.all(F[behind] == dflt["sdf_init"]) and np.all(Wt[behind] == dflt["w_init"])
    assert np.all(F[outside] == dflt["sdf_init"]) and np.all(Wt[outside] == dflt["w_init"])


def test_weight_counts_observing_frames_up_to_cap():
    """Sec. 4.3: the weight is the number of frames that observed the voxel,
    capped at maxW; identical observations average to themselves."""
    T = random_pose(np.random.default_rng(5))
    p = scene_params(max_w=3)
    one = fuse_planes([1.2], T, p)
    five = fuse_planes([1.2] * 5, T, p)
    c1, F1, W1 = one.export()
    c5, F5, W5 = five.export()
    assert np.array_equal(c1, c5)
    seen = W1 > 0
    assert np.all(W5[seen] == 3) and np.all(W5[~seen] == 0)
    np.testing.assert_allclose(F5[seen], F1[seen], atol=2e-7, rtol=0)


def _blocks_present(coords, ref_coords):
    ref = {tuple(int(v) for v in c) for c in ref_coords}
    return np.array([tuple(int(v) for v in c) in ref for c in coords])[:, None]


def test_two_depths_average_and_behind_skip():
    """Sec. 4.3: a second observation averages with the first; a voxel more
    than mu behind the second surface keeps its first value; a block first
    allocated by the second frame (Sec. 4.2 runs before integration) holds
    the second observation alone."""
    T = random_pose(np.random.default_rng(7))
    p = scene_params()
    D1, D2 = 1.00, 0.97
    sc = fuse_planes([D1, D2], T, p)
    coords, F, Wt = sc.export()
    old = _blocks_present(coords, fuse_planes([D1], T, p).export(with_voxels=False)[0])
    pc = voxel_camera_coords(coords, p["voxel_size"], T)
    inside, _ = projection_margin_ok(pc, SMALL)
    e1, e2 = D1 - pc[..., 2], D2 - pc[..., 2]
    mu = p["mu"]
    f1, f2 = np.minimum(1.0, e1 / mu), np.minimum(1.0, e2 / mu)
    see1 = old & (e1 >= -mu + 1e-6)
    both = inside & see1 & (e2 >= -mu + 1e-6)
    first_only = inside & see1 & (e2 < -mu - 1e-6)
    second_only = inside & ~old & (e2 >= -mu + 1e-6)
    assert both.sum() > 500 and first_only.sum() > 100 and second_only.sum() > 100
    np.testing.assert_allclose(F[both], 0.5 * (f1 + f2)[both], atol=1e-5, rtol=0)
    assert np.all(Wt[both] == 2)
    np.testing.assert_allclose(F[first_only], f1[first_only], atol=1e-5, rtol=0)
    assert np.all(Wt[first_only] == 1)
    np.testing.assert_allclose(F[second_only], f2[second_only], atol=1e-5, rtol=0)
    assert np.all(Wt[second_only] == 1)


def test_capped_weight_contracts_geometrically():
    """Sec. 4.3 listing: the running mean divides by the uncapped oldW + newW
    and caps afterwards, so once W sits at maxW every new observation f moves
    F by the factor maxW/(maxW+1) towards f:
    F_k - f2 = (f1 - f2) (maxW/(maxW+1))^k."""
    T = random_pose(np.random.default_rng(11))
    max_w, k1, k2 = 4, 6, 3
    p = scene_params(max_w=max_w)
    D1, D2 = 1.00, 1.012
    sc = fuse_planes([D1] * k1 + [D2] * k2, T, p)
    coords, F, Wt = sc.export()
    old = _blocks_present(coords, fuse_planes([D1], T, p).export(with_voxels=False)[0])
    pc = voxel_camera_coords(coords, p["voxel_size"], T)
    inside, _ = projection_margin_ok(pc, SMALL)
    mu = p["mu"]
    e1, e2 = D1 - pc[..., 2], D2 - pc[..., 2]
    both = inside & old & (e1 >= -mu + 1e-6) & (e2 >= -mu + 1e-6)
    f1, f2 = np.minimum(1.0, e1 / mu), np.minimum(1.0, e2 / mu)
    r = max_w / (max_w + 1.0)
    expect = f2 + (f1 - f2) * r ** k2
    assert both.sum() > 500
    np.testing.assert_allclose(F[both], expect[both], atol=2e-5, rtol=0)
    assert np.all(Wt[both] == max_w)


# ------------------------------------------------------------- allocation

def _segment_meets_box(q0, q1, lo, hi):
    t0, t1 = 0.0, 1.0
    d = q1 - q0
    for i in range(3):
        if abs(d[i]) < 1e-15:
            if q0[i] < lo[i] or q0[i] > hi[i]:
                return False
            continue
        a, b = (lo[i] - q0[i]) / d[i], (hi[i] - q0[i]) / d[i]
        if a > b:
            a, b = b, a
        t0, t1 = max(t0, a), min(t1, b)
        if t0 > t1:
            return False
    return True


def brute_force_blocks(depth, intr, T, s, mu, z_min, z_max, eps):
    """Dense sweep of the block grid around each pixel's segment d-mu..d+mu
    with an fp64 slab test.  Returns blocks the segment surely crosses (even
    with the box shrunk by eps) and blocks it may touch (box grown by eps)."""
    T = T.astype(np.float64)
    B = 8.0 * float(np.float32(s))
    sure, maybe = set(), set()
    H, W = depth.shape
    for v in range(H):
        for u in range(W):
            d = float(depth[v, u])
            if not (d > 0) or d < z_min or d > z_max:
                continue
            r = np.array([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, 1.0])
            z0, z1 = max(d - mu, 1e-3), d + mu
            q0 = (T[:3, :3] @ (r * z0) + T[:3, 3]) / B
            q1 = (T[:3, :3] @ (r * z1) + T[:3, 3]) / B
            lo = np.floor(np.minimum(q0, q1)).astype(int) - 1
            hi = np.floor(np.maximum(q0, q1)).astype(int) + 1
            for bx in range(lo[0], hi[0] + 1):
                for by in range(lo[1], hi[1] + 1):
                    for bz in range(lo[2], hi[2] + 1):
                        b = np.array([bx, by, bz], dtype=np.float64)
                        if _segment_meets_box(q0, q1, b - eps, b + 1 + eps):
                            maybe.add((bx, by, bz))
                            if _segment_meets_box(q0, q1, b + eps, b + 1 - eps):
                                sure.add((bx, by, bz))
    return sure, maybe


@pytest.mark.parametrize("seed", range(4))
def test_allocation_equals_brute_force_sweep(seed):
    """Sec. 4.2: the allocated set is the union over valid pixels of the
    blocks crossed by the segment from depth d-mu to d+mu on the pixel's ray.
    A DDA that skips a block, overshoots, mis-scales the block size or uses
    the wrong pose direction fails this."""
    rng = np.random.default_rng(100 + seed)
    intr = Intrinsics(12, 9, 10.0, 10.0, 5.5, 4.0)
    T = random_pose(rng)
    depth = rng.uniform(0.5, 3.0, size=(9, 12)).astype(np.float32)
    depth[rng.uniform(size=depth.shape) < 0.1] = 0.0
    depth[0, 0] = np.nan
    p = scene_params(mu=0.2, z_min=0.6, z_max=2.9)   # long segments: ~5 blocks each
    sc = oracle.Scene(**p)
    assert sc.allocate(depth, intr.as_array(), T) == 0
    got = {tuple(int(x) for x in c) for c in sc.export(with_voxels=False)[0]}
    sure, maybe = brute_force_blocks(depth, intr, T, p["voxel_size"], p["mu"], p["z_min"],
                                     p["z_max"], eps=1e-4)
    assert len(sure) > 100
    assert sure <= got, sorted(sure - got)[:5]
    assert got <= maybe, sorted(got - maybe)[:5]
    assert sc.num_allocated == len(got)


def test_allocation_near_the_camera_starts_in_front_of_it():
    """Depths closer than mu: the segment's near end is clamped to 1 mm in
    front of the camera (a segment starting behind it would allocate blocks
    there); the allocated set still equals the brute-force sweep."""
    rng = np.random.default_rng(7)
    intr = Intrinsics(12, 9, 10.0, 10.0, 5.5, 4.0)
    T = random_pose(rng)
    depth = rng.uniform(0.02, 0.3, size=(9, 12)).astype(np.float32)
    p = scene_params(mu=0.2, z_min=0.01, z_max=2.9)
    assert (depth < p["mu"]).mean() > 0.5
    sc = oracle.Scene(**p)
    assert sc.allocate(depth, intr.as_array(), T) == 0
    got = {tuple(int(x) for x in c) for c in sc.export(with_voxels=False)[0]}
    sure, maybe = brute_force_blocks(depth, intr, T, p["voxel_size"], p["mu"], p["z_min"], p["z_max"], eps=1e-4)
    assert len(sure) > 50
    assert sure <= got, sorted(sure - got)[:5]
    assert got <= maybe, sorted(got - maybe)[:5]


def test_hash_function_matches_printed_constants():
    """Sec. 3.2: hashIndex xors the coordinates times the three printed primes
    (unsigned 32-bit wrap-around) and masks with buckets - 1."""
    g = golden("hash_function.txt")
    full = 1 << 32
    # the mask passed through is num_buckets - 1; use 2^31 buckets for a wide view
    nb = 1 << 31
    assert oracle.hash_index(1, 0, 0, nb) == g["prime_x"] % nb
    assert oracle.hash_index(0, 1, 0, nb) == g["prime_y"] % nb
    assert oracle.hash_index(0, 0, 1, nb) == g["prime_z"] % nb
    # negative coordinates: the unsigned cast of -1 is 2^32 - 1
    assert oracle.hash_index(-1, 0, 0, nb) == ((full - 1) * g["prime_x"] % full) % nb
    rng = np.random.default_rng(3)
    for x, y, z in rng.integers(-32768, 32768, size=(2000, 3)):
        h = oracle.hash_index(x, y, z, 1 << 20)
        assert 0 <= h < (1 << 20)
        # xor-separable and consistent across mask widths
        assert h == (oracle.hash_index(x, 0, 0, 1 << 20) ^ oracle.hash_index(0, y, 0, 1 << 20)
                     ^ oracle.hash_index(0, 0, z, 1 << 20))
        assert oracle.hash_index(x, y, z, 1 << 16) == h & 0xFFFF
        assert h == ((int(x) % full) * g["prime_x"] % full ^ (int(y) % full) * g["prime_y"] % full
                     ^ (int(z) % full) * g["prime_z"] % full) % (1 << 20)


def check_hash_invariants(entries, coords, nb, ne, nv, n_alloc, hash_fn):
    """Sec. 3.2/3.3 structure: every allocated block is reachable from its own
    bucket through the excess chain, no coordinate appears twice, block
    indices are distinct, chains are acyclic and the free lists add up."""
    g = golden("hash_function.txt")
    ptr = entries[:, 4]
    used = ptr >= 0
    assert used.sum() == n_alloc
    assert len(set(ptr[used].tolist())) == n_alloc
    keys = [tuple(e[:3]) for e in entries[used]]
    assert len(set(keys)) == len(keys)
    assert set(keys) == {tuple(int(v) for v in c) for c in coords}
    for i in np.flatnonzero(used[:nb]):
        assert hash_fn(*entries[i, :3]) == i
    reached = set()
    for b in range(nb):
        idx, seen = b, 0
        while True:
            e = entries[idx]
            if e[4] >= 0:
                assert hash_fn(*e[:3]) == b
                reached.add(idx)
            if e[3] < 1:
                break
            idx = nb + e[3] - g["excess_index_base_minus"]
            seen += 1
            assert seen <= ne, "cycle in excess chain"
    assert reached == set(np.flatnonzero(used).tolist())


def test_hash_invariants_with_excess_chains():
    """Forces collisions with 2^8 buckets so the excess list is exercised."""
    w = tiny_workload(n_frames=3)
    p = dict(w.params, num_buckets=1 << 8, num_excess=1 << 13)
    sc = oracle.Scene(**p)
    for k in range(3):
        f = w.frame(k)
        assert sc.allocate(f.depth, w.intr.as_array(), f.T_wc) == 0
    assert sc.excess_used > 1000
    coords = sc.export(with_voxels=False)[0]
    check_hash_invariants(sc.entries(), coords, p["num_buckets"], p["num_excess"],
                          p["num_blocks"], sc.num_allocated,
                          lambda x, y, z: oracle.hash_index(x, y, z, p["num_buckets"]))


def test_capacity_errors_are_reported():
    w = tiny_workload(n_frames=1)
    f = w.frame(0)
    sc = oracle.Scene(**dict(w.params, num_buckets=1 << 6, num_excess=16))
    assert sc.allocate(f.depth, w.intr.as_array(), f.T_wc) & oracle.ST_HASH_FULL
    assert sc.excess_used == 16
    sc = oracle.Scene(**dict(w.params, num_blocks=100))
    assert sc.allocate(f.depth, w.intr.as_array(), f.T_wc) & oracle.ST_VBA_FULL
    assert sc.num_allocated == 100


def test_degenerate_frames_change_nothing():
    """No valid depth (zeros, negatives, NaN) or a camera facing away from all
    allocated blocks leaves the volume untouched."""
    w = tiny_workload(n_frames=1)
    f = w.frame(0)
    intr = w.intr.as_array()
    sc = oracle.Scene(**w.params)
    for bad in (np.zeros_like(f.depth), np.full_like(f.depth, -1.0), np.full_like(f.depth, np.nan)):
        assert sc.allocate(bad, intr, f.T_wc) == 0
        assert sc.integrate(bad, intr, f.T_wc) == 0
    assert sc.num_allocated == 0
    sc.allocate(f.depth, intr, f.T_wc)
    n0 = sc.integrate(f.depth, intr, f.T_wc)
    assert n0 > 0
    before = sc.export()
    away = f.T_wc.copy()            # half a turn about the camera's y axis
    away[:3, 0] *= -1
    away[:3, 2] *= -1
    assert sc.integrate(np.full_like(f.depth, 1.0), intr, away) == 0
    after = sc.export()
    assert all(np.array_equal(a, b) for a, b in zip(before, after))


def test_depth_u16_conversion_is_correctly_rounded():
    """Sec. 4 view preparation: millimetres to metres; the float result must
    be the float nearest to raw/1000 (checked against exact rationals)."""
    raw = np.arange(65536, dtype=np.uint16)
    out = oracle.depth_u16_to_f32(raw).astype(np.float64)
    exact = raw.astype(np.float64) / 1000.0    # exact to 2^-53 relative
    up = np.nextafter(out.astype(np.float32), np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(out.astype(np.float32), np.float32(-np.inf)).astype(np.float64)
    err = np.abs(out - exact)
    assert np.all(err <= np.abs(up - exact) + 1e-300)
    assert np.all(err <= np.abs(dn - exact) + 1e-300)
    assert out[0] == 0.0 and out[1000] == 1.0 and out[5000] == 5.0


# -------------------------------------------------------------- raycast

def _silhouettes(pid, z, px=2):
    from scipy import ndimage
    sil = np.zeros(pid.shape, dtype=bool)
    for a in (0, 1):
        sil |= np.abs(np.diff(pid, axis=a, prepend=pid.take([0], axis=a))) > 0
        sil |= np.abs(np.diff(z, axis=a, prepend=z.take([0], axis=a))) > 0.05
    return ndimage.binary_dilation(sil, iterations=px)


@pytest.fixture(scope="module")
def fused_tiny_noise_free():
    w = tiny_workload(noise_scale=0.0)
    sc = oracle.Scene(**w.params)
    intr = w.intr.as_array()
    for k in range(w.n_frames):
        f = w.frame(k)
        sc.allocate(f.depth, intr, f.T_wc)
        sc.integrate(f.depth, intr, f.T_wc)
    return w, sc


def test_raycast_depth_matches_analytic_scene(fused_tiny_noise_free):
    """Sec. 4.4: the raycast finds the zero crossing of the fused TSDF; on a
    noise-free analytic scene (sphere, box, floor) its depth must match the
    exact ray/primitive intersection.  Where the depth changes by more than
    s/2 per pixel the listing's nearest-pixel depth read (Sec. 4.3) limits
    the TSDF itself, so the strict bound is taken where it is smaller."""
    w, sc = fused_tiny_noise_free
    f = w.frame(4)
    s = w.params["voxel_size"]
    vtx, nrm = sc.raycast(w.intr.width, w.intr.height, w.intr.as_array(), f.T_wc)
    z_true, pid = w.scene.render(w.intr, f.T_wc.astype(np.float64))
    T = f.T_wc.astype(np.float64)
    z = ((vtx[..., :3].reshape(-1, 3).astype(np.float64) - T[:3, 3]) @ T[:3, :3])[:, 2]
    z = z.reshape(z_true.shape)
    hit = vtx[..., 3] > 0
    ok = (z_true > 0) & (z_true < 4.5) & ~_silhouettes(pid, z_true)
    assert (hit & ok).sum() / ok.sum() > 0.97
    gy, gx = np.gradient(z_true)
    smooth = ok & hit & (np.hypot(gx, gy) <= 0.5 * s)
    err = np.abs(z - z_true)
    assert smooth.sum() > 1500
    assert np.mean(err[smooth] <= 0.25 * s) >= 0.99
    assert np.median(err[ok & hit]) <= 0.1 * s
    # the hit lies on the pixel's ray
    ray_c = np.stack([(np.arange(w.intr.width)[None, :] - w.intr.cx) / w.intr.fx * np.ones_like(z),
                      (np.arange(w.intr.height)[:, None] - w.intr.cy) / w.intr.fy * np.ones_like(z)], -1)
    pc = ((vtx[..., :3].reshape(-1, 3).astype(np.float64) - T[:3, 3]) @ T[:3, :3]).reshape(*z.shape, 3)
    np.testing.assert_allclose(pc[hit][:, :2] / pc[hit][:, 2:3], ray_c[hit], atol=1e-4)


def test_raycast_normals_match_analytic_normals(fused_tiny_noise_free):
    """Normals from the TSDF gradient point out of the solid: radial on the
    sphere, +y on the floor."""
    w, sc = fused_tiny_noise_free
    f = w.frame(4)
    vtx, nrm = sc.raycast(w.intr.width, w.intr.height, w.intr.as_array(), f.T_wc)
    z_true, pid = w.scene.render(w.intr, f.T_wc.astype(np.float64))
    ok = (vtx[..., 3] > 0) & (nrm[..., 3] > 0) & ~_silhouettes(pid, z_true) & (z_true < 2.5)
    n = nrm[..., :3].astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(n[nrm[..., 3] > 0], axis=1), 1.0, atol=1e-5)
    sph = ok & (pid == 1)
    P = vtx[..., :3][sph].astype(np.float64)
    c = np.array([-0.35, 0.3, 0.0])
    radial = (P - c) / np.linalg.norm(P - c, axis=1, keepdims=True)
    ang = np.degrees(np.arccos(np.clip(np.sum(n[sph] * radial, axis=1), -1, 1)))
    assert sph.sum() > 1000
    assert np.median(ang) <= 1.5 and np.percentile(ang, 90) <= 4.0
    flo = ok & (pid == 0)
    ang = np.degrees(np.arccos(np.clip(n[flo] @ np.array([0.0, 1.0, 0.0]), -1, 1)))
    assert flo.sum() > 1000
    assert np.median(ang) <= 2.0 and np.percentile(ang, 90) <= 5.0


def test_raycast_of_empty_volume_misses_everywhere():
    w = tiny_workload(n_frames=1)
    sc = oracle.Scene(**w.params)
    vtx, nrm = sc.raycast(w.intr.width, w.intr.height, w.intr.as_array(), w.frame(0).T_wc)
    assert not vtx.any() and not nrm.any()


def test_raycast_reproduces_a_linear_field():
    """Trilinear interpolation reproduces a field that is linear in the voxel
    coordinates, so over a volume holding the truncated distance of an
    oblique plane (F = (n . (g s - P0)) / mu with every voxel read near the
    crossing inside the band) the raycast's hits lie on the plane up to what
    the march's last step and the two refinement steps leave, a bound known
    per ray, and its normals equal n."""
    s, mu = 0.01, 0.04
    n = np.array([0.5, 0.3, -1.0])
    n /= np.linalg.norm(n)
    P0 = np.array([0.0, 0.0, 1.0])
    sc = oracle.Scene(**scene_params(voxel_size=s, mu=mu))
    l = np.arange(512)
    local = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    n_blocks = 0
    for bx in range(-14, 14):
        for by in range(-10, 10):
            for bz in range(6, 26):
                g = np.array([bx, by, bz]) * 8 + local
                d = (g * float(np.float32(s)) - P0) @ n
                if np.abs(d).min() > 0.12:
                    continue
                sc.set_block((bx, by, bz), np.clip(d / mu, -1.0, 1.0), 1.0)
                n_blocks += 1
    assert n_blocks > 500
    intr = SMALL
    vtx, nrm = sc.raycast(intr.width, intr.height, intr.as_array(), np.eye(4, dtype=np.float32))
    hit = vtx[..., 3] > 0
    assert hit.mean() > 0.99
    X = vtx[..., :3][hit].astype(np.float64)
    dist = (X - P0) @ n
    # the march stops within s cos(theta) past the plane (its smallest step
    # is s along the ray's depth unit), and each refinement step scales the
    # distance by (1 - cos(theta)), theta between the ray and the normal
    u, v = np.meshgrid(np.arange(intr.width), np.arange(intr.height))
    ray = np.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy], -1)[hit]
    c = np.abs(np.c_[ray, np.ones(len(ray))] @ n) / np.linalg.norm(np.c_[ray, np.ones(len(ray))], axis=1)
    bound = s * c * (1.0 - c) ** 2
    assert np.all(np.abs(dist) <= bound + 1e-3 * s), np.max(np.abs(dist) - bound)
    assert np.median(np.abs(dist)) <= 0.02 * s
    # the hit lies on the pixel's ray
    np.testing.assert_allclose(X[:, :2] / X[:, 2:3], ray, atol=1e-5)
    good = nrm[..., 3][hit] > 0
    assert good.mean() > 0.99
    np.testing.assert_allclose(nrm[..., :3][hit][good], np.broadcast_to(n, (good.sum(), 3)), atol=1e-4)


def test_raycast_starts_at_z_min():
    """The march covers depths z_min .. z_max only: a plane at 0.5 m is hit
    with z_min = 0.1 and not reported with z_min = 0.8 (the ray starts beyond
    it, in empty space)."""
    s, mu = 0.01, 0.04
    l = np.arange(512)
    local = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    for z_min, want_hits in ((0.1, True), (0.8, False)):
        sc = oracle.Scene(**scene_params(voxel_size=s, mu=mu, z_min=z_min, z_max=3.0))
        for bx in range(-6, 6):
            for by in range(-5, 5):
                for bz in range(4, 9):
                    g = np.array([bx, by, bz]) * 8 + local
                    d = 0.5 - g[:, 2] * float(np.float32(s))
                    if np.abs(d).min() > 0.12:
                        continue
                    sc.set_block((bx, by, bz), np.clip(d / mu, -1.0, 1.0), 1.0)
        vtx, _ = sc.raycast(SMALL.width, SMALL.height, SMALL.as_array(), np.eye(4, dtype=np.float32))
        hit = vtx[..., 3] > 0
        if want_hits:
            assert hit.mean() > 0.9 and np.allclose(vtx[..., 2][hit], 0.5, atol=0.2 * s)
        else:
            assert not hit.any()
