"""The visible-list pass marks a block interior when the projections of its
eight corners lie inside [1 + m_u, W - 2 - m_u] x [1 + m_v, H - 2 - m_v] with
Z above 1e-3 + e_R, and the integration then skips the per-voxel image-bound
tests of that block.  The margins are e_R (|f| + size + |c|) / z_min + 2e-3
with e_R = 2^-18 R, R the largest sum of the absolute terms of a row of M p
over the corners.  This checks, with float32 arithmetic emulated operation by
operation, that every voxel of a block the test marks passes the integration's
bounds tests (Z > 0, 1 <= u <= W - 2, 1 <= v <= H - 2), on random poses with
large translations and blocks placed along the image border, where the
margins matter."""

import numpy as np

F = np.float32


def f32(x):
    return np.asarray(x, dtype=np.float32)


def voxel_uv(M, intr, b, vs):
    """The integration's exact arithmetic for all 512 voxels of block b:
    p = (8 b + k) s rounded once, each row ((m0 px + m1 py) + m2 pz) + m3 with
    every product and sum rounded, u = RN(RN(fx X) / Z) + cx rounded."""
    fx, fy, cx, cy = (F(x) for x in intr)
    k = np.arange(8, dtype=np.float32)
    vs = F(vs)
    px = f32((F(8 * b[0]) + k) * vs)[None, None, :]
    py = f32((F(8 * b[1]) + k) * vs)[None, :, None]
    pz = f32((F(8 * b[2]) + k) * vs)[:, None, None]

    def row(r):
        a = f32(f32(M[r, 0] * px) + f32(M[r, 1] * py))
        a = f32(a + f32(M[r, 2] * pz))
        return f32(a + M[r, 3])

    X, Y, Z = row(0), row(1), row(2)
    with np.errstate(all="ignore"):
        u = f32(f32(f32(fx * X) / Z) + cx)
        v = f32(f32(f32(fy * Y) / Z) + cy)
    return Z, u, v


def interior(M, intr, W, H, b, vs):
    """The visible-list pass's interior test (corner arithmetic in float32
    with products and sums rounded separately; the kernel's own rounding of
    the corners differs by a few ulps, which the factor of four covers)."""
    fx, fy, cx, cy = (float(x) for x in intr)
    c = np.array([[i, j, k] for k in (0, 7) for j in (0, 7) for i in (0, 7)], dtype=np.float64)
    P = f32((8 * np.asarray(b, dtype=np.float64)[None, :] + c) * float(vs))
    R = 0.0
    Zs, us, vsv = [], [], []
    for p in P:
        rows = []
        for r in range(3):
            t = [f32(M[r, 0] * p[0]), f32(M[r, 1] * p[1]), f32(M[r, 2] * p[2]), f32(M[r, 3])]
            R = max(R, float(sum(abs(float(x)) for x in t)))
            rows.append(f32(f32(f32(t[0] + t[1]) + t[2]) + t[3]))
        X, Y, Z = rows
        if Z < 1e-3:
            return False
        Zs.append(float(Z))
        us.append(float(f32(f32(f32(F(fx) * X) / Z) + F(cx))))
        vsv.append(float(f32(f32(f32(F(fy) * Y) / Z) + F(cy))))
    eR = 2.0 ** -18 * R
    zmin = min(Zs)
    if not zmin > 1e-3 + eR:
        return False
    mu = eR * (abs(fx) + W + abs(cx)) / zmin + 2e-3
    mv = eR * (abs(fy) + H + abs(cy)) / zmin + 2e-3
    return min(us) >= 1 + mu and max(us) <= W - 2 - mu and min(vsv) >= 1 + mv and max(vsv) <= H - 2 - mv


def random_pose(rng, trans):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = rng.uniform(-trans, trans, size=3)
    return T


def test_interior_blocks_pass_every_voxel_bound():
    rng = np.random.default_rng(7)
    W, H = 640, 480
    intr = (525.0, 525.0, 319.5, 239.5)
    marked = 0
    for trial in range(120):
        vs = float(rng.choice([0.002, 0.005, 0.01]))
        T_wc = random_pose(rng, trans=float(rng.choice([1.0, 50.0, 1000.0])))
        M = np.linalg.inv(T_wc)[:3, :].astype(np.float32)
        for _ in range(50):
            # a block near the image border at a random depth
            z = rng.uniform(0.3, 6.0)
            u = rng.choice([rng.uniform(-5, 12), rng.uniform(W - 14, W + 4), rng.uniform(0, W)])
            v = rng.choice([rng.uniform(-5, 12), rng.uniform(H - 14, H + 4), rng.uniform(0, H)])
            pc = np.array([(u - intr[2]) / intr[0] * z, (v - intr[3]) / intr[1] * z, z, 1.0])
            pw = T_wc @ pc
            b = np.floor(pw[:3] / (8 * vs)).astype(np.int64)
            if np.any(np.abs(b) > 32000):
                continue
            if not interior(M, intr, W, H, b, vs):
                continue
            marked += 1
            Z, uu, vv = voxel_uv(M, intr, b, vs)
            assert np.all(Z > 0)
            assert np.all((uu >= 1.0) & (uu <= W - 2)), (trial, b, float(uu.min()), float(uu.max()))
            assert np.all((vv >= 1.0) & (vv <= H - 2)), (trial, b, float(vv.min()), float(vv.max()))
    assert marked > 1000
