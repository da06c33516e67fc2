"""Pins of the oracle's Marching-Cubes mesh (Sec. 4, Lorensen & Cline 1987).

The paper names the algorithm for mesh generation and nothing more.  The
readings (recorded in the design notes): cells are the voxel cubes g +
{0,1}^3 whose eight corners are allocated and observed; the surface is F = 0
with inside F < 0; a crossing sits at t = F_a / (F_a - F_b) along its edge;
on a face with diagonal inside corners those corners are kept apart.  The
pins check the triangulation of all 256 corner configurations, the closure
and orientation of meshes of random fields, and the geometry of meshes of a
plane and a sphere against their closed forms.
"""

import collections
import itertools

import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import scene_params

S = 0.01


def _edge_corners(e):
    axis, o = divmod(e, 4)
    o1, o2 = o & 1, o >> 1
    lo = [(o1 << 1) | (o2 << 2), o1 | (o2 << 2), o1 | (o2 << 1)][axis]
    return lo, lo | (1 << axis)


FACES = [[k for k in range(8) if ((k >> a) & 1) == side] for a in range(3) for side in (0, 1)]


def test_all_corner_configurations():
    """For each of the 256 inside/outside patterns: triangles use exactly the
    sign-changing edges; the boundary of the cell's surface lies on the cube
    faces, where it pairs the crossings of a face two by two; on a face with
    diagonal inside corners each segment cuts off one inside corner."""
    for cfg in range(256):
        F = np.array([-1.0 if (cfg >> k) & 1 else 1.0 for k in range(8)], np.float32)
        tri = oracle.cell_triangles(F)
        crossing = {e for e in range(12) if (F[_edge_corners(e)[0]] < 0) != (F[_edge_corners(e)[1]] < 0)}
        used = set(tri.ravel().tolist())
        assert used == crossing, cfg
        if cfg in (0, 255):
            assert len(tri) == 0
            continue
        # boundary edges of the cell's surface: used by one triangle
        cnt = collections.Counter()
        for t in tri:
            for i in range(3):
                cnt[frozenset((int(t[i]), int(t[(i + 1) % 3])))] += 1
        boundary = [tuple(e) for e, c in cnt.items() if c == 1]
        assert all(c <= 2 for c in cnt.values()), cfg
        face_edges = [{e for e in range(12) if set(_edge_corners(e)) <= set(f)} for f in FACES]
        for a, b in boundary:
            faces = [i for i, fe in enumerate(face_edges) if a in fe and b in fe]
            assert len(faces) == 1, (cfg, a, b)
        for i, fe in enumerate(face_edges):
            on_face = [(a, b) for a, b in boundary if a in fe and b in fe]
            cross = fe & crossing
            assert len(on_face) * 2 == len(cross), (cfg, i)
            assert {x for s in on_face for x in s} == cross, (cfg, i)
            # on a face with diagonal inside corners each segment joins the two
            # crossings around one corner, and that corner is inside
            if len(cross) == 4:
                inside = [k for k in FACES[i] if F[k] < 0]
                for a, b in on_face:
                    common = set(_edge_corners(a)) & set(_edge_corners(b))
                    assert len(common) == 1 and common.pop() in inside, (cfg, a, b)


def _mesh_stats(tris):
    """(vertices, edges, faces, boundary edges, misoriented interior edges)
    with vertices identified by their exact coordinates."""
    vid = {}
    F = []
    for t in tris:
        F.append(tuple(vid.setdefault(tuple(v.tolist()), len(vid)) for v in t))
    directed = collections.Counter()
    for a, b, c in F:
        for u, v in ((a, b), (b, c), (c, a)):
            directed[(u, v)] += 1
    und = collections.Counter()
    for (u, v), c in directed.items():
        und[frozenset((u, v))] += c
    boundary = [e for e, c in und.items() if c == 1]
    bad = []
    for e, c in und.items():
        if c == 2:
            u, v = tuple(e)
            if not (directed[(u, v)] == 1 and directed[(v, u)] == 1):
                bad.append(e)
    nonmanifold = [e for e, c in und.items() if c > 2]
    return len(vid), len(und), len(F), boundary, bad, nonmanifold


def test_random_field_mesh_is_closed_and_consistently_oriented():
    """Random values on one block: inside the block every mesh edge is shared
    by exactly two triangles traversing it in opposite directions (cells that
    share a face agree on it); only edges on the outer faces of the meshed
    region are boundary edges."""
    rng = np.random.default_rng(1)
    sc = oracle.Scene(**scene_params(voxel_size=S))
    sc.set_block((0, 0, 0), rng.uniform(-1, 1, 512).astype(np.float32), 1.0)
    tris = sc.mesh()
    assert len(tris) > 200
    V, E, Fn, boundary, bad, nonman = _mesh_stats(tris)
    assert not nonman and not bad
    # every boundary edge lies on the outer faces x, y, z in {0, 7} voxels
    vid = {}
    for t in tris:
        for v in t:
            vid.setdefault(tuple(v.tolist()), len(vid))
    inv = {i: np.asarray(k, np.float64) / S for k, i in vid.items()}
    for e in boundary:
        u, v = tuple(e)
        pu, pv = inv[u], inv[v]
        on = [(abs(pu[a] - x) < 1e-4 and abs(pv[a] - x) < 1e-4) for a in range(3) for x in (0.0, 7.0)]
        assert any(on), (pu, pv)


def _block_field(sc, fn, blocks, mu):
    for b in blocks:
        l = np.arange(512)
        g = np.stack([8 * b[0] + (l & 7), 8 * b[1] + ((l >> 3) & 7), 8 * b[2] + (l >> 6)], 1).astype(np.float64)
        sc.set_block(b, np.clip(fn(g * S) / mu, -1, 1).astype(np.float32), 1.0)


def test_plane_mesh_lies_on_the_plane_with_its_area():
    """F = (z - z0) / mu over 2x2x2 blocks: the mesh is the plane z = z0 over
    the 15 x 15 meshable cells (area (15 s)^2), every normal +z."""
    z0 = 0.0734
    mu = 0.04
    sc = oracle.Scene(**scene_params(voxel_size=S))
    _block_field(sc, lambda p: p[:, 2] - z0, list(itertools.product(range(2), range(2), range(2))), mu)
    tris = sc.mesh().astype(np.float64)
    assert np.all(np.abs(tris[..., 2] - z0) < 1e-6)
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    area = 0.5 * np.linalg.norm(n, axis=1)
    assert np.all(n[:, 2] > 0)
    assert area.sum() == pytest.approx((15 * S) ** 2, rel=1e-5)


def test_sphere_mesh_is_a_closed_outward_sphere():
    """A truncated sphere SDF (r = 0.1 m): vertices on the sphere within s/50,
    every edge shared by two oppositely directed triangles, Euler
    characteristic 2 (one closed genus-0 surface), normals outward, enclosed
    volume 4/3 pi r^3 within 1%."""
    r, c, mu = 0.1, np.array([0.0423, 0.0611, 0.0507]), 0.04
    blocks = list(itertools.product(range(-1, 3), range(-1, 3), range(-1, 3)))
    sc = oracle.Scene(**scene_params(voxel_size=S))
    _block_field(sc, lambda p: np.linalg.norm(p - c, axis=1) - r, blocks, mu)
    tris = sc.mesh().astype(np.float64)
    d = np.linalg.norm(tris - c, axis=2)
    assert np.all(np.abs(d - r) < S / 50)
    V, E, Fn, boundary, bad, nonman = _mesh_stats(sc.mesh())
    assert not boundary and not bad and not nonman
    assert V - E + Fn == 2
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert np.all(np.sum(n * (tris.mean(axis=1) - c), axis=1) > 0)
    vol = np.sum(np.einsum("ij,ij->i", tris[:, 0] - c, np.cross(tris[:, 1] - c, tris[:, 2] - c))) / 6.0
    assert vol == pytest.approx(4.0 / 3.0 * np.pi * r ** 3, rel=0.01)


def test_unobserved_or_missing_corners_are_not_meshed():
    """Cells with a corner in an unallocated block or with weight 0 produce
    nothing: a single block meshes only its 7x7x7 interior cells, and zero
    weights remove the cells that touch them."""
    sc = oracle.Scene(**scene_params(voxel_size=S))
    l = np.arange(512)
    F = ((l >> 6) - 3.5).astype(np.float32) / 4.0      # z plane through the block
    sc.set_block((0, 0, 0), F, 1.0)
    n_full = len(sc.mesh())
    assert n_full == 2 * 7 * 7
    w = np.ones(512, np.float32)
    w[(l & 7) == 0] = 0.0                               # the x = 0 voxel column
    sc2 = oracle.Scene(**scene_params(voxel_size=S))
    sc2.set_block((0, 0, 0), F, w)
    assert len(sc2.mesh()) == 2 * 6 * 7


def test_a_field_touching_zero_without_changing_sign_has_no_surface():
    """Inside is F < 0: a non-negative field that is exactly 0 on a voxel
    layer (|z - 3 s| / mu) has no sign change and no surface, while the
    signed field (z - 3 s) / mu is meshed exactly on that layer."""
    l = np.arange(512)
    z = (l >> 6).astype(np.float32)
    sc = oracle.Scene(**scene_params(voxel_size=S))
    sc.set_block((0, 0, 0), (np.abs(z - 3.0) / 4.0).astype(np.float32), 1.0)
    assert len(sc.mesh()) == 0
    sc2 = oracle.Scene(**scene_params(voxel_size=S))
    sc2.set_block((0, 0, 0), ((z - 3.0) / 4.0).astype(np.float32), 1.0)
    tris = sc2.mesh()
    assert len(tris) == 2 * 7 * 7 and np.all(tris[..., 2] == np.float32(3.0) * np.float32(S))


def test_library_case_table_equals_the_oracle_cells():
    """The library builds its Marching-Cubes case table by its own derivation
    (crossings linked face by face, loops oriented by a geometric test); the
    oracle triangulates each cell by walking the faces counter-clockwise.  On
    all 256 inside/outside patterns the two give the same triangles, as sets
    (each loop is found in its own order; host call, no GPU)."""
    import paper_1708_00783_gb300 as itm
    count, edges = itm.itm_mesh_case_table()
    for cfg in range(256):
        F = np.array([-1.0 if (cfg >> k) & 1 else 1.0 for k in range(8)], np.float32)
        want = sorted(map(tuple, oracle.cell_triangles(F).tolist()))
        got = sorted(map(tuple, edges[cfg, :count[cfg]].astype(int).tolist()))
        assert got == want, (cfg, got, want)
