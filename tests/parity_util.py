"""Helpers for the GPU-vs-oracle parity tests.

Tolerances (from the arithmetic, written here once):
  * allocated block set, integer weights: bit-exact (both sides take every
    deciding float operation unfused, round-to-nearest, in the same order);
  * |sdf_gpu - sdf_oracle| <= 1e-4 on every voxel (normalised units);
  * raycast: on >= 99.9% of pixels both miss, or both hit with camera depth
    within 0.5 mm and normals (where both have one) within 0.5 degrees.
"""

import numpy as np

SDF_TOL = 1e-4
DEPTH_TOL_M = 5e-4
NORMAL_TOL_DEG = 0.5
PIXEL_FRACTION = 0.999


def key_of(coords):
    c = coords.astype(np.int64) + 32768
    return (c[:, 0] << 32) | (c[:, 1] << 16) | c[:, 2]


def compare_volumes(gpu, orc, check_voxels=True):
    """gpu, orc: (coords, sdf, w) exports.  Returns a report dict; asserts the
    block sets are equal and voxels within tolerance."""
    cg, Fg, Wg = gpu
    co, Fo, Wo = orc
    kg, ko = key_of(cg), key_of(co)
    assert len(set(kg.tolist())) == len(kg), "duplicate block on the GPU"
    sg, so = set(kg.tolist()), set(ko.tolist())
    assert sg == so, "block sets differ: %d only on GPU, %d only in oracle" % (len(sg - so), len(so - sg))
    rep = {"blocks": len(kg)}
    if check_voxels and len(kg):
        ig, io = np.argsort(kg), np.argsort(ko)
        dF = np.abs(Fg[ig] - Fo[io])
        rep["max_dsdf"] = float(dF.max())
        rep["sdf_bitexact_frac"] = float(np.mean(Fg[ig] == Fo[io]))
        assert rep["max_dsdf"] <= SDF_TOL, rep
        assert np.array_equal(Wg[ig], Wo[io]), "weights differ on %d voxels" % int(np.sum(Wg[ig] != Wo[io]))
    return rep


def camera_depth(vtx, T_wc):
    T = np.asarray(T_wc, dtype=np.float64)
    p = vtx[..., :3].reshape(-1, 3).astype(np.float64)
    return ((p - T[:3, 3]) @ T[:3, :3])[:, 2].reshape(vtx.shape[:-1])


def compare_raycast(vg, ng, vo, no, T_wc):
    hg, ho = vg[..., 3] > 0, vo[..., 3] > 0
    zg, zo = camera_depth(vg, T_wc), camera_depth(vo, T_wc)
    both = hg & ho
    dz = np.where(both, np.abs(zg - zo), 0.0)
    nbg, nbo = ng[..., 3] > 0, no[..., 3] > 0
    cosang = np.clip(np.sum(ng[..., :3].astype(np.float64) * no[..., :3], axis=-1), -1, 1)
    ang = np.where(nbg & nbo, np.degrees(np.arccos(cosang)), 0.0)
    ok = (~hg & ~ho) | (both & (dz <= DEPTH_TOL_M) & (nbg == nbo) & (ang <= NORMAL_TOL_DEG))
    rep = {
        "pixels": int(ok.size),
        "hits": int(ho.sum()),
        "hit_agree": float(np.mean(hg == ho)),
        "pass_frac": float(np.mean(ok)),
        "bitexact_frac": float(np.mean(np.all(vg == vo, axis=-1) & np.all(ng == no, axis=-1))),
        "max_dz": float(dz.max()) if dz.size else 0.0,
    }
    assert rep["hit_agree"] >= PIXEL_FRACTION, rep
    assert rep["pass_frac"] >= PIXEL_FRACTION, rep
    return rep
