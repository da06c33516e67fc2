"""The C ABI library loads and exports every function the header declares.
No GPU calls: symbol presence, the host-only functions (the hash function and
the tracker's Gauss-Newton step) and the argument checks every call makes on
the host before it touches the device."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "itm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(itm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libitm():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_core_calls():
    fns = header_functions()
    for name in ("itm_scene_create", "itm_allocate", "itm_integrate", "itm_raycast", "itm_scene_destroy"):
        assert name in fns


def test_library_exports_every_declared_symbol(libitm):
    missing = [f for f in header_functions() if not hasattr(libitm, f)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1708_00783_gb300 as itm
    for f in header_functions():
        assert callable(getattr(itm, f, None)), f


def test_host_hash_index_follows_printed_function():
    """Sec. 3.2 primes, unsigned wrap-around, mask by buckets - 1 (the values
    come from the paper's printed constants, not from the oracle)."""
    import paper_1708_00783_gb300 as itm
    from tests.test_oracle_pins import golden
    g = golden("hash_function.txt")
    nb = 1 << 30
    assert itm.itm_hash_index(1, 0, 0, nb) == g["prime_x"] % nb
    assert itm.itm_hash_index(0, 1, 0, nb) == g["prime_y"] % nb
    assert itm.itm_hash_index(0, 0, 1, nb) == g["prime_z"] % nb
    assert itm.itm_hash_index(-1, -1, -1, 1 << 20) == (
        ((1 << 32) - g["prime_x"]) ^ ((1 << 32) - g["prime_y"]) ^ ((1 << 32) - g["prime_z"])) % (1 << 20)


def test_version_string():
    import paper_1708_00783_gb300 as itm
    assert "sm_103a" in itm.itm_version()


def test_binding_knows_every_error_code_and_constant():
    """Every ITM_ERR_* value of the header has its name in the binding's error
    map, and the binding's copies of the header's #define constants agree."""
    import paper_1708_00783_gb300 as itm
    text = open(os.path.join(ROOT, "include", "itm.h")).read()
    codes = {int(v): n for n, v in re.findall(r"(ITM_ERR_[A-Z_]+)\s*=\s*(\d+)", text)}
    assert codes and codes == itm.ERRORS
    assert all(getattr(itm, n) == v for v, n in codes.items())
    defines = dict(re.findall(r"#define\s+(ITM_[A-Z0-9_]+)\s+\(?([0-9]+)", text))
    for name in ("ITM_MLP_FEATURES", "ITM_MLP_HIDDEN", "ITM_MLP_PARAMS", "ITM_MLP_PACKED_BYTES",
                 "ITM_MLP_SCRATCH_PER_SAMPLE", "ITM_BATCH_STAGES"):
        if name in defines and hasattr(itm, name):
            assert int(defines[name]) == getattr(itm, name), name


def _icp_sums(rng, n=500, scale=1.0):
    """Point-to-plane sums (layout of itm_icp_reduce) of n random rows."""
    J = rng.normal(size=(n, 6)) * scale
    r = rng.normal(size=n) * 1e-3
    H = J.T @ J
    iu = np.triu_indices(6)
    return np.concatenate([H[iu], J.T @ r, [r @ r, n]])


def test_host_icp_step_equals_oracle():
    """itm_icp_step is host code: its Cholesky solve and pose update equal
    the oracle's Gauss-Newton step on random systems, and it refuses the
    systems without a unique solution (fewer than 6 pixels, a rank-deficient
    H)."""
    import oracle
    import paper_1708_00783_gb300 as itm
    from tests.test_oracle_track_pins import exp_pose
    rng = np.random.default_rng(21)
    for k in range(20):
        T = exp_pose(rng.normal(size=6) * 0.3, np.eye(4)).astype(np.float32)
        s = _icp_sums(rng, scale=10.0 ** rng.uniform(-2, 1))
        T1, x1 = itm.itm_icp_step(s, T)
        T2, x2, ok = oracle.icp_update(s, T)
        assert ok
        np.testing.assert_allclose(x1, x2, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(T1, T2, atol=2e-7)
    s = _icp_sums(rng)
    few = s.copy()
    few[28] = 5.0
    flat = _icp_sums(rng)
    J = rng.normal(size=(100, 6))
    J[:, 5] = 0.0  # no constraint on the z translation
    iu = np.triu_indices(6)
    flat[:21] = (J.T @ J)[iu]
    for bad in (few, flat):
        with pytest.raises(itm.ItmError):
            itm.itm_icp_step(bad, T)
    # the oracle takes the pixel-count rule in its tracking loop, before the
    # step; the step itself refuses only the rank-deficient system
    assert not oracle.icp_update(flat, T)[2]


_NULL_CHILD = r'''
import ctypes, re, sys
import paper_1708_00783_gb300 as itm
text = re.sub(r"/\*.*?\*/", "", open(sys.argv[1]).read(), flags=re.S)
for name in sorted(set(re.findall(r"\b(itm_[a-z0-9_]+)\s*\(", text))):
    if name in ("itm_version", "itm_hash_index", "itm_track_scratch_bytes"):
        continue
    f = getattr(itm._lib, name)
    args = [None if (a is ctypes.c_void_p or issubclass(a, ctypes._Pointer)) else a(0) for a in f.argtypes]
    print(name, f(*args), flush=True)
'''


def test_null_arguments_rejected_before_any_device_call():
    """Every call that takes a scene, a buffer or a pointer answers NULL /
    zero arguments with ITM_ERR_ARG from its host-side checks, before any
    CUDA call (this host has no GPU); a zero-length depth conversion is an
    empty no-op.  Run in a child process so a crash would fail the test, not
    end the session."""
    import subprocess
    import sys
    import paper_1708_00783_gb300 as itm
    r = subprocess.run([sys.executable, "-c", _NULL_CHILD, os.path.join(ROOT, "include", "itm.h")],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-400:] + r.stderr[-400:]
    got = dict(ln.split() for ln in r.stdout.splitlines())
    assert len(got) == len(header_functions()) - 3
    for name, code in got.items():
        want = itm.ITM_OK if name == "itm_depth_u16_to_f32" else itm.ITM_ERR_ARG
        assert int(code) == want, (name, code)


def test_scene_parameters_checked_on_the_host():
    """itm_scene_create refuses each invalid parameter with ITM_ERR_ARG
    before allocating anything."""
    import paper_1708_00783_gb300 as itm
    base = dict(voxel_size=0.005, mu=0.02, max_w=100, num_buckets=1 << 10, num_excess=64, num_blocks=256,
                z_min=0.4, z_max=5.0, weight_mode=0)
    bad = [dict(voxel_size=0.0), dict(voxel_size=float("nan")), dict(mu=-0.01), dict(weight_mode=2),
           dict(max_w=0), dict(max_w=256), dict(num_buckets=1000), dict(num_buckets=0), dict(num_excess=-1),
           dict(num_blocks=-1), dict(num_blocks=(1 << 24) + 1), dict(z_min=0.0), dict(z_max=0.4)]
    for change in bad:
        p = itm.itm_scene_params(**dict(base, **change))
        out = ctypes.c_void_p()
        assert itm._lib.itm_scene_create(ctypes.byref(p), ctypes.byref(out)) == itm.ITM_ERR_ARG, change
        assert not out.value
    # the learned mode keeps float weights, so its cap may exceed 255
    import torch
    if not torch.cuda.is_available():
        p = itm.itm_scene_params(**dict(base, weight_mode=1, max_w=1000))
        out = ctypes.c_void_p()
        assert itm._lib.itm_scene_create(ctypes.byref(p), ctypes.byref(out)) == itm.ITM_ERR_CUDA


def test_host_hash_on_a_million_triples():
    """The library's hash (the same __host__ __device__ function the kernels
    call) on 10^6 random int16 triples, extremes and negatives included,
    equals the printed function of Sec. 3.2 evaluated with numpy's uint32
    wrap-around from the golden primes, and the oracle's."""
    import oracle
    import paper_1708_00783_gb300 as itm
    from tests.test_oracle_pins import golden
    g = golden("hash_function.txt")
    rng = np.random.default_rng(3)
    xyz = rng.integers(-32768, 32768, size=(10 ** 6, 3))
    xyz[:8] = [[-32768, -32768, -32768], [32767, 32767, 32767], [-1, 0, 1], [0, 0, 0],
               [-32768, 32767, 0], [1, -1, -32768], [32767, -32768, -1], [-2, -3, -4]]
    for nb in (1 << 10, 1 << 20):
        p = np.array([g["prime_x"], g["prime_y"], g["prime_z"]], dtype=np.uint64)
        u = (xyz.astype(np.int64) & 0xFFFFFFFF).astype(np.uint64)
        h = ((u * p) & 0xFFFFFFFF)
        want = ((h[:, 0] ^ h[:, 1] ^ h[:, 2]) & (nb - 1)).astype(np.int64)
        f = itm._lib.itm_hash_index
        got = np.fromiter((f(int(x), int(y), int(z), nb) for x, y, z in xyz), dtype=np.int64, count=len(xyz))
        assert np.array_equal(got, want)
        sample = xyz[:2000]
        assert all(oracle.hash_index(x, y, z, nb) == want[i] for i, (x, y, z) in enumerate(sample))


_POSE_CHILD = r'''
import ctypes, sys
import numpy as np
import paper_1708_00783_gb300 as itm
intr = itm.make_intrinsics(64, 48, 60.0, 60.0, 31.5, 23.5)
R = np.array([[0.36, 0.48, -0.8], [-0.8, 0.6, 0.0], [0.48, 0.64, 0.6]])
def call(T):
    T = np.ascontiguousarray(T, dtype=np.float32).ravel()
    p = T.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the host checks come first
    return itm._lib.itm_frame_blocks_noalloc(fake, ctypes.byref(intr), p, 0.01, 0.04, 0.2, 5.0, fake, 16, fake, None)
rigid = np.eye(4); rigid[:3, :3] = R; rigid[:3, 3] = [0.5, -1.0, 2.0]
scaled = rigid.copy(); scaled[:3, :3] *= 3.0
sheared = rigid.copy(); sheared[0, 1] += 0.2
projective = rigid.copy(); projective[3, 2] = 0.1
for name, T in (("rigid", rigid), ("scaled", scaled), ("sheared", sheared), ("projective", projective)):
    print(name, call(T), flush=True)
'''


def test_noalloc_rejects_a_pose_that_is_not_rigid():
    """itm_frame_blocks_noalloc bounds its work by assuming a rigid pose; a
    scaled, sheared or projective pose is refused with ITM_ERR_ARG on the
    host, before any CUDA call (this host has no GPU: a rigid pose gets as far
    as the device lookup and fails there with ITM_ERR_CUDA)."""
    import subprocess
    import sys
    import paper_1708_00783_gb300 as itm
    r = subprocess.run([sys.executable, "-c", _POSE_CHILD], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-400:] + r.stderr[-400:]
    got = {k: int(v) for k, v in (ln.split() for ln in r.stdout.splitlines())}
    assert got["scaled"] == got["sheared"] == got["projective"] == itm.ITM_ERR_ARG
    assert got["rigid"] != itm.ITM_ERR_ARG
