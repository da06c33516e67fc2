"""The C ABI library loads and exports every function the header declares.
No GPU calls: symbol presence and the host-only functions (the hash function
and the tracker's Gauss-Newton step)."""

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
