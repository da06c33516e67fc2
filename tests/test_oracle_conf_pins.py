"""Pins of the oracle's learned-confidence part (features, MLP, gradients).

The paper has no learned weight; the definitions are this repository's (the
depth patch, the depth normal, a 52-64-64-1 ReLU network with a sigmoid
output and a cross-entropy loss).  Each is checked against mathematics that
fixes it: the patch and normal of planes in closed form, networks built to
compute a known value, and the gradient against central finite differences.
"""

import numpy as np
import pytest

import oracle
from synth import Intrinsics

INTR = Intrinsics(64, 48, 60.0, 60.0, 31.5, 23.5)
MU = 0.02


def plane_depth(N, c, intr=INTR):
    """Exact depth (fp64) of the plane N . P = c seen through every pixel."""
    u = np.arange(intr.width)[None, :]
    v = np.arange(intr.height)[:, None]
    rx = (u - intr.cx) / intr.fx
    ry = (v - intr.cy) / intr.fy
    return c / (N[0] * rx + N[1] * ry + N[2])


def test_fronto_parallel_plane_has_flat_patch_and_facing_normal():
    D = np.full((INTR.height, INTR.width), 1.3, dtype=np.float32)
    x, ok = oracle.conf_features(D, INTR.as_array(), MU, 20, 17)
    assert ok
    assert np.all(x[:49] == 0.0)
    np.testing.assert_allclose(x[49:], [0.0, 0.0, -1.0], atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tilted_plane_patch_and_normal_closed_form(seed):
    rng = np.random.default_rng(seed)
    N = rng.normal(size=3)
    N[2] = -abs(N[2]) - 1.0                       # a plane the camera faces
    N /= np.linalg.norm(N)
    c = N @ np.array([0.0, 0.0, 1.5])
    Dt = plane_depth(N, c)
    D = Dt.astype(np.float32)
    u, v = 30, 22
    x, ok = oracle.conf_features(D, INTR.as_array(), MU, u, v)
    assert ok
    for i in range(-3, 4):
        for j in range(-3, 4):
            want = np.clip((Dt[v + i, u + j] - Dt[v, u]) / MU, -4, 4)
            assert abs(x[(i + 3) * 7 + (j + 3)] - want) < 1e-4
    np.testing.assert_allclose(x[49:], N, atol=2e-3)   # the plane's normal, facing the camera


def test_borders_invalid_pixels_and_clamp():
    D = np.full((INTR.height, INTR.width), 2.0, dtype=np.float32)
    D[:, 33:] = 3.0                                  # a 1 m step: features clamp to +4
    D[10, 11] = 0.0                                  # a hole
    x, ok = oracle.conf_features(D, INTR.as_array(), MU, 31, 20)
    assert ok
    assert x[(0 + 3) * 7 + (2 + 3)] == 4.0 and x[(0 + 3) * 7 + (1 + 3)] == 0.0
    x, ok = oracle.conf_features(D, INTR.as_array(), MU, 0, 0)   # corner: outside entries are 0
    assert ok and np.all(x[:3 * 7].reshape(3, 7) == 0.0) and np.all(x[49:] == 0.0)
    x, ok = oracle.conf_features(D, INTR.as_array(), MU, 11, 11)  # hole above: no normal
    assert ok and x[(-1 + 3) * 7 + 3] == 0.0 and np.all(x[49:] == 0.0)
    x, ok = oracle.conf_features(D, INTR.as_array(), MU, 11, 10)  # the hole itself
    assert not ok and not x.any()


def _zeros():
    return np.zeros(oracle.N_PARAMS, dtype=np.float32)


def _views(P):
    nf, nh = oracle.N_FEATURES, oracle.N_HIDDEN
    o = 0
    W1 = P[o:o + nh * nf].reshape(nh, nf); o += nh * nf
    b1 = P[o:o + nh]; o += nh
    W2 = P[o:o + nh * nh].reshape(nh, nh); o += nh * nh
    b2 = P[o:o + nh]; o += nh
    w3 = P[o:o + nh]; o += nh
    b3 = P[o:o + 1]
    return W1, b1, W2, b2, w3, b3


def test_forward_of_constructed_networks():
    P = _zeros()
    W1, b1, W2, b2, w3, b3 = _views(P)
    b3[0] = 0.7
    x = np.zeros(52)
    o, h1, h2 = oracle.mlp_forward(P, x)
    assert o == pytest.approx(0.7) and not h1.any() and not h2.any()
    # o = 3 * relu(2 * relu(x25)) + b3 with x25 = 0.5 (exact in bfloat16)
    W1[0, 25] = 1.0
    W2[0, 0] = 2.0
    w3[0] = 3.0
    x[25] = 0.5
    o, h1, h2 = oracle.mlp_forward(P, x)
    assert o == pytest.approx(3.0 + 0.7) and h1[0] == 0.5 and h2[0] == 1.0
    x[25] = -0.5                                      # ReLU cuts it
    o, _, _ = oracle.mlp_forward(P, x)
    assert o == pytest.approx(0.7)
    # rounding to bfloat16: 1 + 2^-9 rounds to 1 (ties to even would keep 1)
    x[25] = 1.0 + 2.0 ** -9
    o, _, _ = oracle.mlp_forward(P, x, round_bf16=True)
    assert o == pytest.approx(6.0 + 0.7)
    o, _, _ = oracle.mlp_forward(P, x, round_bf16=False)
    assert o == pytest.approx(6.0 * (1.0 + 2.0 ** -9) + 0.7)


def test_forward_rounds_each_product_input_to_bfloat16():
    """Both products take bfloat16 inputs (as the tensor cores do): the
    features before layer 1 and the layer-1 activations before layer 2.
    Each case is built so that only one of the two roundings decides it."""
    P = _zeros()
    W1, b1, W2, b2, w3, b3 = _views(P)
    # features: x = 1 + 2^-8 is a tie and rounds to 1; with the weight 1.5
    # the activation 1.5 is exact, while 1.5 (1 + 2^-8) would round up to
    # 1.5 + 2^-7 before layer 2
    W1[0, 10], W2[0, 0], w3[0] = 1.5, 1.0, 1.0
    x = np.zeros(52)
    x[10] = 1.0 + 2.0 ** -8
    o, h1, _ = oracle.mlp_forward(P, x, round_bf16=True)
    assert o == 1.5 and h1[0] == 1.5
    # layer-1 activation: an exact feature plus the float bias 2^-9 gives
    # 1 + 2^-9, which rounds to 1 before layer 2
    P = _zeros()
    W1, b1, W2, b2, w3, b3 = _views(P)
    W1[1, 11], b1[1], W2[2, 1], w3[2] = 1.0, 2.0 ** -9, 1.0, 1.0
    x = np.zeros(52)
    x[11] = 1.0
    o, h1, h2 = oracle.mlp_forward(P, x, round_bf16=True)
    assert h1[1] == 1.0 + 2.0 ** -9 and h2[2] == 1.0 and o == 1.0
    o, _, _ = oracle.mlp_forward(P, x, round_bf16=False)
    assert o == 1.0 + 2.0 ** -9


def test_forward_uses_both_hidden_biases():
    P = _zeros()
    W1, b1, W2, b2, w3, b3 = _views(P)
    b1[3], W2[3, 3], w3[3] = 0.5, 1.0, 2.0     # 2 relu(relu(0.5)) = 1
    b2[4], w3[4] = 0.25, 4.0                   # 4 relu(0.25) = 1
    o, h1, h2 = oracle.mlp_forward(P, np.zeros(52))
    assert o == pytest.approx(2.0) and h1[3] == 0.5 and h2[3] == 0.5 and h2[4] == 0.25


def test_bfloat16_rounds_to_nearest_even():
    """bfloat16 keeps 8 significant bits: below half an ulp rounds down, above
    rounds up, an exact half goes to the even neighbour."""
    ulp = 2.0 ** -7
    vals = np.array([1 + 0.4 * ulp, 1 + 0.6 * ulp, 1 + 0.5 * ulp, 1 + 1.5 * ulp, -(1 + 0.6 * ulp), 3.0],
                    dtype=np.float32)
    want = np.array([1.0, 1 + ulp, 1.0, 1 + 2 * ulp, -(1 + ulp), 3.0], dtype=np.float32)
    assert np.array_equal(oracle.bf16(vals), want)


def test_loss_at_zero_logit_is_log2():
    X = np.random.default_rng(0).normal(size=(10, 52))
    y = np.array([0, 1] * 5, dtype=np.float32)
    loss, g = oracle.mlp_loss_grad(_zeros(), X, y)
    assert loss == pytest.approx(np.log(2.0))
    _, _, _, _, _, gb3 = _views(g)
    assert gb3[0] == pytest.approx(0.0)               # mean of (0.5 - y)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    P = (rng.normal(size=oracle.N_PARAMS) * 0.2).astype(np.float32)
    X = rng.normal(size=(16, 52))
    y = (rng.uniform(size=16) > 0.5).astype(np.float32)
    loss, g = oracle.mlp_loss_grad(P, X, y, round_bf16=False)
    idx = rng.choice(oracle.N_PARAMS, size=150, replace=False)
    idx = np.concatenate([idx, [oracle.N_PARAMS - 1]])
    P64 = P.astype(np.float64)
    bad = []
    for i in idx:
        # finite differences in the parameter's float32 representation
        h = 1e-4 * max(abs(P64[i]), 1e-1)
        Pp, Pm = P.copy(), P.copy()
        Pp[i] = np.float32(P64[i] + h)
        Pm[i] = np.float32(P64[i] - h)
        hh = (np.float64(Pp[i]) - np.float64(Pm[i])) / 2
        fd = (oracle.mlp_loss_grad(Pp, X, y, False)[0] - oracle.mlp_loss_grad(Pm, X, y, False)[0]) / (2 * hh)
        if not abs(fd - g[i]) <= 1e-4 * max(1.0, abs(g[i])) + 2e-6:
            bad.append((i, fd, g[i]))
    # a step may still cross a ReLU kink of one sample; allow 1% such coordinates
    assert len(bad) <= len(idx) // 100, bad


def test_confidence_map_is_zero_without_depth_and_in_unit_interval():
    rng = np.random.default_rng(5)
    P = (rng.normal(size=oracle.N_PARAMS) * 0.1).astype(np.float32)
    D = np.full((INTR.height, INTR.width), 1.5, dtype=np.float32)
    D[5:9, 5:9] = 0.0
    w = oracle.conf_weights(D, INTR.as_array(), MU, P)
    assert np.all(w[5:9, 5:9] == 0.0)
    m = D > 0
    assert np.all((w[m] > 0.0) & (w[m] < 1.0))
