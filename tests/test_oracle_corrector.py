"""Pins of the corrector's CPU oracle: finite differences of the loss, and convolutions
that reduce to known operations."""
import numpy as np

from oracle import corrector as C


def small_params(rng, scale=0.3):
    flat = []
    for ci, co in C.LAYERS:
        flat += [rng.standard_normal(co * ci * 9) * scale / np.sqrt(ci), rng.standard_normal(co) * 0.1]
    return np.concatenate(flat)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = small_params(rng)
    x = rng.random((2, 6, 7))
    hr = rng.random((2, 6, 7))
    L, g = C.loss_grad(p, x, hr)
    assert abs(L - C.loss(p, x, hr)) < 1e-14
    idx = rng.choice(p.size, 40, replace=False)
    idx = np.concatenate([idx, [0, 287, 288, p.size - 1, p.size - 2]])   # first/last weights and biases
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (C.loss(p + e, x, hr) - C.loss(p - e, x, hr)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_conv_identity_and_shift():
    rng = np.random.default_rng(2)
    x = rng.random((1, 3, 5, 6))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1] = 1.0                           # identity tap
    np.testing.assert_allclose(C.conv(x, w, np.zeros(3)), x)
    w2 = np.zeros((1, 1, 3, 3))
    w2[0, 0, 2, 0] = 1.0                              # reads x(p + (1, -1))
    y = C.conv(x[:, :1], w2, np.array([0.5]))
    np.testing.assert_allclose(y[0, 0], np.roll(x[0, 0], (-1, 1), axis=(0, 1)) + 0.5)


def test_zero_last_layer_returns_input():
    rng = np.random.default_rng(3)
    p = small_params(rng)
    p[-(32 * 9 + 1):] = 0
    x = rng.random((1, 8, 8))
    pred, _ = C.forward(p, x)
    np.testing.assert_array_equal(pred, x)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265], np.float32)
    r = C.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7 and r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12
