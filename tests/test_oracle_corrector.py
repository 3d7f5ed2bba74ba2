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


def _tap(w, co, ci, dy, dx, v):
    """Weight of output channel co on input channel ci at offset (dy, dx): the conv reads
    x(p + (dy, dx)), p = (row, column)."""
    w[co, ci, dy + 1, dx + 1] = v


def test_forward_composition_closed_form():
    """Each layer made of single taps (identity, negation, shifts) and biases, so that the
    five-layer output has a closed form written here with explicit periodic indexing.  A ReLU
    after the last layer, a missing ReLU after any hidden layer, a swapped layer order or a
    wrong shift direction changes the result (the input takes both signs)."""
    H, W = 7, 9
    rng = np.random.default_rng(11)
    x = rng.uniform(-1.0, 1.0, (2, H, W))
    layers = [(np.zeros((co, ci, 3, 3)), np.zeros(co)) for ci, co in C.LAYERS]
    (w1, b1), (w2, b2), (w3, b3), (w4, b4), (w5, b5) = layers
    # layer 1: a1 = [relu(x), relu(-x), relu(x(i, j+1)), relu(-1) = 0, ...]
    _tap(w1, 0, 0, 0, 0, 1.0)
    _tap(w1, 1, 0, 0, 0, -1.0)
    _tap(w1, 2, 0, 0, 1, 1.0)
    b1[3:] = -1.0
    # layer 2: a2 = [relu(a1_0 + a1_1) = |x|, relu(a1_0 - a1_1 - 0.5) = relu(x - 0.5),
    #                relu(a1_2(i+1, j)) = relu(x(i+1, j+1))]
    _tap(w2, 0, 0, 0, 0, 1.0)
    _tap(w2, 0, 1, 0, 0, 1.0)
    _tap(w2, 1, 0, 0, 0, 1.0)
    _tap(w2, 1, 1, 0, 0, -1.0)
    b2[1] = -0.5
    _tap(w2, 2, 2, 1, 0, 1.0)
    # layer 3: a3 = [relu(a2_0 - a2_1), relu(0.3 - a2_2), relu(a2_1)]
    _tap(w3, 0, 0, 0, 0, 1.0)
    _tap(w3, 0, 1, 0, 0, -1.0)
    _tap(w3, 1, 2, 0, 0, -1.0)
    b3[1] = 0.3
    _tap(w3, 2, 1, 0, 0, 1.0)
    # layer 4: a4 = [relu(a3_0 - a3_1 - 2 a3_2(i, j-1)), relu(a3_1)]
    _tap(w4, 0, 0, 0, 0, 1.0)
    _tap(w4, 0, 1, 0, 0, -1.0)
    _tap(w4, 0, 2, 0, -1, -2.0)
    _tap(w4, 1, 1, 0, 0, 1.0)
    # layer 5 (no ReLU): out = a4_0 - 2 a4_1(i-1, j) - 0.1
    _tap(w5, 0, 0, 0, 0, 1.0)
    _tap(w5, 0, 1, -1, 0, -2.0)
    b5[0] = -0.1
    flat = C.flatten(layers)

    relu = lambda v: np.maximum(v, 0.0)                               # noqa: E731
    r, c = np.arange(H)[:, None], np.arange(W)[None, :]

    def at(v, dy, dx):                 # v(i + dy, j + dx), periodic
        return v[:, (r + dy) % H, (c + dx) % W]

    a2_0 = np.abs(x)
    a2_1 = relu(x - 0.5)
    a2_2 = relu(at(x, 1, 1))
    a3_0 = relu(a2_0 - a2_1)
    a3_1 = relu(0.3 - a2_2)
    a3_2 = relu(a2_1)
    a4_0 = relu(a3_0 - a3_1 - 2.0 * at(a3_2, 0, -1))
    a4_1 = relu(a3_1)
    out = a4_0 - 2.0 * at(a4_1, -1, 0) - 0.1
    assert np.min(out) < -0.05 and np.max(out) > 0.05                 # both signs reach the output
    pred, cache = C.forward(flat, x)
    np.testing.assert_allclose(pred, x + out, rtol=0, atol=1e-14)
    np.testing.assert_allclose(cache[2][:, 2], a2_2, rtol=0, atol=1e-14)
    hr = rng.uniform(0.0, 1.0, x.shape)
    assert abs(C.loss(flat, x, hr) - np.mean((x + out - hr) ** 2)) < 1e-14
