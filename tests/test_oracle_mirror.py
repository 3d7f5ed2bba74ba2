"""Pins of the oracle's mirror-boundary 2-D upsampling (CPU).

Mirror mode interpolates the half-sample-symmetric extension of the image, so a product of
half-sample cosines cos(pi k (n + 1/2) / P), which is a trigonometric polynomial of integer
frequency k on the extension of length 2P, comes back exactly at every output point when
the single channel {f} carries it (its system matrix is invertible on the band); the
periodic wrap of the same image cannot, for odd k (the wrapped image jumps at its edges).
"""
import numpy as np
import pytest

import oracle

F = ("identity",)
D1 = ("deriv", 1)


def _half_cosines(h, w, k1, k2, s):
    n1, n2 = np.arange(h)[:, None], np.arange(w)[None, :]
    img = np.cos(np.pi * k1 * (n1 + 0.5) / h) * np.cos(np.pi * k2 * (n2 + 0.5) / w)
    m1, m2 = np.arange(s * h)[:, None] / s, np.arange(s * w)[None, :] / s
    exact = np.cos(np.pi * k1 * (m1 + 0.5) / h) * np.cos(np.pi * k2 * (m2 + 0.5) / w)
    return img, exact


@pytest.mark.parametrize("h,w,k1,k2,s", [(12, 16, 3, 5, 2), (10, 8, 1, 3, 3), (16, 12, 7, 2, 4)])
def test_mirror_reproduces_half_sample_cosines(h, w, k1, k2, s):
    img, exact = _half_cosines(h, w, k1, k2, s)
    got = oracle.upsample_2d_mirror(img, s, [F])
    assert got.shape == (s * h, s * w)
    assert np.max(np.abs(got - exact)) < 1e-10


def test_periodic_wrap_misses_them():
    img, exact = _half_cosines(12, 16, 3, 5, 2)
    assert np.max(np.abs(oracle.upsample_2d(img, 2, [F]) - exact)) > 0.05


def test_mirror_keeps_the_samples_and_constants():
    rng = np.random.default_rng(5)
    img = rng.random((9, 14))
    for s in (2, 3):
        out = oracle.upsample_2d_mirror(img, s, [F, D1])
        # output pixel (s i, s j) sits on input sample (i, j): the method interpolates
        assert np.allclose(out[::s, ::s], img, atol=1e-10)
    assert np.allclose(oracle.upsample_2d_mirror(np.full((6, 10), 0.3), 3, [F, D1]), 0.3, atol=1e-12)
