"""Pins of the oracle's blur-aware channel model (the open extension at the end of
Section 5.2: MCI reconstructs a signal from samples of filtered versions of it, so
a blur before sampling is one more filter on every channel).

The blur is the circular convolution with a normalised Gaussian on the output grid;
the test inputs are blurred in the SPATIAL domain (np.roll sums in the input module),
so the oracle's spectral factor beta(n) is checked against a computation that never
forms it."""
import numpy as np
import pytest

import oracle as O
from paper_1802_10291_gb300 import synth as S

F, D1, D2 = ("identity",), ("deriv", 1), ("deriv", 2)


@pytest.mark.parametrize("T,taps,sigma", [(48, 5, 1.0), (64, 7, 1.4), (30, 3, 0.7), (96, 9, 2.5)])
def test_blur_factor_is_the_spatial_convolution(T, taps, sigma):
    x = np.random.default_rng(T).standard_normal(T)
    y = S.blur_periodic(x, taps, sigma)
    beta = O.blur_factor(np.arange(T), T, taps, sigma)
    assert np.max(np.abs(np.fft.fft(y) - np.fft.fft(x) * beta)) <= 1e-12 * np.max(np.abs(np.fft.fft(x)))
    # periodic in n with period T, and beta(0) = 1 (normalised taps)
    assert np.allclose(O.blur_factor(np.arange(-T, 0), T, taps, sigma), beta, atol=1e-14)
    assert abs(O.blur_factor(0, T, taps, sigma) - 1.0) <= 1e-15


def _blurred_channels(a, band, systems, P, T, taps, sigma):
    """Samples at t_p of every channel: the exact response on the T-grid, blurred there by a
    spatial circular convolution, then every (T/P)-th point."""
    s = T // P
    chans = []
    for sy in systems:
        fine = S.sample_coeffs(a * S.response(sy, band), band, T).real
        chans.append(S.blur_periodic(fine, taps, sigma)[::s])
    return np.stack(chans)


@pytest.mark.parametrize("systems,P,s,taps,sigma", [([F, D1], 16, 3, 5, 1.0), ([F, D1, D2], 8, 2, 7, 1.4),
                                                    ([F], 12, 4, 5, 1.0), ([F, D1], 9, 3, 3, 0.8)])
def test_blur_aware_reconstruction_is_exact(systems, P, s, taps, sigma):
    M, T = len(systems), s * P
    band = S.band_of(M, P)
    a = S.trig_poly(np.random.default_rng(P * 10 + M), band)
    g = _blurred_channels(a, band, systems, P, T, taps, sigma)
    truth = S.sample_coeffs(a, band, T).real
    blurred_truth = S.blur_periodic(truth, taps, sigma)
    scale = np.max(np.abs(truth))
    aware = O.mci_direct(O.blur_systems(systems, P, T, taps, sigma), g, T)[0]
    plain = O.mci_direct(systems, g, T)[0]
    assert np.max(np.abs(aware - truth)) <= 1e-10 * scale
    # the plain channel model reconstructs the blurred signal, which differs from f
    assert np.max(np.abs(plain - blurred_truth)) <= 1e-10 * scale
    assert np.max(np.abs(plain - truth)) > 1e-3 * scale


def test_wiener_factor_closed_form():
    """f = cos(n0 t): the blurred samples give beta(n0) cos(n0 t) to the plain model, and the
    regularised model returns (1 + lam) beta^2 / (beta^2 + lam) cos(n0 t)."""
    P, s, taps, sigma, lam = 16, 3, 5, 1.0, 0.1
    T, systems = s * P, [F, D1]
    band = S.band_of(2, P)
    for n0 in (0, 3, 11, 15):
        a = np.zeros(band.size, np.complex128)
        a[band == n0] += 0.5
        a[band == -n0] += 0.5
        g = _blurred_channels(a, band, systems, P, T, taps, sigma)
        out = O.mci_direct(O.blur_systems(systems, P, T, taps, sigma, lam), g, T)[0]
        b = O.blur_factor(n0, T, taps, sigma).real
        t = 2 * np.pi * np.arange(T) / T
        expect = (1 + lam) * b * b / (b * b + lam) * np.cos(n0 * t)
        assert np.max(np.abs(out - expect)) <= 1e-11


def test_blur_aware_2d_exact_on_bandlimited_image():
    """One measured channel per axis: an image whose spectrum lies in the LR band, blurred by the
    separable taps x taps Gaussian and decimated, comes back exactly at HR."""
    P, s, taps, sigma = 12, 3, 5, 1.0
    Hh = s * P
    rng = np.random.default_rng(7)
    y, x = np.meshgrid(np.arange(Hh), np.arange(Hh), indexing="ij")
    img = np.full((Hh, Hh), 0.5)
    for _ in range(12):
        ky, kx = rng.integers(-P // 2 + 1, P // 2, size=2)
        img += 0.1 * rng.standard_normal() * np.cos(2 * np.pi * (ky * y + kx * x) / Hh + rng.uniform(0, 6.3))
    lr = S.degrade(img, s, taps, sigma)
    out = O.upsample_2d(lr, s, [F], blur=(taps, sigma, 0.0))
    assert np.max(np.abs(out - img)) <= 1e-10
    plain = O.upsample_2d(lr, s, [F])
    assert np.max(np.abs(plain - S.blur_periodic(img, taps, sigma, axes=(-2, -1)))) <= 1e-10


@pytest.mark.parametrize("lam", [0.0, 0.1])
def test_blur_aware_paper_mode_keeps_constants(lam):
    """Finite-difference channels of a constant image vanish and beta(0) = 1, so the
    blur-aware paper-mode upsampling returns the constant for any regularisation."""
    lr = np.full((8, 10), 0.3)
    out = O.upsample_2d(lr, 3, [F, D1, D2], blur=(7, 1.4, lam))
    assert out.shape == (24, 30)
    assert np.max(np.abs(out - 0.3)) <= 1e-12
