"""Pins of the oracle's complex-signal routes (Examples 4 and 5 reconstruct complex
signals; no real part is taken): exact reconstruction of complex trigonometric
polynomials, agreement with the brute-force least-squares solve, and an analytic
signal on the one-sided band of Example 4 (f, Hf with Hf = -i f there)."""
import numpy as np
import pytest

import oracle as O
from paper_1802_10291_gb300 import synth as S

F, H, D1, D2 = ("identity",), ("hilbert",), ("deriv", 1), ("deriv", 2)


def _coeffs(rng, band):
    return (rng.standard_normal(len(band)) + 1j * rng.standard_normal(len(band))) / (1.0 + np.abs(band))


@pytest.mark.parametrize("systems,P,s", [([F], 16, 2), ([F, D1], 16, 3), ([F, H, D1], 12, 2),
                                         ([F, ("shift", 0.5)], 8, 4), ([D1, F], 10, 2)])
def test_complex_exact_reconstruction(systems, P, s):
    M = len(systems)
    N1 = O.default_n1(M, P)
    band = np.arange(N1, N1 + M * P)
    rng = np.random.default_rng(M * 100 + P)
    a = _coeffs(rng, band)
    if M == 3 and systems[1] == H:
        # the singular residue of {f, Hf, f'} holds n = -P, 0, P: exact only when all vanish
        a[np.isin(band, [-P, 0, P])] = 0.0
    g = O.samples_from_coeffs_complex(a, band, systems, P)
    T = s * P
    for op in ("f", "hilbert", "deriv"):
        got = O.mci_direct_complex(systems, g, T, outputs=(op,))[0]
        truth = O.truth_from_coeffs_complex(a, band, T, op)
        assert np.max(np.abs(got - truth)) <= 1e-11 * max(1.0, np.max(np.abs(truth)))


@pytest.mark.parametrize("systems,P", [([F, D1], 8), ([F, H], 6), ([F, H, D1], 4)])
def test_complex_matches_bruteforce_on_arbitrary_samples(systems, P):
    rng = np.random.default_rng(P)
    g = rng.standard_normal((len(systems), P)) + 1j * rng.standard_normal((len(systems), P))
    T = 4 * P
    a = O.mci_direct_complex(systems, g, T, outputs=("f", "hilbert"))
    b = O.mci_bruteforce_complex(systems, g, T, outputs=("f", "hilbert"))
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_analytic_signal_one_sided_band():
    """Example 4: f analytic (a(n) = 0 for n < 0), band {0 .. 2P - 1}, channels f and f'.
    Hilbert output equals -i f on a one-sided positive band."""
    P = 16
    band = np.arange(0, 2 * P)
    rng = np.random.default_rng(4)
    a = _coeffs(rng, band)
    a[0] = 0.0                        # sgn(0) = 0: keep the identity Hf = -i f exact
    g = O.samples_from_coeffs_complex(a, band, [F, D1], P)
    out = O.mci_direct_complex([F, D1], g, 8 * P, N1=0, outputs=("f", "hilbert"))
    f_true = O.truth_from_coeffs_complex(a, band, 8 * P, "f")
    assert np.max(np.abs(out[0] - f_true)) <= 1e-11 * np.max(np.abs(f_true))
    assert np.max(np.abs(out[1] + 1j * out[0])) <= 1e-11 * np.max(np.abs(f_true))
