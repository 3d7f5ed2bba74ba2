"""Pins of the oracle's bound of Eq. (errorestimate): it is an upper bound of Eq.
(averageerror) (Cauchy-Schwarz), and equality holds for one identity channel."""
import numpy as np
import pytest

import oracle as O

F, H, D1, D2 = ("identity",), ("hilbert",), ("deriv", 1), ("deriv", 2)


def _coeffs(seed, decay):
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 100001)

    def fn(n):
        return np.exp(1j * ph[np.abs(n) % ph.size] * np.sign(n)) / (1.0 + np.abs(n)) ** decay
    return fn


def test_identity_channel_bound_is_exact():
    fn = _coeffs(1, 1.5)
    e = O.averaged_error(fn, [F], 32, n_max=400)
    b = O.error_bound(fn, [F], 32, n_max=400)
    assert abs(e - b) <= 1e-13 * b


@pytest.mark.parametrize("systems,P", [([F, D1], 16), ([F, H], 16), ([F, H, D1], 12),
                                       ([F, D1, D2], 10), ([F, ("shift", 0.3)], 16)])
def test_bound_dominates_averaged_error(systems, P):
    for seed, decay in ((2, 2.0), (3, 3.0)):
        fn = _coeffs(seed, decay)
        e = O.averaged_error(fn, systems, P, n_max=12 * P * len(systems))
        b = O.error_bound(fn, systems, P, n_max=12 * P * len(systems))
        assert e > 0 and b >= e * (1 - 1e-12)
