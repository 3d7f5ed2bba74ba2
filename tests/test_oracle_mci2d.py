"""Pins of the 2-D MCI oracle (oracle/mci2d.py): exact reconstruction of 2-D bandlimited
real signals from separable and non-separable channel sets, agreement with the brute-force
least-squares solve of the sampling equations on arbitrary samples, and, for a product
channel set {1, d/dx} x {1, d/dy}, equality with rows-then-columns 1-D MCI (complex 1-D
oracle, real part at the end) on arbitrary samples."""
import numpy as np
import pytest

import oracle as O
from oracle import mci2d as O2
from paper_1802_10291_gb300 import synth as S

F = ("identity",)
DX, DY, DXY = ("partial", 0, 1), ("partial", 1, 0), ("partial", 1, 1)
DYY = ("partial", 2, 0)

SETS = [
    ("f", [F], (1, 1), (8, 6), (16, 18)),
    ("f,fx", [F, DX], (1, 2), (8, 6), (16, 12)),
    ("f,fy", [F, DY], (2, 1), (6, 8), (12, 24)),
    ("f,fy,fyy", [F, DY, DYY], (3, 1), (4, 6), (12, 12)),
    ("product", [F, DX, DY, DXY], (2, 2), (6, 8), (12, 16)),
    ("shift", [F, DX, DY, ("shift", 0.3, 0.7)], (2, 2), (6, 6), (12, 18)),
    ("riesz", [F, ("riesz", 0), ("riesz", 1), DXY], (2, 2), (8, 8), (16, 16)),
    ("riesz-shift", [F, ("riesz", 0), ("riesz", 1), ("shift", 0.3, 0.7)], (2, 2), (6, 8), (12, 24)),
]


@pytest.mark.parametrize("name,systems,grid,P,T", SETS, ids=[s[0] for s in SETS])
def test_exact_reconstruction(name, systems, grid, P, T):
    by, bx = O2.band(grid, P)
    a = S.trig_poly_2d(np.random.default_rng(len(systems) * 7 + P[0]), by, bx)
    g = S.channel_samples_2d(a, by, bx, systems, P)
    Q, n_sing = O2.q_table(systems, grid, P)
    assert n_sing == 0
    out = O2.mci2_direct(systems, grid, g, T)
    truth = S.sample_coeffs_2d(a, by, bx, T).real
    assert np.max(np.abs(out - truth)) <= 1e-10 * np.max(np.abs(truth))


@pytest.mark.parametrize("systems,grid,P,T", [([F, DX, DY, DXY], (2, 2), (4, 4), (8, 12)),
                                              ([F, DX, DY, ("shift", 0.3, 0.7)], (2, 2), (3, 4), (6, 8)),
                                              ([F, DY, DYY], (3, 1), (4, 3), (8, 9)),
                                              ([F], (1, 1), (6, 4), (12, 12))])
def test_matches_bruteforce_on_arbitrary_samples(systems, grid, P, T):
    g = np.random.default_rng(P[0] * 10 + P[1]).standard_normal((len(systems),) + P)
    a = O2.mci2_direct(systems, grid, g, T)
    b = O2.mci2_bruteforce(systems, grid, g, T)
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_product_channels_equal_rows_then_columns():
    """H_r of {1, i nx} x {1, i ny} is a Kronecker product, so 2-D MCI is 1-D MCI along x then
    along y; with the real part taken only at the end (complex 1-D oracle)."""
    P1, P2, s1, s2 = 6, 8, 2, 3
    g = np.random.default_rng(3).standard_normal((4, P1, P2))
    two_d = O2.mci2_direct([F, DX, DY, DXY], (2, 2), g, (s1 * P1, s2 * P2))
    sys1 = [("identity",), ("deriv", 1)]
    # rows: (f, fx) -> f on the fine x grid; (fy, fxy) -> fy on the fine x grid
    u0 = O.mci_direct_complex(sys1, np.stack([g[0], g[1]], axis=1), s2 * P2)[:, 0, :]   # P1 x T2
    u1 = O.mci_direct_complex(sys1, np.stack([g[2], g[3]], axis=1), s2 * P2)[:, 0, :]
    cols = O.mci_direct_complex(sys1, np.stack([u0.T, u1.T], axis=1), s1 * P1)[:, 0, :]  # T2 x T1
    assert np.max(np.abs(two_d - cols.T.real)) <= 1e-11 * np.max(np.abs(two_d))
    # rows-then-columns with the real part taken after each pass differs in general (even bands)
    r0 = O.mci_direct(sys1, np.stack([g[0], g[1]], axis=1), s2 * P2)[:, 0, :]
    r1 = O.mci_direct(sys1, np.stack([g[2], g[3]], axis=1), s2 * P2)[:, 0, :]
    sep = O.mci_direct(sys1, np.stack([r0.T, r1.T], axis=1), s1 * P1)[:, 0, :].T
    assert np.max(np.abs(two_d - sep)) > 1e-6


def test_singular_residue_policies():
    """{f, Laplacian, d/dx, d/dy}: the Laplacian is a sum of separable terms, so on the 2 x 2
    alias lattice H_r has rank 3 at every residue."""
    systems = [F, ("laplacian",), DX, DY]
    Q, n_sing = O2.q_table(systems, (2, 2), (4, 4))
    assert n_sing == 16
    with pytest.raises(np.linalg.LinAlgError):
        O2.q_table(systems, (2, 2), (4, 4), policy="error")
    Qz, _ = O2.q_table(systems, (2, 2), (4, 4), policy="zero")
    assert np.all(Qz == 0)
    # the pseudo-inverse gives the minimum-norm least-squares solution: the brute-force route
    g = np.random.default_rng(5).standard_normal((4, 4, 4))
    a = O2.mci2_direct(systems, (2, 2), g, (8, 8))
    b = O2.mci2_bruteforce(systems, (2, 2), g, (8, 8))
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))
