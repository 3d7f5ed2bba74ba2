"""Parity of the 2-D MCI kernels (include/mci2d.h, through the C ABI) with the 2-D oracle
(oracle/mci2d.py) and with the exact signal.

Tolerances as for 1-D: FP64 max-abs <= 1e-12 x max(1, max |ref|); FP32 max-abs <= 1e-5 x RMS
of the reference."""
import numpy as np
import pytest
import torch

from oracle import mci2d as O2
from paper_1802_10291_gb300 import mci
from paper_1802_10291_gb300 import mci2d
from paper_1802_10291_gb300 import synth as S

pytestmark = pytest.mark.gpu

F = ("identity",)
DX, DY, DXY, DYY = ("partial", 0, 1), ("partial", 1, 0), ("partial", 1, 1), ("partial", 2, 0)
DT = {"fp64": torch.float64, "fp32": torch.float32}


def run(g, systems, grid, T, prec, **kw):
    batch, M, P1, P2 = g.shape
    plan = mci2d.Plan2D(systems, grid, (P1, P2), T, precision=prec, max_batch=batch, **kw)
    x = torch.tensor(g, dtype=DT[prec], device="cuda")
    y = torch.full((batch,) + tuple(T), float("nan"), dtype=DT[prec], device="cuda")
    plan.interp(x, y)
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    return y.cpu().double().numpy(), info


def check(out, ref, prec):
    assert np.all(np.isfinite(out))
    if prec == "fp64":
        err = np.max(np.abs(out - ref))
        assert err <= 1e-12 * max(1.0, np.max(np.abs(ref))), err
    else:
        err = np.max(np.abs(out - ref)) / np.sqrt(np.mean(ref ** 2))
        assert err <= 1e-5, err
    return err


CASES = [
    ("f", [F], (1, 1), (16, 12), (32, 48)),
    ("f,fx", [F, DX], (1, 2), (12, 16), (36, 32)),
    ("f,fy,fyy", [F, DY, DYY], (3, 1), (8, 24), (16, 48)),
    ("product", [F, DX, DY, DXY], (2, 2), (16, 16), (48, 32)),
    ("shift", [F, DX, DY, ("shift", 0.3, 0.7)], (2, 2), (12, 8), (24, 32)),
    ("riesz", [F, ("riesz", 0), ("riesz", 1), DXY], (2, 2), (16, 24), (32, 48)),
    ("six", [F, DX, ("partial", 0, 2), DY, DXY, ("partial", 1, 2)], (2, 3), (8, 12), (32, 24)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,systems,grid,P,T", CASES, ids=[c[0] for c in CASES])
def test_arbitrary_samples_match_oracle(cuda_device, prec, name, systems, grid, P, T):
    g = S.rng_for(15, P[0] * 100 + P[1]).standard_normal((3, len(systems)) + P)
    out, info = run(g, systems, grid, T, prec)
    assert info["n_singular"] == 0
    ref = O2.mci2_direct(systems, grid, g, T)
    check(out, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,systems,grid,P,T", CASES[1:5], ids=[c[0] for c in CASES[1:5]])
def test_bandlimited_exact(cuda_device, prec, name, systems, grid, P, T):
    by, bx = O2.band(grid, P)
    a = S.trig_poly_2d(S.rng_for(15, 1), by, bx, 2)
    g = S.channel_samples_2d(a, by, bx, systems, P)
    out, _ = run(g, systems, grid, T, prec)
    truth = S.sample_coeffs_2d(a, by, bx, T).real
    check(out, truth, prec)
    if prec == "fp64":   # unit-scale bandlimited image: the unscaled bound holds as well
        assert np.max(np.abs(out - truth)) <= 1e-12


def test_singular_policies(cuda_device):
    """{f, Laplacian, d/dx, d/dy}: rank 3 at every residue of the 2 x 2 alias lattice."""
    systems = [F, ("laplacian",), DX, DY]
    g = S.rng_for(15, 2).standard_normal((2, 4, 8, 8))
    out, info = run(g, systems, (2, 2), (16, 16), "fp64")
    assert info["n_singular"] == 64
    check(out, O2.mci2_direct(systems, (2, 2), g, (16, 16)), "fp64")
    out, _ = run(g, systems, (2, 2), (16, 16), "fp64", singular="zero")
    assert np.max(np.abs(out)) == 0.0
    with pytest.raises(mci.MciError) as e:
        mci2d.Plan2D(systems, (2, 2), (8, 8), (16, 16), singular="error")
    assert e.value.status == mci.MCI_ERR_SINGULAR


def test_band_offset(cuda_device):
    """A band that is not centred: N1 = (-4, 0) for My P1 = 16, Mx P2 = 32 ({f, fx, fy, fxy})."""
    systems, grid, P, T, N1 = [F, DX, DY, DXY], (2, 2), (8, 16), (24, 32), (-4, 0)
    g = S.rng_for(15, 3).standard_normal((2, 4) + P)
    out, _ = run(g, systems, grid, T, "fp64", N1=N1)
    check(out, O2.mci2_direct(systems, grid, g, T, N1=N1), "fp64")


@pytest.mark.parametrize("P,T,prec", [((256, 256), (768, 768), "fp32"), ((96, 384), (192, 768), "fp64"),
                                      ((1024, 1024), (2048, 2048), "fp32")])
def test_large_bandlimited(cuda_device, P, T, prec):
    """At image sizes the oracle's direct sum is out of reach: exact reconstruction of a
    bandlimited image holds at any size."""
    systems, grid = ([F, DX, DY, DXY], (2, 2)) if P[0] <= 256 else ([F, DX], (1, 2))
    by, bx = O2.band(grid, P)
    a = S.trig_poly_2d(S.rng_for(15, 4), by, bx)
    g = S.channel_samples_2d(a, by, bx, systems, P)[None]
    out, _ = run(g, systems, grid, T, prec)
    check(out[0], S.sample_coeffs_2d(a, by, bx, T).real, prec)


def test_batch_checks(cuda_device):
    plan = mci2d.Plan2D([F, DX], (1, 2), (8, 8), (16, 16), max_batch=2)
    x = torch.zeros((3, 2, 8, 8), device="cuda")
    y = torch.zeros((3, 16, 16), device="cuda")
    plan.interp(x, y, batch=0)
    with pytest.raises(mci.MciError):
        plan.interp(x, y, batch=3)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("grid,P,T", [((5, 1), (8, 8), (40, 16)), ((1, 7), (6, 8), (12, 56)),
                                      ((2, 4), (8, 6), (16, 24)), ((3, 1), (12, 4), (36, 8))])
def test_interlaced_shift_channels(cuda_device, prec, grid, P, T):
    """Channels that are the signal shifted by (ky / (My P1), kx / (Mx P2)) of a period: the
    samples of all channels together are those of a My P1 x Mx P2 grid, each H_r is a scaled
    DFT matrix (well conditioned), and every channel count from 3 to 8 runs its own kernel."""
    My, Mx = grid
    systems = [("shift", 2 * np.pi * (j // Mx) / (My * P[0]), 2 * np.pi * (j % Mx) / (Mx * P[1]))
               for j in range(My * Mx)]
    g = S.rng_for(15, 5 + My * 10 + Mx).standard_normal((2, My * Mx) + P)
    out, info = run(g, systems, grid, T, prec)
    assert info["n_singular"] == 0
    check(out, O2.mci2_direct(systems, grid, g, T), prec)
