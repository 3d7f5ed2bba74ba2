"""Complex-signal mode (Examples 4, 5: complex samples, complex outputs, no real part)
against the oracle's complex sum formula and the exact values from the coefficients."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci

pytestmark = pytest.mark.gpu

F, H, D1, D2 = ("identity",), ("hilbert",), ("deriv", 1), ("deriv", 2)
CDT = {"fp64": torch.complex128, "fp32": torch.complex64}
TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _coeffs(rng, band):
    return (rng.standard_normal(len(band)) + 1j * rng.standard_normal(len(band))) / (1.0 + np.abs(band))


def _run(systems, g, T, prec, outputs=("f",), N1=None):
    batch, M, P = g.shape
    plan = mci.Plan(systems, P, T, outputs=outputs, precision=prec, max_batch=batch, N1=N1,
                    complex_signal=True)
    x = torch.tensor(g, dtype=CDT[prec], device="cuda")
    y = torch.full((batch, len(outputs), T), complex("nan"), dtype=CDT[prec], device="cuda")
    plan.interp_1d(torch.view_as_real(x), torch.view_as_real(y), batch=batch)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    plan.close()
    return y.cpu().numpy().astype(np.complex128)


def _check(got, ref, prec, scale=None):
    """FP64: max-abs error <= 1e-12 x scale (default max(1, max |ref|); for a trigonometric
    sum the natural scale of its rounding error is the l1 norm of its coefficients).
    FP32: max-abs error <= 1e-5 x RMS of ref."""
    assert np.all(np.isfinite(got))
    if prec == "fp64":
        sc = max(1.0, np.max(np.abs(ref))) if scale is None else scale
        assert np.max(np.abs(got - ref)) <= TOL[prec] * sc
    else:
        assert np.max(np.abs(got - ref)) <= TOL[prec] * np.sqrt(np.mean(np.abs(ref) ** 2))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("systems,P,s", [([F], 64, 4), ([F, D1], 128, 4), ([F, H, D1], 256, 4),
                                         ([F, ("shift", 0.7)], 96, 2), ([F, D1, D2], 48, 3),
                                         ([F, H, D1], 2048, 2), ([F, D1], 4096, 2)])
def test_complex_trig_polynomials_exact(cuda_device, prec, systems, P, s):
    M = len(systems)
    N1 = O.default_n1(M, P)
    band = np.arange(N1, N1 + M * P)
    rng = np.random.default_rng(P + M)
    a = np.stack([_coeffs(rng, band) for _ in range(3)])
    if M == 3 and systems[1] == H:
        a[:, np.isin(band, [-P, 0, P])] = 0.0    # the singular residue
    g = np.stack([O.samples_from_coeffs_complex(a[b], band, systems, P) for b in range(3)])
    T = s * P
    # the largest size keeps one output so that an FP64 tile (max(M, s n_out) buffers of P
    # complex values) fits in shared memory
    outs = ("f", "hilbert", "deriv") if P < 4096 else ("f",)
    got = _run(systems, g, T, prec, outs)
    truth = np.stack([[O.truth_from_coeffs_complex(a[b], band, T, o) for o in outs] for b in range(3)])
    for o, op in enumerate(outs):
        l1 = np.max(np.sum(np.abs(a * O.out_operator(op, band)[None, :]), axis=1))
        _check(got[:, o], truth[:, o], prec, scale=max(1.0, l1))
        if prec == "fp64" and op != "deriv":   # unit-scale outputs: the unscaled bound too
            assert np.max(np.abs(got[:, o] - truth[:, o])) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("systems,P", [([F, D1], 16), ([F, H], 32), ([F, H, D1], 64)])
def test_complex_arbitrary_samples_match_oracle(cuda_device, prec, systems, P):
    rng = np.random.default_rng(7 * P)
    g = rng.standard_normal((4, len(systems), P)) + 1j * rng.standard_normal((4, len(systems), P))
    T = 4 * P
    got = _run(systems, g, T, prec, ("f", "hilbert"))
    ref = O.mci_direct_complex(systems, g, T, outputs=("f", "hilbert"))
    _check(got, ref, prec)


def test_analytic_one_sided_band(cuda_device):
    """Example 4: a(n) = 0 for n < 0, band {0 .. 2P - 1} (N1 = 0), channels f and f'."""
    P = 64
    band = np.arange(0, 2 * P)
    rng = np.random.default_rng(4)
    a = _coeffs(rng, band)
    a[0] = 0.0
    g = O.samples_from_coeffs_complex(a, band, [F, D1], P)[None]
    got = _run([F, D1], g, 8 * P, "fp64", ("f", "hilbert"), N1=0)[0]
    f_true = O.truth_from_coeffs_complex(a, band, 8 * P, "f")
    assert np.max(np.abs(got[0] - f_true)) <= 1e-12 * np.max(np.abs(f_true))
    assert np.max(np.abs(got[1] + 1j * got[0])) <= 1e-12 * np.max(np.abs(f_true))


def test_complex_uneven_batch_host_grouped(cuda_device):
    systems, Ps = [F, H, D1], [64, 256, 96]
    rng = np.random.default_rng(11)
    cls = rng.integers(0, 3, 20).astype(np.int32)
    cls[:3] = [0, 1, 2]
    gs = [rng.standard_normal((3, Ps[c])) + 1j * rng.standard_normal((3, Ps[c])) for c in cls]
    T = [4 * p for p in Ps]
    plan = mci.Plan(systems, Ps, T, max_batch=20, complex_signal=True)
    flat = np.concatenate([g.ravel() for g in gs])
    x = torch.view_as_real(torch.tensor(flat, dtype=torch.complex64, device="cuda"))
    n_out = sum(T[c] for c in cls)
    y = torch.full((n_out,), complex("nan"), dtype=torch.complex64, device="cuda")
    mci.mci_interp_1d(plan.handle, x, None, torch.view_as_real(y), None, cls, 20)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    yh = y.cpu().numpy().astype(np.complex128)
    pos = 0
    for b, c in enumerate(cls):
        ref = O.mci_direct_complex(systems, gs[b], T[c])[0]
        _check(yh[pos:pos + T[c]], ref, "fp32")
        pos += T[c]
    plan.close()


def test_complex_mode_argument_checks(cuda_device):
    import ctypes
    lib = mci.load()
    for kw, st in ((dict(channels="fd", systems=[F, D1]), mci.MCI_ERR_INVALID_ARG),
                   (dict(max_images=1, max_intermediate=10, systems=[F]), mci.MCI_ERR_INVALID_ARG),
                   (dict(P=8192, T=8192, systems=[F]), mci.MCI_ERR_UNSUPPORTED_SIZE)):
        systems = kw.pop("systems")
        P, T = kw.pop("P", 64), kw.pop("T", 256)
        d = mci.make_desc(systems, P, T, complex_signal=True, max_batch=1, **kw)
        h = ctypes.c_void_p()
        assert lib.mci_plan(ctypes.byref(h), ctypes.byref(d), None) == st
