"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 path max-abs error <= 1e-12 on unit-scale signals; FP32 path
max-abs error <= 1e-5 x RMS of the oracle output (relative to signal RMS).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci
from paper_1802_10291_gb300 import synth as S

pytestmark = pytest.mark.gpu

F, H, D1, D2 = ("identity",), ("hilbert",), ("deriv", 1), ("deriv", 2)
TOL = {"fp64": 1e-12, "fp32": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32}


def run_1d(g, systems, T, prec, outputs=("f",), N1=None, **kw):
    batch, M_in, P = g.shape
    plan = mci.Plan(systems, P, T, outputs=outputs, precision=prec, max_batch=batch,
                    N1=N1, **kw)
    x = torch.tensor(g, dtype=DT[prec], device="cuda")
    y = torch.full((batch, len(outputs), T), float("nan"), dtype=DT[prec], device="cuda")
    plan.interp_1d(x, y)
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    assert info["device_status"] == 0
    return y.cpu().double().numpy()


def check(out, ref, prec, plain=False):
    """FP64: max-abs error <= 1e-12, scaled by max(1, max |ref|) unless plain (unit-scale
    bandlimited cases assert the unscaled bound); FP32: max-abs <= 1e-5 x RMS of ref."""
    assert np.all(np.isfinite(out))
    if prec == "fp64":
        err = np.max(np.abs(out - ref))
        assert err <= TOL[prec] * (1.0 if plain else max(1.0, np.max(np.abs(ref)))), err
    else:
        err = np.max(np.abs(out - ref)) / np.sqrt(np.mean(ref ** 2))
        assert err <= TOL[prec], err
    return err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_exactness_m2_p64_t4096(cuda_device, prec):
    """M = 2 {f, f'}, P = 64, band {-64..63} with a(-64) = 0, f and Hf at T = 4096."""
    systems = [F, D1]
    band = S.band_of(2, 64)
    a = S.trig_poly(S.rng_for(0), band, 5)
    g = S.channel_samples(a, band, systems, 64)
    out = run_1d(g, systems, 4096, prec, outputs=("f", "hilbert"))
    ref = O.mci_direct(systems, g, 4096, outputs=("f", "hilbert"))
    check(out, ref, prec, plain=True)
    truth = np.stack([[O.truth_from_coeffs(a[b], band, 4096, o) for o in ("f", "hilbert")]
                      for b in range(5)])
    check(out, truth, prec, plain=True)


CASES = [
    ([F], 4, 2), ([F], 8, 3), ([F], 12, 2), ([F], 16, 1), ([F, D1], 32, 4), ([F, H, D1], 64, 4),
    ([F, D1, D2], 48, 2), ([F, H], 96, 3), ([F, ("shift", 0.4)], 24, 2), ([D1, F], 128, 2),
    ([F, H, D1], 256, 4), ([F], 384, 2), ([F, D1], 768, 2), ([F, H, D1], 1024, 4),
    ([F, H, D1], 2048, 4), ([F, H, D1], 4096, 4), ([F, H, D1], 4096, 2), ([F, D1], 1536, 2),
    ([F], 8192, 1),
]


def outputs_for(P, s, prec):
    """f, Hf, f' up to P = 2048; f and Hf above.  The FP64 tile of the P = 4096, s = 4 class
    (the batched workload's largest class) holds s x n_out phase buffers of P/2 complex
    values: f alone fits in shared memory, which is how that workload runs."""
    if P <= 2048:
        return ("f", "hilbert", "deriv")
    if prec == "fp64" and P == 4096 and s == 4:
        return ("f",)
    return ("f", "hilbert")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("systems,P,s", CASES, ids=lambda v: str(v))
def test_random_samples(cuda_device, prec, systems, P, s):
    """Arbitrary (not bandlimited) samples; batch with a ragged last tile; f, Hf, f'."""
    rng = S.rng_for(1, P * 7 + s)
    M = len(systems)
    batch = 3 + (4096 // P if P <= 4096 else 1) + 1
    g = rng.standard_normal((batch, M, P))
    T = s * P
    outs = outputs_for(P, s, prec)
    out = run_1d(g, systems, T, prec, outputs=outs)
    sel = np.unique(np.r_[0, 1, batch - 1])
    ref = O.mci_direct(systems, g[sel], T, outputs=outs)
    check(out[sel], ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_smooth_periodic_non_bandlimited(cuda_device, prec):
    systems = [F, H, D1]
    g, _, _ = S.signal_batch_1d(S.rng_for(1, 5), 512, 6, systems, "smooth")
    out = run_1d(g, systems, 2048, prec, outputs=("f", "hilbert"))
    ref = O.mci_direct(systems, g, 2048, outputs=("f", "hilbert"))
    check(out, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_singular_residue_policies(cuda_device, prec):
    """M = 3 {f, Hf, f'} on {-3P/2 .. 3P/2 - 1}: one singular residue (n = -P)."""
    systems = [F, H, D1]
    P = 64
    g = S.rng_for(1, 9).standard_normal((4, 3, P))
    for policy in ("pinv", "zero"):
        out = run_1d(g, systems, 4 * P, prec, singular=policy)
        ref = O.mci_direct(systems, g, 4 * P, policy=policy)
        check(out, ref, prec)
    plan = mci.Plan(systems, P, 4 * P, precision=prec, max_batch=1)
    assert plan.info()["n_singular"] == 1
    plan.close()
    with pytest.raises(mci.MciError) as ei:
        mci.Plan(systems, P, 4 * P, precision=prec, max_batch=1, singular="error")
    assert ei.value.status == mci.MCI_ERR_SINGULAR


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_band_offsets(cuda_device, prec):
    systems = [F, D1]
    P = 32
    g = S.rng_for(1, 10).standard_normal((3, 2, P))
    for N1 in (-64, -40, 0, 17):
        out = run_1d(g, systems, 2 * P, prec, N1=N1, outputs=("f", "deriv"))
        ref = O.mci_direct(systems, g, 2 * P, N1=N1, outputs=("f", "deriv"))
        check(out, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fd_channels(cuda_device, prec):
    """One measured channel, derivative channels from centred differences (Section 5.2)."""
    for systems in ([F, D1], [F, D1, D2]):
        x = S.rng_for(1, 11).standard_normal((5, 1, 128))
        out = run_1d(x, systems, 512, prec, channels="fd")
        ref = O.mci_direct(systems, O.fd_channels(x[:, 0], systems), 512)
        check(out, ref, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("packed", [True, False])
@pytest.mark.parametrize("where", ["device", "host"])
def test_uneven_batch(cuda_device, prec, packed, where):
    """Signals of several sizes in one call; size classes in device memory (grouped and
    launched on the device) or in host memory (grouped and launched from the host)."""
    systems = [F, H, D1]
    Ps = [256, 64, 512, 24]
    rng = S.rng_for(1, 12)
    batch = 41
    cls = rng.integers(0, len(Ps), batch)
    cls[:4] = [0, 1, 2, 3]
    gs = [rng.standard_normal((3, Ps[c])) for c in cls]
    T = [4 * p for p in Ps]
    plan = mci.Plan(systems, Ps, T, outputs=("f", "hilbert"), precision=prec, max_batch=batch)
    in_len = [3 * Ps[c] for c in cls]
    out_len = [2 * T[c] for c in cls]
    pad = 0 if packed else 8
    in_off = np.cumsum([0] + [n + pad for n in in_len])[:-1]
    out_off = np.cumsum([0] + [n + pad for n in out_len])[:-1]
    flat = np.zeros(in_off[-1] + in_len[-1] + pad)
    for b in range(batch):
        flat[in_off[b]:in_off[b] + in_len[b]] = gs[b].ravel()
    x = torch.tensor(flat, dtype=DT[prec], device="cuda")
    y = torch.full((int(out_off[-1] + out_len[-1] + pad),), float("nan"), dtype=DT[prec], device="cuda")
    sc = torch.tensor(cls, dtype=torch.int32, device="cuda") if where == "device" else \
        np.ascontiguousarray(cls, dtype=np.int32)
    io = None if packed else torch.tensor(in_off, dtype=torch.int64, device="cuda")
    oo = None if packed else torch.tensor(out_off, dtype=torch.int64, device="cuda")
    mci.mci_interp_1d(plan.handle, x, io, y, oo, sc, batch)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    yh = y.cpu().double().numpy()
    for b in range(batch):
        ref = O.mci_direct(systems, gs[b], T[cls[b]], outputs=("f", "hilbert"))
        got = yh[out_off[b]:out_off[b] + out_len[b]].reshape(2, T[cls[b]])
        check(got, ref, prec)
    plan.close()


def test_host_classes_out_of_range(cuda_device):
    plan = mci.Plan([F], [16, 32], [32, 64], max_batch=4)
    x = torch.zeros(200, device="cuda")
    y = torch.zeros(400, device="cuda")
    with pytest.raises(mci.MciError) as ei:
        mci.mci_interp_1d(plan.handle, x, None, y, None, np.array([0, 1, 7, 0], np.int32), 4)
    assert ei.value.status == mci.MCI_ERR_INVALID_ARG
    # repeated host-grouped calls reuse the two pinned staging blocks
    cls = np.array([1, 0, 1, 0], np.int32)
    g = torch.randn(16 + 32 + 16 + 32, device="cuda")
    outs = []
    for _ in range(5):
        o = torch.empty(64 + 32 + 64 + 32, device="cuda")
        mci.mci_interp_1d(plan.handle, g, None, o, None, cls, 4)
        outs.append(o)
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    plan.close()


def test_bad_size_class_sets_status(cuda_device):
    plan = mci.Plan([F], [16, 32], [32, 64], max_batch=4)
    x = torch.zeros(200, device="cuda")
    y = torch.zeros(400, device="cuda")
    sc = torch.tensor([0, 1, 7, -1], dtype=torch.int32, device="cuda")
    mci.mci_interp_1d(plan.handle, x, None, y, None, sc, 4)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] & 1
    assert plan.info()["device_status"] == 0   # cleared by the previous query
    plan.close()


def test_empty_batch_is_noop(cuda_device):
    plan = mci.Plan([F], 16, 32, max_batch=4)
    mci.mci_interp_1d(plan.handle, 0, None, 0, None, None, 0)
    with pytest.raises(mci.MciError):
        mci.mci_interp_1d(plan.handle, 0, None, 0, None, None, 5)   # above max_batch
    plan.close()


@pytest.mark.parametrize("where", ["device", "host"])
def test_upsample_2d_matches_oracle(cuda_device, where):
    """Rows then columns (Section 5.2), FD derivative channel, images of different sizes;
    image sizes in device memory (device-side grouping) or host memory (host-side)."""
    systems = [F, D1]
    shapes = [(16, 16, 2), (32, 16, 4), (12, 24, 3), (16, 32, 2), (16, 16, 3), (32, 32, 2)]
    sizes = sorted({(w, s * w) for h, w, s in shapes} | {(h, s * h) for h, w, s in shapes})
    plan = mci.Plan(systems, [p for p, _ in sizes], [t for _, t in sizes], channels="fd",
                    max_batch=1, max_images=len(shapes),
                    max_intermediate=sum(h * s * w for h, w, s in shapes))
    rng = S.rng_for(2, 3)
    imgs = [rng.random((h, w)) for h, w, s in shapes]
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]), dtype=torch.float32, device="cuda")
    hr_len = [s * s * h * w for h, w, s in shapes]
    hr = torch.full((sum(hr_len),), float("nan"), device="cuda")
    dev = "cuda" if where == "device" else "cpu"
    hh = torch.tensor([h for h, w, s in shapes], dtype=torch.int32, device=dev)
    ww = torch.tensor([w for h, w, s in shapes], dtype=torch.int32, device=dev)
    ss = torch.tensor([s for h, w, s in shapes], dtype=torch.int32, device=dev)
    plan.upsample_2d(lr, hh, ww, ss, hr, len(shapes))
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    out = hr.cpu().double().numpy()
    pos = 0
    for (h, w, s), im in zip(shapes, imgs):
        ref = O.upsample_2d(im.astype(np.float32).astype(np.float64), s, systems)
        got = out[pos:pos + s * s * h * w].reshape(s * h, s * w)
        pos += s * s * h * w
        check(got, ref, "fp32")
    plan.close()


def test_upsample_2d_paper_mode_three_channels(cuda_device):
    """Section 5.2 with M = 3 systems {f, f', f''} formed from the LR samples by centred
    differences, scale 3: a 128 x 128 image and rectangular ones (all on the FFT route: the
    plan keeps M = 3 image classes off the tensor-core route for accuracy)."""
    systems = [F, D1, D2]
    shapes = [(128, 128, 3), (24, 48, 3), (48, 24, 3)]
    sizes = sorted({(w, s * w) for h, w, s in shapes} | {(h, s * h) for h, w, s in shapes})
    plan = mci.Plan(systems, [p for p, _ in sizes], [t for _, t in sizes], channels="fd",
                    max_batch=1, max_images=len(shapes),
                    max_intermediate=sum(h * s * w for h, w, s in shapes))
    rng = S.rng_for(2, 4)
    imgs = [rng.random((h, w)) for h, w, s in shapes]
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]), dtype=torch.float32, device="cuda")
    hr_len = [s * s * h * w for h, w, s in shapes]
    hr = torch.full((sum(hr_len),), float("nan"), device="cuda")
    hh = np.array([h for h, w, s in shapes], np.int32)
    ww = np.array([w for h, w, s in shapes], np.int32)
    ss = np.array([s for h, w, s in shapes], np.int32)
    plan.upsample_2d(lr, hh, ww, ss, hr, len(shapes))
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    out = hr.cpu().double().numpy()
    pos = 0
    for (h, w, s), im in zip(shapes, imgs):
        ref = O.upsample_2d(im.astype(np.float32).astype(np.float64), s, systems)
        got = out[pos:pos + s * s * h * w].reshape(s * h, s * w)
        check(got, ref, "fp32")
        pos += s * s * h * w
    plan.close()


_LARGE_2D = [(1024, 2), (768, 3), (512, 2), (384, 4)]   # (LR side, scale): N = 512, 384, 256, 192


def _large_2d_images():
    rng = S.rng_for(2, 9)
    return [S.synthetic_image(rng, L).astype(np.float32) for L, _ in _LARGE_2D]


def _oracle_columns(img, s, systems, cols):
    """Rows then columns (Section 5.2) restricted to the HR columns `cols`: the row pass is
    evaluated only at those positions of every row (they are all the column pass reads),
    then every selected column is interpolated in full."""
    h, w = img.shape
    x = img.astype(np.float64)
    inter = O.mci_direct(systems, O.fd_channels(x, systems), s * w, idx=cols)[:, 0, :]   # h x |cols|
    return O.mci_direct(systems, O.fd_channels(inter.T, systems), s * h)[:, 0, :].T       # sh x |cols|


@pytest.mark.parametrize("where", ["host", "device"])
def test_upsample_2d_large_images_match_oracle(cuda_device, where):
    """The uneven image workload's largest classes (LR 1024^2 x2, 768^2 x3, 512^2 x2, 384^2 x4,
    M = 2 {f, FD f'}) in one call; the oracle evaluates a set of HR columns (first, last,
    tile edges, random), each over its whole length."""
    systems = [F, D1]
    imgs = _large_2d_images()
    PT = sorted({(L, s * L) for L, s in _LARGE_2D})
    plan = mci.Plan(systems, [p for p, _ in PT], [t for _, t in PT], channels="fd", max_batch=1,
                    max_images=len(imgs), max_intermediate=sum(L * s * L for L, s in _LARGE_2D))
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]), device="cuda")
    n_hr = sum(s * s * L * L for L, s in _LARGE_2D)
    hr = torch.full((n_hr,), float("nan"), device="cuda")
    dev = "cuda" if where == "device" else "cpu"
    hh = torch.tensor([L for L, _ in _LARGE_2D], dtype=torch.int32, device=dev)
    ss = torch.tensor([s for _, s in _LARGE_2D], dtype=torch.int32, device=dev)
    plan.upsample_2d(lr, hh, hh, ss, hr, len(imgs))
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    out = hr.cpu().double().numpy()
    assert np.all(np.isfinite(out))
    pos = 0
    rng = S.rng_for(2, 10)
    for (L, s), im in zip(_LARGE_2D, imgs):
        W = s * L
        cols = np.unique(np.r_[0, 1, 2, 31, 32, 33, W // 2, W - 3, W - 2, W - 1,
                               rng.integers(0, W, 4)])
        got = out[pos:pos + W * W].reshape(W, W)[:, cols]
        pos += W * W
        check(got, _oracle_columns(im, s, systems, cols), "fp32")
    plan.close()


@pytest.mark.parametrize("P", [256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("aligned", [True, False])
def test_fused_radix8_classes(cuda_device, P, aligned):
    """The batched workload's classes (M = 3 {f, Hf, f'}, T = 4P, f only, FP32) run on the
    fused radix-8 kernel (2048 / (P/2) signals per CTA); a ragged last tile, half trig
    polynomials and half smooth non-bandlimited signals.  Unaligned offsets take the
    element-wise load and store branches."""
    systems = [F, H, D1]
    N = P // 2
    G = 2048 // N
    batch = 2 * G + 3
    rng = S.rng_for(1, 40 + P)
    g = np.concatenate([S.signal_batch_1d(rng, P, batch // 2, systems, "trig")[0],
                        S.signal_batch_1d(rng, P, batch - batch // 2, systems, "smooth")[0]])
    plan = mci.Plan(systems, P, 4 * P, max_batch=batch)
    assert plan.info()["signals_per_cta"][0] == G
    pad = 0 if aligned else 1
    in_off = np.arange(batch, dtype=np.int64) * (3 * P + pad) + pad
    out_off = np.arange(batch, dtype=np.int64) * (4 * P + pad) + pad
    flat = np.zeros(int(in_off[-1]) + 3 * P + pad)
    for b in range(batch):
        flat[in_off[b]:in_off[b] + 3 * P] = g[b].ravel()
    x = torch.tensor(flat, dtype=torch.float32, device="cuda")
    y = torch.full((int(out_off[-1]) + 4 * P + pad,), float("nan"), device="cuda")
    mci.mci_interp_1d(plan.handle, x, torch.tensor(in_off, device="cuda"), y,
                      torch.tensor(out_off, device="cuda"), None, batch)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    plan.close()
    yh = y.cpu().double().numpy()
    xs = x.cpu().double().numpy()
    sel = np.unique(np.r_[0, 1, G - 1, G, batch // 2, batch - 2, batch - 1])
    gs = np.stack([xs[in_off[b]:in_off[b] + 3 * P].reshape(3, P) for b in sel])
    ref = O.mci_direct(systems, gs, 4 * P)
    got = np.stack([yh[out_off[b]:out_off[b] + 4 * P] for b in sel])[:, None, :]
    check(got, ref, "fp32")
    if not aligned:   # the padding elements between signals stay untouched
        gaps = np.concatenate([yh[out_off[b] - 1:out_off[b]] for b in range(batch)])
        assert np.all(np.isnan(gaps))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("systems,P,s,batch", [([F, D1], 64, 64, 1), ([F, H, D1], 32, 32, 3),
                                               ([F], 128, 16, 2), ([F, D2], 48, 24, 1)],
                         ids=lambda v: str(v))
def test_few_signals_many_phases(cuda_device, prec, systems, P, s, batch):
    """A few short signals on a long output grid: the s n_out phases of each tile are spread
    over several CTAs; f, Hf and f' against the oracle."""
    outs = ("f", "hilbert", "deriv")
    g = S.rng_for(1, 50 + P + s).standard_normal((batch, len(systems), P))
    out = run_1d(g, systems, s * P, prec, outputs=outs)
    check(out, O.mci_direct(systems, g, s * P, outputs=outs), prec)


# (h, w, s): row class (w, s w) and column class (h, s h).  Power-of-two sides 256 .. 1024 run
# on the fused kernels (rows and columns); 12 and 200-ish sides on the generic ones.  The last
# image's 36 columns leave a ragged tile of the 16-column tiles of the (256, 768) class.
_FUSED_2D = [(512, 512, 3), (1024, 256, 4), (256, 1024, 3), (512, 256, 2), (256, 12, 3)]


@pytest.mark.parametrize("where", ["host", "device"])
def test_upsample_2d_fused_classes_match_oracle(cuda_device, where):
    systems = [F, D1]
    rng = S.rng_for(2, 11)
    # the generator's blobs and edges need sides of 64 or more: the narrow image is uniform noise
    imgs = [(S.synthetic_image(rng, h, w) if min(h, w) >= 64 else rng.random((h, w))).astype(np.float32)
            for h, w, _ in _FUSED_2D]
    PT = sorted({(w, s * w) for h, w, s in _FUSED_2D} | {(h, s * h) for h, w, s in _FUSED_2D})
    plan = mci.Plan(systems, [p for p, _ in PT], [t for _, t in PT], channels="fd", max_batch=1,
                    max_images=len(imgs), max_intermediate=sum(h * s * w for h, w, s in _FUSED_2D))
    mask = plan.info()["fused_mask"]
    for k, (p_, t_) in enumerate(PT):
        assert bool(mask & (1 << k)) == (p_ in (256, 512, 1024)), (p_, t_)
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]), device="cuda")
    n_hr = sum(s * s * h * w for h, w, s in _FUSED_2D)
    hr = torch.full((n_hr,), float("nan"), device="cuda")
    dev = "cuda" if where == "device" else "cpu"
    hh = torch.tensor([h for h, _, _ in _FUSED_2D], dtype=torch.int32, device=dev)
    ww = torch.tensor([w for _, w, _ in _FUSED_2D], dtype=torch.int32, device=dev)
    ss = torch.tensor([s for _, _, s in _FUSED_2D], dtype=torch.int32, device=dev)
    plan.upsample_2d(lr, hh, ww, ss, hr, len(imgs))
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    out = hr.cpu().double().numpy()
    assert np.all(np.isfinite(out))
    pos = 0
    crng = S.rng_for(2, 12)
    for (h, w, s), im in zip(_FUSED_2D, imgs):
        Wd = s * w
        cols = np.unique(np.r_[0, 1, 15, 16, 17, Wd // 2, Wd - 3, Wd - 2, Wd - 1, crng.integers(0, Wd, 3)])
        cols = cols[cols < Wd]
        got = out[pos:pos + s * h * Wd].reshape(s * h, Wd)[:, cols]
        pos += s * h * Wd
        check(got, _oracle_columns(im, s, systems, cols), "fp32")
    plan.close()


# images 768 and 384 high: columns of P = 6 N' (N' = 128: tiles of 16 columns; N' = 64: tiles
# of 32, two columns per half warp) on the fused factor-3 column kernel, s = 2, 3, 4; widths
# give full tiles and ragged last tiles (s w = 36, 72)
_FACTOR3_2D = [(768, 64, 2), (768, 48, 3), (768, 96, 4), (768, 12, 3),
               (384, 64, 2), (384, 24, 3), (384, 48, 4)]


@pytest.mark.parametrize("where", ["host", "device"])
def test_upsample_2d_factor3_columns_match_oracle(cuda_device, where):
    systems = [F, D1]
    rng = S.rng_for(2, 13)
    imgs = [(S.synthetic_image(rng, h, w) if min(h, w) >= 64 else rng.random((h, w))).astype(np.float32)
            for h, w, _ in _FACTOR3_2D]
    PT = sorted({(w, s * w) for h, w, s in _FACTOR3_2D} | {(h, s * h) for h, w, s in _FACTOR3_2D})
    plan = mci.Plan(systems, [p for p, _ in PT], [t for _, t in PT], channels="fd", max_batch=1,
                    max_images=len(imgs), max_intermediate=sum(h * s * w for h, w, s in _FACTOR3_2D))
    mask3 = plan.info()["fused3_mask"]
    for k, (p_, t_) in enumerate(PT):
        assert bool(mask3 & (1 << k)) == (p_ in (384, 768)), (p_, t_)
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]), device="cuda")
    n_hr = sum(s * s * h * w for h, w, s in _FACTOR3_2D)
    hr = torch.full((n_hr,), float("nan"), device="cuda")
    dev = "cuda" if where == "device" else "cpu"
    hh = torch.tensor([h for h, _, _ in _FACTOR3_2D], dtype=torch.int32, device=dev)
    ww = torch.tensor([w for _, w, _ in _FACTOR3_2D], dtype=torch.int32, device=dev)
    ss = torch.tensor([s for _, _, s in _FACTOR3_2D], dtype=torch.int32, device=dev)
    plan.upsample_2d(lr, hh, ww, ss, hr, len(imgs))
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    out = hr.cpu().double().numpy()
    assert np.all(np.isfinite(out))
    pos = 0
    crng = S.rng_for(2, 14)
    for (h, w, s), im in zip(_FACTOR3_2D, imgs):
        Wd = s * w
        cols = np.unique(np.r_[0, 1, 15, 16, 17, Wd // 2, Wd - 3, Wd - 2, Wd - 1, crng.integers(0, Wd, 3)])
        cols = cols[cols < Wd]
        got = out[pos:pos + s * h * Wd].reshape(s * h, Wd)[:, cols]
        pos += s * h * Wd
        check(got, _oracle_columns(im, s, systems, cols), "fp32")
    plan.close()
