"""Mirror image boundaries on the GPU (mci_upsample_2d_mirror through the C ABI) against the
oracle's upsample_2d_mirror, element by element; the half-sample cosines that the mirror
mode reproduces exactly come back to FP32 accuracy; the scratch and size errors.

Tolerance as in the parity tests: FP32 max-abs <= 1e-5 x RMS of the oracle output."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci
from paper_1802_10291_gb300 import synth as S

pytestmark = pytest.mark.gpu

F, D1 = ("identity",), ("deriv", 1)
TOL = 1e-5

# (h, w, s): the extensions are 96 x 128, 128 x 64, 192 x 96 and 24 x 32 (a small image whose
# column tiles are ragged)
_IMGS = [(48, 64, 2), (64, 32, 3), (96, 48, 4), (12, 16, 3)]


def _plan(systems, dims):
    PT = sorted({(2 * w, 2 * s * w) for h, w, s in dims} | {(2 * h, 2 * s * h) for h, w, s in dims})
    return mci.Plan(systems, [p for p, _ in PT], [t for _, t in PT], channels="fd", max_batch=1,
                    max_images=len(dims), max_intermediate=sum(4 * s * h * w for h, w, s in dims))


def _run(plan, imgs, dims):
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]).astype(np.float32), device="cuda")
    hr = torch.full((sum(s * s * h * w for h, w, s in dims),), float("nan"), device="cuda")
    ext_lr = torch.empty(sum(4 * h * w for h, w, _ in dims), device="cuda")
    ext_hr = torch.empty(sum(4 * s * s * h * w for h, w, s in dims), device="cuda")
    hh = np.array([h for h, _, _ in dims], np.int32)
    ww = np.array([w for _, w, _ in dims], np.int32)
    ss = np.array([s for _, _, s in dims], np.int32)
    mci.mci_upsample_2d_mirror(plan.handle, lr, hh, ww, ss, hr, len(dims), ext_lr, ext_hr)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    out, pos = [], 0
    for h, w, s in dims:
        out.append(hr[pos:pos + s * s * h * w].cpu().double().numpy().reshape(s * h, s * w))
        pos += s * s * h * w
    return out


def test_mirror_matches_oracle(cuda_device):
    systems = [F, D1]
    rng = S.rng_for(2, 21)
    imgs = [(S.synthetic_image(rng, h, w) if min(h, w) >= 64 else rng.random((h, w))) for h, w, _ in _IMGS]
    plan = _plan(systems, _IMGS)
    for _ in range(2):   # two calls in a row: the scratch and workspace carry nothing over
        got = _run(plan, imgs, _IMGS)
        for (h, w, s), im, g in zip(_IMGS, imgs, got):
            ref = O.upsample_2d_mirror(np.asarray(im, np.float32).astype(np.float64), s, systems)
            assert np.all(np.isfinite(g))
            err = np.max(np.abs(g - ref)) / np.sqrt(np.mean(ref ** 2))
            assert err <= TOL, (h, w, s, err)
    plan.close()


def test_mirror_reproduces_half_sample_cosines(cuda_device):
    """With the channel {f} the mirror mode reproduces cos(pi k (n + 1/2) / P) products at every
    output pixel (the oracle's pin), here to FP32 accuracy."""
    dims = [(32, 48, 2), (64, 32, 3)]
    imgs, exact = [], []
    for (h, w, s), (k1, k2) in zip(dims, [(3, 5), (7, 2)]):
        n1, n2 = np.arange(h)[:, None], np.arange(w)[None, :]
        imgs.append(np.cos(np.pi * k1 * (n1 + 0.5) / h) * np.cos(np.pi * k2 * (n2 + 0.5) / w))
        m1, m2 = np.arange(s * h)[:, None] / s, np.arange(s * w)[None, :] / s
        exact.append(np.cos(np.pi * k1 * (m1 + 0.5) / h) * np.cos(np.pi * k2 * (m2 + 0.5) / w))
    plan = _plan([F], dims)
    for g, e in zip(_run(plan, imgs, dims), exact):
        assert np.max(np.abs(g - e)) < 2e-5
    plan.close()


def test_mirror_rejects_bad_arguments(cuda_device):
    dims = [(16, 16, 2)]
    plan = _plan([F, D1], dims)
    lr = torch.zeros(256, device="cuda")
    hr = torch.zeros(1024, device="cuda")
    ext = torch.zeros(4096, device="cuda")
    one = np.ones(1, np.int32)
    with pytest.raises(mci.MciError) as e:   # the plan holds no class for an extension of 2 x 8
        mci.mci_upsample_2d_mirror(plan.handle, lr, one * 8, one * 8, one * 2, hr, 1, ext, ext)
    assert e.value.status == mci.MCI_ERR_UNSUPPORTED_SIZE
    with pytest.raises(mci.MciError) as e:   # more than 256 images
        many = np.full(257, 16, np.int32)
        mci.mci_upsample_2d_mirror(plan.handle, lr, many, many, many, hr, 257, ext, ext)
    assert e.value.status == mci.MCI_ERR_UNSUPPORTED_SIZE
    with pytest.raises(mci.MciError) as e:   # no scratch
        mci.mci_upsample_2d_mirror(plan.handle, lr, one * 16, one * 16, one * 2, hr, 1, None, ext)
    assert e.value.status == mci.MCI_ERR_INVALID_ARG
    with pytest.raises(mci.MciError) as e:   # scratch in host memory: refused before any kernel
        host_ext = torch.zeros(4096)
        mci.mci_upsample_2d_mirror(plan.handle, lr, one * 16, one * 16, one * 2, hr, 1, host_ext, ext)
    assert e.value.status == mci.MCI_ERR_INVALID_ARG
    plan.close()
