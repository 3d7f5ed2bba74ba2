"""Residual corrector on the GPU through the C ABI: forward and gradients against the
FP64 CPU oracle (same BF16-rounded weights), the image generator against its formula,
checkpoint/resume, and a short training run that must beat plain MCI."""
import os

import numpy as np
import pytest

from oracle import corrector as oc
from paper_1802_10291_gb300 import synth

pytestmark = pytest.mark.gpu


def _params(seed, last_scale=0.3):
    from paper_1802_10291_gb300 import corrector
    p = corrector.init_params(seed, zero_last=False).astype(np.float64)
    n_last = 32 * 9 + 1
    p[-n_last:] *= last_scale
    rng = np.random.default_rng(seed)
    # non-zero biases so that the bias path is exercised
    k = 0
    for ci, co in oc.LAYERS:
        k += co * ci * 9
        p[k:k + co] = rng.uniform(-0.05, 0.05, co)
        k += co
    return p.astype(np.float32)


def _oracle_params(p32):
    """The values the GPU computes with: BF16 weights, FP32 biases."""
    p = np.asarray(p32, np.float64).copy()
    k = 0
    for ci, co in oc.LAYERS:
        n = co * ci * 9
        p[k:k + n] = oc.bf16_round(p32[k:k + n])
        k += n + co
    return p


# (1, 12, 96) and (2, 9, 100): rows of 16-byte-aligned tiles inside the image (vector loads)
# next to tiles at the right edge (wrapped columns)
@pytest.mark.parametrize("shape", [(2, 20, 24), (1, 33, 17), (3, 16, 16), (1, 37, 70), (1, 12, 96),
                                   (2, 9, 100)])
def test_forward_and_gradient_parity(cuda_device, shape):
    import torch
    from paper_1802_10291_gb300 import corrector
    b, h, w = shape
    rng = np.random.default_rng(11 + h)
    x = rng.random(shape).astype(np.float32)
    hr = np.clip(x + 0.1 * rng.standard_normal(shape), 0, 1).astype(np.float32)
    p32 = _params(3)
    net = corrector.Corrector(b * h * w, p32)
    xd = torch.tensor(x, device="cuda")
    hd = torch.tensor(hr, device="cuda")
    out = torch.empty_like(xd)
    net.forward(xd, out, b, h, w)
    g = torch.empty(net.n, device="cuda")
    L = torch.empty(1, device="cuda")
    net.loss_grad(xd, hd, b, h, w, grad=g, loss=L)
    torch.cuda.synchronize()
    assert net.status() == 0
    po = _oracle_params(p32)
    pred, _ = oc.forward(po, x.astype(np.float64))
    Lo, go = oc.loss_grad(po, x.astype(np.float64), hr.astype(np.float64))
    # FP32 accumulation over <= 288 products per output of O(1) values
    assert np.max(np.abs(out.cpu().numpy() - pred)) <= 1e-4 * max(1.0, np.abs(pred).max())
    assert abs(float(L.item()) - Lo) <= 1e-4 * Lo
    gd = g.cpu().numpy().astype(np.float64)
    scale = np.abs(go).max()
    assert np.max(np.abs(gd - go)) <= 2e-3 * scale, np.max(np.abs(gd - go)) / scale
    # relative agreement per layer (gradients differ in magnitude across layers)
    k = 0
    for ci, co in oc.LAYERS:
        n = co * ci * 9 + co
        a, r = gd[k:k + n], go[k:k + n]
        assert np.linalg.norm(a - r) <= 1e-3 * np.linalg.norm(r) + 1e-12, (ci, co)
        k += n
    net.close()


def test_zero_last_layer_is_plain_mci(cuda_device):
    import torch
    from paper_1802_10291_gb300 import corrector
    x = torch.rand((2, 40, 48), device="cuda")
    net = corrector.Corrector(x.numel(), corrector.init_params(0))
    out = torch.empty_like(x)
    net.forward(x, out, 2, 40, 48)
    torch.cuda.synchronize()
    assert torch.equal(out, x)
    net.close()


def _image_formula(q, H, W):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    v = np.full((H, W), 0.5)
    for k in range(20):
        cy, cx, ism, isn, ang, amp = q[6 * k:6 * k + 6].astype(np.float64)
        dy, dx = y - cy, x - cx
        u = (dx * np.cos(ang) + dy * np.sin(ang)) * ism
        w = (-dx * np.sin(ang) + dy * np.cos(ang)) * isn
        v += amp * np.exp(-0.5 * (u * u + w * w))
    edge_margin = np.full((H, W), np.inf)
    for k in range(10):
        py, px, ang, step = q[120 + 4 * k:124 + 4 * k].astype(np.float64)
        d = (x - px) * np.sin(ang) - (y - py) * np.cos(ang)
        v += np.where(d > 0, step, 0.0)
        edge_margin = np.minimum(edge_margin, np.abs(d))
    for k in range(8):
        fy, fx, ph, amp = q[160 + 4 * k:164 + 4 * k].astype(np.float64)
        v += amp * np.cos(2 * np.pi * (fy * y / H + fx * x / W) + ph)
    return np.clip(v, 0, 1), edge_margin


def test_image_generator_and_decimation(cuda_device):
    import torch
    from paper_1802_10291_gb300 import corrector
    H, W, n = 96, 64, 3
    prm = synth.image_params(synth.rng_for(5, 99), n, 96)
    img = torch.empty((n, H, W), device="cuda")
    corrector.generate_images(torch.tensor(prm, device="cuda"), img, n, H, W)
    lr = torch.empty((n, H // 4, W // 4), device="cuda")
    corrector.decimate(img, lr, n, H, W, 4)
    torch.cuda.synchronize()
    got = img.cpu().numpy()
    for i in range(n):
        ref, margin = _image_formula(prm[i], H, W)
        ok = margin > 1e-3                        # pixels on an edge may round either way
        assert ok.mean() > 0.99
        assert np.max(np.abs(got[i] - ref)[ok]) < 1e-4
    np.testing.assert_array_equal(lr.cpu().numpy(), got[:, ::4, ::4])


def test_checkpoint_resume_is_exact(cuda_device, tmp_path):
    import torch
    from paper_1802_10291_gb300 import corrector
    src = corrector.PairSource(4, 64, s=4, seed=1)
    x, hr = src.next()
    netA = corrector.Corrector(x.numel(), corrector.init_params(1))
    L = torch.empty(1, device="cuda")
    for _ in range(3):
        netA.train_step(x, hr, 4, 64, 64, 1e-3, loss=L)
    netA.save(str(tmp_path / "ck.npz"))
    netA.train_step(x, hr, 4, 64, 64, 1e-3, loss=L)
    netA.train_step(x, hr, 4, 64, 64, 1e-3, loss=L)
    torch.cuda.synchronize()
    a = float(L.item())
    stA, stepA = netA.get_state()
    netB = corrector.Corrector(x.numel())
    netB.load(str(tmp_path / "ck.npz"))
    netB.train_step(x, hr, 4, 64, 64, 1e-3, loss=L)
    netB.train_step(x, hr, 4, 64, 64, 1e-3, loss=L)
    torch.cuda.synchronize()
    stB, stepB = netB.get_state()
    assert stepA == stepB == 5
    # per-CTA atomics make the weight gradients order-dependent in the last bits
    assert abs(float(L.item()) - a) <= 1e-5 * a
    assert np.max(np.abs(stA[:netA.n] - stB[:netB.n])) < 1e-4
    netA.close()
    netB.close()


def test_training_beats_plain_mci(cuda_device):
    import torch
    from paper_1802_10291_gb300 import corrector
    n, size = 8, 128
    src = corrector.PairSource(n, size, s=4, seed=2)
    held = corrector.PairSource(n, size, s=4, seed=3)
    xv, hv = held.next()
    xv, hv = xv.clone(), hv.clone()
    net = corrector.Corrector(n * size * size, corrector.init_params(2))
    for it in range(150):
        x, hr = src.next() if it % 5 == 0 else (x, hr)
        net.train_step(x, hr, n, size, size, 1e-3)
    out = torch.empty_like(xv)
    net.forward(xv, out, n, size, size)
    torch.cuda.synchronize()
    base = corrector.psnr(xv, hv)
    got = corrector.psnr(out, hv)
    assert got > base + 0.3, (base, got)
    net.close()
