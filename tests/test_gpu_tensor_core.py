"""The tensor-core image path: for size classes with P = 128 and T <= 512 (where it beats
the FFT route) the row and column passes run as tcgen05 GEMMs with split-BF16 operands (six products,
FP32 accumulation).  Checked against the FP64 oracle (Section 5.2 separable
interpolation) and against the FFT path on the same images."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci
from paper_1802_10291_gb300 import synth as S

pytestmark = pytest.mark.gpu

SYS = [("identity",), ("deriv", 1)]


def run(shapes, imgs, where):
    sizes = sorted({(w, s * w) for h, w, s in shapes} | {(h, s * h) for h, w, s in shapes})
    plan = mci.Plan(SYS, [p for p, _ in sizes], [t for _, t in sizes], channels="fd",
                    max_batch=1, max_images=len(shapes),
                    max_intermediate=sum(h * s * w for h, w, s in shapes))
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]), dtype=torch.float32, device="cuda")
    hr = torch.full((sum(s * s * h * w for h, w, s in shapes),), float("nan"), device="cuda")
    dev = "cuda" if where == "device" else "cpu"
    hh = torch.tensor([h for h, w, s in shapes], dtype=torch.int32, device=dev)
    ww = torch.tensor([w for h, w, s in shapes], dtype=torch.int32, device=dev)
    ss = torch.tensor([s for h, w, s in shapes], dtype=torch.int32, device=dev)
    plan.upsample_2d(lr, hh, ww, ss, hr, len(shapes))
    torch.cuda.synchronize()
    st = plan.info()["device_status"]
    plan.close()
    assert st == 0, st
    out, pos = [], 0
    for h, w, s in shapes:
        out.append(hr[pos:pos + s * s * h * w].view(s * h, s * w).cpu().double().numpy())
        pos += s * s * h * w
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(b ** 2)))


def test_gemm_single_image_vs_oracle(cuda_device):
    shapes = [(128, 128, 2)]
    imgs = [S.synthetic_image(S.rng_for(4, 1), 128).astype(np.float32)]
    got = run(shapes, imgs, "host")[0]
    ref = O.upsample_2d(imgs[0].astype(np.float64), 2, SYS)
    assert rel(got, ref) <= 1e-5


def test_gemm_mixed_batch(cuda_device):
    shapes = [(128, 128, 2), (128, 128, 4), (256, 256, 2), (128, 256, 3), (64, 64, 4), (256, 128, 2)]
    rng = S.rng_for(4, 2)
    imgs = [S.synthetic_image(rng, h, w).astype(np.float32) for h, w, s in shapes]
    by_gemm = run(shapes, imgs, "host")
    by_fft = run(shapes, imgs, "device")
    for g, f in zip(by_gemm, by_fft):
        assert rel(g, f) <= 1e-5
    for k in (1, 3):
        h, w, s = shapes[k]
        ref = O.upsample_2d(imgs[k].astype(np.float64), s, SYS)
        assert rel(by_gemm[k], ref) <= 1e-5
