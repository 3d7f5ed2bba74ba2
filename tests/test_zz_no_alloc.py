"""mci_interp_1d_noalloc: the entry point for callers that cannot allocate device
memory when they know their batch (global-mode stream capture refuses cudaMalloc;
some frameworks hand out all device memory up front).  Its scratch lives in a
static device array inside the library.  Checked against mci_interp_1d through
the C ABI on two calls in a row (the second call reuses the array the first
left behind)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci
from paper_1802_10291_gb300 import synth as S

pytestmark = pytest.mark.gpu

SYSTEMS = [("identity",), ("hilbert",), ("deriv", 1)]


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(b ** 2)))


@pytest.mark.parametrize("packed", [True, False])
def test_noalloc_matches_interp_1d(cuda_device, mci_lib, packed):
    Ps = [64, 256, 128]
    T = [4 * p for p in Ps]
    rng = S.rng_for(5, 1 if packed else 2)
    batch = 37
    cls = rng.integers(0, 3, batch).astype(np.int32)
    in_len = np.array([3 * Ps[c] for c in cls])
    out_len = np.array([T[c] for c in cls])
    in_off = np.concatenate([[0], np.cumsum(in_len)[:-1]]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(out_len)[:-1]]).astype(np.int64)
    x = torch.tensor(rng.standard_normal(int(in_len.sum())), dtype=torch.float32, device="cuda")
    sc = torch.tensor(cls, device="cuda")
    io = None if packed else torch.tensor(in_off, device="cuda")
    oo = None if packed else torch.tensor(out_off, device="cuda")
    plan = mci.Plan(SYSTEMS, Ps, T, max_batch=batch)
    ref = torch.full((int(out_len.sum()),), float("nan"), device="cuda")
    mci.mci_interp_1d(plan.handle, x, io, ref, oo, sc, batch)
    outs = []
    for _ in range(2):
        y = torch.full_like(ref, float("nan"))
        mci.mci_interp_1d_noalloc(plan.handle, x, io, y, oo, sc, batch)
        outs.append(y)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    r = ref.cpu().double().numpy()
    for y in outs:
        assert rel_err(y.cpu().double().numpy(), r) <= 1e-5
    plan.close()


def test_noalloc_uniform_and_limits(cuda_device, mci_lib):
    plan = mci.Plan(SYSTEMS, 512, 2048, precision="fp64", max_batch=1)
    g = torch.tensor(S.rng_for(5, 3).standard_normal((9, 3, 512)), device="cuda")
    ref = torch.empty((9, 1, 2048), dtype=torch.float64, device="cuda")
    # the plan holds workspace for one signal; the no-allocation entry point takes nine
    for b in range(9):
        mci.mci_interp_1d(plan.handle, g[b], None, ref[b], None, None, 1)
    for _ in range(2):
        y = torch.full_like(ref, float("nan"))
        mci.mci_interp_1d_noalloc(plan.handle, g, None, y, None, None, 9)
        torch.cuda.synchronize()
        assert float((y - ref).abs().max()) <= 1e-12
    with pytest.raises(mci.MciError) as ei:
        mci.mci_interp_1d_noalloc(plan.handle, g, None, y, None, None,
                                  mci.MCI_NOALLOC_MAX_BATCH + 1)
    assert ei.value.status == mci.MCI_ERR_UNSUPPORTED_SIZE
    plan.close()


def test_noalloc_uneven_plan_for_one_signal(cuda_device, mci_lib):
    """The intended use: a plan made at start-up for one signal (max_batch = 1), then an
    uneven batch of thousands of signals of three size classes through the no-allocation
    entry point.  Checked against mci_interp_1d on a plan sized for the whole batch, and
    one signal of every class against the oracle."""
    Ps = [128, 512, 256]
    T = [4 * p for p in Ps]
    rng = S.rng_for(5, 4)
    batch = 3000
    cls = rng.integers(0, 3, batch).astype(np.int32)
    cls[:3] = [0, 1, 2]
    in_len = np.array([3 * Ps[c] for c in cls])
    out_len = np.array([T[c] for c in cls])
    out_off = np.concatenate([[0], np.cumsum(out_len)[:-1]]).astype(np.int64)
    in_off = np.concatenate([[0], np.cumsum(in_len)[:-1]]).astype(np.int64)
    xh = rng.standard_normal(int(in_len.sum()))
    x = torch.tensor(xh, dtype=torch.float32, device="cuda")
    sc = torch.tensor(cls, device="cuda")
    big = mci.Plan(SYSTEMS, Ps, T, max_batch=batch)
    ref = torch.full((int(out_len.sum()),), float("nan"), device="cuda")
    mci.mci_interp_1d(big.handle, x, None, ref, None, sc, batch)
    small = mci.Plan(SYSTEMS, Ps, T, max_batch=1)
    outs = []
    for _ in range(2):
        y = torch.full_like(ref, float("nan"))
        mci.mci_interp_1d_noalloc(small.handle, x, None, y, None, sc, batch)
        outs.append(y)
    torch.cuda.synchronize()
    assert big.info()["device_status"] == 0
    assert small.info()["device_status"] == 0
    r = ref.cpu().double().numpy()
    for y in outs:
        assert rel_err(y.cpu().double().numpy(), r) <= 1e-5
    got = outs[1].cpu().double().numpy()
    xr = x.cpu().double().numpy()       # the FP32 samples the GPU saw
    for c in range(3):
        b = int(np.flatnonzero(cls == c)[-1])
        g = xr[in_off[b]:in_off[b] + in_len[b]].reshape(3, Ps[c])
        want = O.mci_direct(SYSTEMS, g, T[c])[0]
        assert rel_err(got[out_off[b]:out_off[b] + out_len[b]], want) <= 1e-5
    big.close()
    small.close()


def test_noalloc_refuses_host_size_classes(cuda_device, mci_lib):
    """The grouping runs on the device, so size classes in host memory are refused with
    MCI_ERR_INVALID_ARG (mci_interp_1d groups such batches on the host instead)."""
    plan = mci.Plan(SYSTEMS, [64, 128], [256, 512], max_batch=1)
    x = torch.zeros(3 * (64 + 128), device="cuda")
    y = torch.zeros(256 + 512, device="cuda")
    with pytest.raises(mci.MciError) as ei:
        mci.mci_interp_1d_noalloc(plan.handle, x, None, y, None, np.array([0, 1], np.int32), 2)
    assert ei.value.status == mci.MCI_ERR_INVALID_ARG
    with pytest.raises(mci.MciError) as ei:
        mci.mci_interp_1d_noalloc(plan.handle, x, None, y, None, None, 2)
    assert ei.value.status == mci.MCI_ERR_INVALID_ARG
    plan.close()
