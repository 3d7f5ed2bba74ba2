"""The persistent launch of uneven batches whose size classes are all on the fused radix-8
kernel (M = 3 {f, Hf, f'}, T = 4P, f only; P in 256 .. 4096): size classes in host memory
(grouped on the host), in device memory (grouped on the device), through the no-allocation
entry point, and replayed from a CUDA graph, each against the oracle on every class and
against each other."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci
from paper_1802_10291_gb300 import synth as S

pytestmark = pytest.mark.gpu

SYSTEMS = [("identity",), ("hilbert",), ("deriv", 1)]
PS = [256, 512, 1024, 2048, 4096]


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(b ** 2)))


def _batch(seed, batch, packed):
    rng = S.rng_for(7, seed)
    cls = rng.integers(0, len(PS), batch).astype(np.int32)
    cls[:len(PS)] = np.arange(len(PS))
    in_len = np.array([3 * PS[c] for c in cls])
    out_len = np.array([4 * PS[c] for c in cls])
    pad = 0 if packed else 4
    in_off = np.concatenate([[0], np.cumsum(in_len + pad)[:-1]]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(out_len + pad)[:-1]]).astype(np.int64)
    x = torch.tensor(rng.standard_normal(int(in_off[-1] + in_len[-1] + pad)), dtype=torch.float32,
                     device="cuda")
    n_out = int(out_off[-1] + out_len[-1] + pad)
    return cls, in_off, out_off, in_len, out_len, x, n_out


def _oracle_check(cls, in_off, out_off, x, y):
    xs, ys = x.cpu().double().numpy(), y.cpu().double().numpy()
    for c, P in enumerate(PS):
        for b in np.flatnonzero(cls == c)[[0, -1]]:
            g = xs[in_off[b]:in_off[b] + 3 * P].reshape(3, P)
            want = O.mci_direct(SYSTEMS, g, 4 * P)[0]
            assert rel(ys[out_off[b]:out_off[b] + 4 * P], want) <= 1e-5, (P, b)


@pytest.mark.parametrize("packed", [True, False])
def test_persistent_host_device_noalloc_graph(cuda_device, packed):
    batch = 300
    cls, in_off, out_off, in_len, out_len, x, n_out = _batch(1 if packed else 2, batch, packed)
    plan = mci.Plan(SYSTEMS, PS, [4 * p for p in PS], max_batch=batch)
    info = plan.info()
    assert info["fused_mask"] == (1 << len(PS)) - 1 and info["persistent_ctas"] > 0
    io = None if packed else torch.tensor(in_off, device="cuda")
    oo = None if packed else torch.tensor(out_off, device="cuda")
    outs = {}
    for where in ("host", "device", "noalloc", "graph"):
        y = torch.full((n_out,), float("nan"), device="cuda")
        sc = cls if where == "host" else torch.tensor(cls, device="cuda")
        if where == "host":
            mci.mci_interp_1d(plan.handle, x, io, y, oo, sc, batch)
        elif where == "device":
            mci.mci_interp_1d(plan.handle, x, io, y, oo, sc, batch)
        elif where == "noalloc":
            mci.mci_interp_1d_noalloc(plan.handle, x, io, y, oo, sc, batch)
        else:
            mci.mci_interp_1d_noalloc(plan.handle, x, io, y, oo, sc, batch)   # first call: set-up
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                mci.mci_interp_1d_noalloc(plan.handle, x, io, y, oo, sc, batch)
            y.fill_(float("nan"))
            for _ in range(2):
                graph.replay()
        torch.cuda.synchronize()
        assert plan.info()["device_status"] == 0
        outs[where] = y
    _oracle_check(cls, in_off, out_off, x, outs["host"])
    for where in ("device", "noalloc", "graph"):
        torch.testing.assert_close(outs[where], outs["host"], rtol=0, atol=0, equal_nan=True)
    if not packed:   # the padding between signals is untouched
        yh = outs["host"].cpu().numpy()
        assert np.all(np.isnan(yh[out_off[1:] - 1]))
    plan.close()


def test_persistent_single_and_empty_classes(cuda_device):
    """Classes with no signals, and a batch smaller than one tile of the small classes."""
    plan = mci.Plan(SYSTEMS, PS, [4 * p for p in PS], max_batch=16)
    rng = S.rng_for(7, 3)
    cls = np.array([4, 0, 4, 2], np.int32)          # classes 1 and 3 empty
    in_len = [3 * PS[c] for c in cls]
    x = torch.tensor(rng.standard_normal(sum(in_len)), dtype=torch.float32, device="cuda")
    out_off = np.concatenate([[0], np.cumsum([4 * PS[c] for c in cls])[:-1]]).astype(np.int64)
    in_off = np.concatenate([[0], np.cumsum(in_len)[:-1]]).astype(np.int64)
    n_out = int(sum(4 * PS[c] for c in cls))
    ys = []
    for sc in (cls, torch.tensor(cls, device="cuda")):
        y = torch.full((n_out,), float("nan"), device="cuda")
        mci.mci_interp_1d(plan.handle, x, None, y, None, sc, len(cls))
        ys.append(y)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    assert torch.equal(ys[0], ys[1])
    xs, yh = x.cpu().double().numpy(), ys[0].cpu().double().numpy()
    for b, c in enumerate(cls):
        P = PS[c]
        want = O.mci_direct(SYSTEMS, xs[in_off[b]:in_off[b] + 3 * P].reshape(3, P), 4 * P)[0]
        assert rel(yh[out_off[b]:out_off[b] + 4 * P], want) <= 1e-5
    plan.close()
