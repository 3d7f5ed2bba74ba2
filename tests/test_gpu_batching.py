"""Batching machinery of the 1-D path: the plan-time tile autotuner (results must not
depend on the tile height it picks) and CUDA-graph capture of the launches that allow
it (uniform batches; device-side grouping through the no-allocation entry point)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1802_10291_gb300 import mci
from paper_1802_10291_gb300 import synth as S

pytestmark = pytest.mark.gpu

SYSTEMS = [("identity",), ("hilbert",), ("deriv", 1)]
PS = [256, 512, 1024, 2048, 4096]


def _uneven(seed, batch):
    rng = S.rng_for(7, seed)
    cls = rng.integers(0, len(PS), batch).astype(np.int32)
    cls[:len(PS)] = np.arange(len(PS))
    in_len = np.array([3 * PS[c] for c in cls])
    out_len = np.array([4 * PS[c] for c in cls])
    x = rng.standard_normal(int(in_len.sum()))
    return cls, in_len, out_len, x


def test_autotune_gives_identical_results(cuda_device):
    cls, in_len, out_len, xh = _uneven(1, 60)
    x = torch.tensor(xh, dtype=torch.float32, device="cuda")
    outs, infos = [], []
    for tune in (False, True):
        plan = mci.Plan(SYSTEMS, PS, [4 * p for p in PS], max_batch=60, autotune=tune)
        y = torch.full((int(out_len.sum()),), float("nan"), device="cuda")
        mci.mci_interp_1d(plan.handle, x, None, y, None, cls, 60)
        torch.cuda.synchronize()
        infos.append(plan.info())
        assert infos[-1]["device_status"] == 0
        outs.append(y)
        plan.close()
    # each signal's arithmetic is independent of how many share a CTA
    assert torch.equal(outs[0], outs[1])
    assert all(1 <= g <= 64 for g in infos[1]["signals_per_cta"][:len(PS)])
    # and both match the oracle on the first signal of every class
    out_off = np.concatenate([[0], np.cumsum(out_len)[:-1]])
    in_off = np.concatenate([[0], np.cumsum(in_len)[:-1]])
    yh = outs[1].cpu().double().numpy()
    for b in range(len(PS)):
        P = PS[cls[b]]
        ref = O.mci_direct(SYSTEMS, xh[in_off[b]:in_off[b] + 3 * P].reshape(1, 3, P), 4 * P)[0, 0]
        got = yh[out_off[b]:out_off[b] + 4 * P]
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.sqrt(np.mean(ref ** 2))


def test_graph_capture_uniform_batch(cuda_device):
    P, batch = 1024, 300
    rng = S.rng_for(7, 2)
    plan = mci.Plan(SYSTEMS, P, 4 * P, max_batch=batch)
    x = torch.tensor(rng.standard_normal((batch, 3, P)), dtype=torch.float32, device="cuda")
    y = torch.empty((batch, 1, 4 * P), device="cuda")
    plan.interp_1d(x, y)                       # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.interp_1d(x, y)
    x.copy_(torch.tensor(rng.standard_normal((batch, 3, P)), dtype=torch.float32))
    y.fill_(float("nan"))
    g.replay()
    ref = torch.empty_like(y)
    plan.interp_1d(x, ref)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    assert torch.equal(y, ref)
    plan.close()


def test_graph_capture_device_grouping(cuda_device):
    """Size classes in device memory, scratch in the library's static array: the whole
    uneven step (grouping kernel and its device-side class launches) replays from a graph."""
    cls, in_len, out_len, xh = _uneven(3, 50)
    x = torch.tensor(xh, dtype=torch.float32, device="cuda")
    sc = torch.tensor(cls, device="cuda")
    plan = mci.Plan(SYSTEMS, PS, [4 * p for p in PS], max_batch=50)
    y = torch.full((int(out_len.sum()),), float("nan"), device="cuda")
    mci.mci_interp_1d_noalloc(plan.handle, x, None, y, None, sc, 50)   # warm-up, symbol lookup
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mci.mci_interp_1d_noalloc(plan.handle, x, None, y, None, sc, 50)
    y.fill_(float("nan"))
    g.replay()
    ref = torch.full_like(y, float("nan"))
    mci.mci_interp_1d(plan.handle, x, None, ref, None, sc, 50)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    assert torch.equal(y, ref)
    plan.close()


@pytest.mark.parametrize("pinned,access", [(True, "auto"), (True, "staged"), (False, "auto")])
def test_host_buffers_pipeline(cuda_device, pinned, access):
    """mci_interp_1d_host: the same results as the device-buffer call, with page-locked
    buffers accessed in place (auto) or staged over several chunks (so the three buffer
    slots are reused), and with pageable buffers (always staged)."""
    cls, in_len, out_len, xh = _uneven(4, 6000)
    plan = mci.Plan(SYSTEMS, PS, [4 * p for p in PS], max_batch=6000, host_access=access)
    x = torch.tensor(xh, dtype=torch.float32)
    y = torch.full((int(out_len.sum()),), float("nan"), dtype=torch.float32)
    if pinned:
        x, y = x.pin_memory(), y.pin_memory()
    mci.mci_interp_1d_host(plan.handle, x, y, cls, 6000)
    xd = x.cuda()
    ref = torch.full((int(out_len.sum()),), float("nan"), device="cuda")
    mci.mci_interp_1d(plan.handle, xd, None, ref, None, cls, 6000)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0
    assert torch.equal(y, ref.cpu())
    plan.close()


@pytest.mark.parametrize("access", ["auto", "staged"])
def test_refused_allocations_return_oom_and_free(cuda_device, access):
    """Every allocation of plan creation refused in turn (test hook): MCI_ERR_OOM, nothing
    leaked on the device, and the first plan that gets all its memory works.  A staged plan
    also allocates its host-path chunk buffers at creation."""
    from paper_1802_10291_gb300 import mci as M
    systems = [("identity",), ("hilbert",), ("deriv", 1)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    refused = 0
    try:
        for k in range(32):
            M.mci_debug_fail_allocation(k)
            try:
                plan = M.Plan(systems, [256, 512], [1024, 2048], max_batch=64, host_access=access)
            except M.MciError as e:
                assert e.status == M.MCI_ERR_OOM, e.status
                refused += 1
                continue
            break
    finally:
        M.mci_debug_fail_allocation(-1)
    assert refused >= 3
    x = torch.randn((5, 3, 256), device="cuda")
    y = torch.empty((5, 1, 1024), device="cuda")
    M.mci_interp_1d(plan.handle, x, None, y, None, np.zeros(5, np.int32), 5)
    torch.cuda.synchronize()
    assert plan.info()["device_status"] == 0 and torch.isfinite(y).all()
    plan.close()
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 64 << 20


def test_auto_host_route_settles_and_agrees(cuda_device):
    """host_access auto with device-mapped buffers: the first three calls time the zero-copy
    and the staged routes, then the plan keeps one; every call's output equals the
    device-buffer call bit for bit."""
    systems = [("identity",), ("hilbert",), ("deriv", 1)]
    PS = [256, 512, 1024]
    plan = mci.Plan(systems, PS, [4 * p for p in PS], max_batch=8192)
    rng = np.random.default_rng(11)
    cls = rng.integers(0, 3, 6000).astype(np.int32)   # several 16 MB chunks when staged
    P = np.array(PS)[cls]
    h_in = torch.tensor(rng.standard_normal(int(3 * P.sum())), dtype=torch.float32).pin_memory()
    h_out = torch.empty(int(4 * P.sum()), dtype=torch.float32).pin_memory()
    d_out = torch.empty_like(h_out, device="cuda")
    mci.mci_interp_1d(plan.handle, h_in.cuda(), None, d_out, None, torch.tensor(cls, device="cuda"), len(cls))
    torch.cuda.synchronize()
    ref = d_out.cpu()
    routes = []
    for _ in range(5):
        h_out.fill_(float("nan"))
        mci.mci_interp_1d_host(plan.handle, h_in, h_out, cls, len(cls))
        assert torch.equal(h_out, ref)
        routes.append(plan.info()["host_route"])
    assert routes[:2] == [0, 0] and routes[2] in (1, 2) and len(set(routes[2:])) == 1, routes
    assert plan.info()["device_status"] == 0
    plan.close()


def test_staged_plan_host_calls_allocate_nothing(cuda_device):
    """A plan made with host_access = staged holds its chunk buffers from creation: its
    host-buffer calls, the first included, leave the device's free memory unchanged."""
    systems = [("identity",), ("hilbert",), ("deriv", 1)]
    PS = [256, 512, 1024]
    plan = mci.Plan(systems, PS, [4 * p for p in PS], max_batch=4096, host_access="staged")
    rng = np.random.default_rng(7)
    cls = rng.integers(0, 3, 3000).astype(np.int32)
    P = np.array(PS)[cls]
    h_in = torch.tensor(rng.standard_normal(int(3 * P.sum())), dtype=torch.float32).pin_memory()
    h_out = torch.empty(int(4 * P.sum()), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        mci.mci_interp_1d_host(plan.handle, h_in, h_out, cls, len(cls))
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 4 << 20
    assert plan.info()["device_status"] == 0 and torch.isfinite(h_out).all()
    # the same batch through device buffers gives the same samples
    d_out = torch.empty_like(h_out, device="cuda")
    mci.mci_interp_1d(plan.handle, h_in.cuda(), None, d_out, None, torch.tensor(cls, device="cuda"), len(cls))
    torch.cuda.synchronize()
    assert torch.equal(d_out.cpu(), h_out)
    plan.close()


def test_autotune_cache_reused_and_saved(cuda_device, tmp_path):
    """A second autotuned plan with the same classes takes the tile heights from the cache
    (no timing: much faster plan creation, same heights); save / load round-trips them."""
    import json
    import time
    systems = [("identity",), ("deriv", 1)]
    Ps, Ts = [96, 192, 384], [288, 576, 1152]    # generic-kernel classes (3 x 2^a)
    t0 = time.perf_counter()
    a = mci.Plan(systems, Ps, Ts, max_batch=64, autotune=True)
    t1 = time.perf_counter()
    b = mci.Plan(systems, Ps, Ts, max_batch=64, autotune=True)
    t2 = time.perf_counter()
    ga, gb = a.info()["signals_per_cta"][:3], b.info()["signals_per_cta"][:3]
    assert ga == gb
    assert t2 - t1 < 0.5 * (t1 - t0)
    path = tmp_path / "tune.json"
    mci.mci_tune_cache_save(str(path))
    saved = json.loads(path.read_text())
    keys = [k for k in saved if "|P=384|T=1152|" in k]
    assert keys and saved[keys[0]] == ga[2]
    mci.mci_tune_cache_load(str(path))
    a.close()
    b.close()
