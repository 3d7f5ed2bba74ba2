"""Benchmark: batched 1-D FFT multichannel interpolation on GB300.

Workload (one step = one mci_interp_1d call over the whole batch):
16384 signals, M = 3 channels {identity, Hilbert, derivative}, P drawn
uniformly from {256, 512, 1024, 2048, 4096} per signal, T = 4P output
samples, half trigonometric polynomials over the band {-3P/2 .. 3P/2 - 1},
half exp(a cos(t - phi)) (synthetic, seeded).  FP32 is the headline; the FP64
path runs the same batch for the FP32-vs-FP64 comparison.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank processes its own batch (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import select
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MCI output Msamples/s & HR Mpixel/s, FP32 vs FP64 GPU at stated err; % HBM peak"
UNIT = "Msamples/s"
SYSTEMS = [("identity",), ("hilbert",), ("deriv", 1)]
P_CHOICES = [256, 512, 1024, 2048, 4096]
N_SIGNALS = 16384
S_FACTOR = 4
WORKLOAD = ("batched 1-D MCI: 16384 signals, M=3 {identity, Hilbert -i sgn, derivative i n}, "
            "P ~ U{256,512,1024,2048,4096}, T=4P, half trig polynomials, half exp(a cos(t-phi))")


# Signals per size class in the CPU-oracle sample (about 10 s on 16 host cores); the
# same sample gives the realised FP32/FP64 errors.
CPU_PER_CLASS = 100

# DRAM bytes (read + write) of one launch of the roofline kernel (the persistent launch that
# serves the whole batched step), from one ncu capture of that launch on this workload.
# None whenever the kernel has changed since the capture.
ROOFLINE_TRAFFIC_PER_STEP = 310034944 + 357062144
# the same for the P = 4096 class kernel timed alone (3201 signals), per signal
CLASS4096_TRAFFIC_PER_SIGNAL = (157665024 + 153586688) / 3201


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_batch(rank: int, n_signals: int = N_SIGNALS):
    """This rank's own batch: seeded by the rank, so ranks process different signals."""
    from paper_1802_10291_gb300 import synth
    rng = synth.rng_for(1, 1000 + rank)
    b = synth.uneven_batch_1d(rng, n_signals, P_CHOICES, SYSTEMS)
    P_of = b["P"]
    cls = np.searchsorted(np.asarray(P_CHOICES), P_of).astype(np.int32)
    flat = np.concatenate([g.ravel() for g in b["g"]])
    in_len = 3 * P_of
    out_len = S_FACTOR * P_of
    in_off = np.concatenate([[0], np.cumsum(in_len)[:-1]]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(out_len)[:-1]]).astype(np.int64)
    return dict(P=P_of, cls=cls, flat=flat, g=b["g"], kind=b["kind"], in_off=in_off,
                out_off=out_off, n_in=int(in_len.sum()), n_out=int(out_len.sum()))


# Child process that polls NVML (read-only queries) every millisecond and prints
# "sm_mhz,max_sm_mhz,event_reason_bits" per sample; argv[1] is the GPU's PCI bus id.
_NVML_POLLER = r"""
import ctypes, sys, time
nv = ctypes.CDLL("libnvidia-ml.so.1")
assert nv.nvmlInit_v2() == 0
h = ctypes.c_void_p()
assert nv.nvmlDeviceGetHandleByPciBusId_v2(sys.argv[1].encode(), ctypes.byref(h)) == 0
get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
    nv.nvmlDeviceGetCurrentClocksThrottleReasons
cur, mx, bits = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
while True:
    nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(cur))
    nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
    get_reasons(h, ctypes.byref(bits))
    sys.stdout.write("%d,%d,%d\n" % (cur.value, mx.value, bits.value))
    sys.stdout.flush()
    time.sleep(0.001)
"""


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled during the timed region: every
    millisecond through NVML in a child process (so that the launching thread shares no
    interpreter lock with it), else every 50 ms through nvidia-smi.  The sampler's first line
    (taken before the region starts) is awaited and then left out."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int, bus_id: str = None):
        self.index = index
        self.bus_id = bus_id
        self.proc = None
        self.kind = None

    def _start(self, cmd, kind):
        proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        ready, _, _ = select.select([proc.stdout], [], [], 10.0)
        if ready and proc.stdout.readline().strip():
            self.proc, self.kind = proc, kind          # first sample: before the timed region
            return True
        proc.kill()
        proc.communicate()
        return False

    def __enter__(self):
        try:
            if self.bus_id and self._start([sys.executable, "-c", _NVML_POLLER, self.bus_id], "nvml"):
                return self
        except Exception:
            self.proc = None
        try:
            self._start(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                         "--format=csv,noheader,nounits", "-lms", "50"], "nvidia-smi")
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                if self.kind == "nvml":
                    sm.append(float(f[0]))
                    mx.append(float(f[1]))
                    bits = int(f[2])
                    reasons.update(n for n, b in self.BITS.items() if bits & b)
                    continue
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "source": self.kind}


def bind_host_to_gpu(torch, index: int):
    """Run this process on the CPU cores local to GPU `index` (from the PCI device's
    local_cpulist), so that the page-locked host buffers of the end-to-end measurement are
    placed in the memory next to that GPU.  Returns the core list, or None if unknown."""
    try:
        pr = torch.cuda.get_device_properties(index)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        text = open(f"/sys/bus/pci/devices/{bus}/local_cpulist").read().strip()
        cpus = set()
        for part in text.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
            return text
    except (OSError, ValueError, AttributeError):
        return None
    return None


def dist_setup(n_gpus: int, backend: str = "nccl"):
    """(world, rank, local rank) from the torchrun environment; joins the process group
    when world > 1 (NCCL on the GPU machine; the CPU tests use gloo)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of x over all ranks (the step time every rank reports is the slowest one)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, steps: int, max_seconds: float) -> float:
    """Weak scaling: every rank processes its own batch of units_per_rank per step, so the
    job's throughput is all ranks' units over the slowest rank's time (units/s)."""
    return units_per_rank * world * steps / max_seconds


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_sample(batch, n_per_class=2, seed=0):
    """Indices of a stratified sample: n_per_class signals of every P (half of each kind)."""
    rng = np.random.default_rng(seed)
    idx = []
    for P in P_CHOICES:
        for kind in ("trig", "smooth"):
            cand = np.nonzero((batch["P"] == P) & (batch["kind"] == kind))[0]
            k = max(1, n_per_class // 2)
            idx.extend(rng.choice(cand, size=min(k, cand.size), replace=False).tolist())
    return sorted(idx)


def run_oracle(batch, idx, nthreads=0):
    """FP64 oracle (direct sum formula) on the signals idx; returns {b: [1, T]} and seconds.
    nthreads = 0: all host cores."""
    import oracle
    t0 = time.perf_counter()
    res = {}
    for P in P_CHOICES:
        sel = [b for b in idx if batch["P"][b] == P]
        if not sel:
            continue
        g = np.stack([batch["g"][b] for b in sel])
        out = oracle.mci_direct(SYSTEMS, g, S_FACTOR * P, nthreads=nthreads)
        for i, b in enumerate(sel):
            res[b] = out[i]
    return res, time.perf_counter() - t0


def reference_arm(args, world, rank):
    """The oracle on the host cores: step i is one signal of P class i mod 5 (distinct signals,
    rotating over the classes), so that K steps cover all classes evenly.  The warm-up steps'
    signals run first, untimed; the K timed steps' signals then run through the oracle grouped
    by class (one call per class, as the oracle takes a batch), timed as a whole."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    batch = make_batch(0)
    members = {P: np.nonzero(batch["P"] == P)[0] for P in P_CHOICES}
    idx = []
    for step in range(args.warmup + args.steps):
        P = P_CHOICES[step % len(P_CHOICES)]
        idx.append(int(members[P][(step // len(P_CHOICES)) % len(members[P])]))
    if args.warmup:
        run_oracle(batch, idx[:args.warmup])
    timed_idx = idx[args.warmup:]
    _, total = run_oracle(batch, timed_idx)
    outs = sum(S_FACTOR * int(batch["P"][b]) for b in timed_idx)
    value = outs / total / 1e6
    cores = os.cpu_count()
    sample = (f"{args.steps} steps of one signal each, rotating over the five P classes, run by the "
              "FP64 oracle (direct sum formula, interpolating functions tabulated per class) in one "
              f"call per class: {total:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def uneven_2d_section(mci, torch, dev, timed, steps):
    """256 images, LR side ~ U{128..1024}, s ~ U{2,3,4}, M = 2 {f, FD f'}."""
    from paper_1802_10291_gb300 import synth
    sysd = [("identity",), ("deriv", 1)]
    out = {}
    # --- 256 images, LR side ~ U{128..1024}, s ~ U{2,3,4}
    rng = synth.rng_for(3, 0)
    sides = [128, 256, 384, 512, 768, 1024]
    scales = [2, 3, 4]
    side = rng.choice(sides, 256)
    sc = rng.choice(scales, 256)
    pool = {L: [synth.synthetic_image(rng, L).astype(np.float32) for _ in range(4)] for L in sides}
    imgs = [pool[int(L)][i % 4] for i, L in enumerate(side)]
    PT = sorted({(int(L), int(L) * int(k)) for L in sides for k in scales})
    inter = int(sum(int(L) * int(k) * int(L) for L, k in zip(side, sc)))
    plan = mci.Plan(sysd, [p for p, _ in PT], [t for _, t in PT], channels="fd", max_batch=1,
                    max_images=256, max_intermediate=inter)
    lr = torch.tensor(np.concatenate([im.ravel() for im in imgs]), device=dev)
    n_hr = int(sum(int(k) * int(k) * int(L) * int(L) for L, k in zip(side, sc)))
    hr = torch.empty(n_hr, device=dev)
    hh = np.ascontiguousarray(side, np.int32)
    ss = np.ascontiguousarray(sc, np.int32)
    n = max(5, steps // 10)
    t, _ = timed(lambda: plan.upsample_2d(lr, hh, hh, ss, hr, 256), n, 3)
    ms = 1e3 * t / n
    out["uneven_256_images"] = {"hr_mpixel_s": n_hr / (ms / 1e3) / 1e6, "ms_per_batch": ms,
                                "hr_pixels": n_hr, "gbs_lr_plus_hr": 4 * (lr.numel() + n_hr) / (ms / 1e3) / 1e9,
                                "note": "LR images generated at LR size from a pool of 4 per side"}
    plan.close()
    return out


def images_2d_section(mci, torch, dev, timed, steps):
    """Image workloads: SISR of 64 synthetic 512^2 images from x2 and x4 decimations, and an
    uneven batch of 256 images (LR side in {128..1024}, scale in {2,3,4})."""
    from paper_1802_10291_gb300 import synth
    import oracle
    sysd = [("identity",), ("deriv", 1)]
    out = {}
    # --- 64 x 512^2 HR, decimated by 2 and by 4
    rng = synth.rng_for(2, 0)
    hr_np = np.stack([synth.synthetic_image(rng, 512) for _ in range(64)]).astype(np.float32)
    for s_ in (2, 4):
        lr_np = synth.decimate(hr_np, s_)
        L = lr_np.shape[-1]
        plan = mci.Plan(sysd, L, s_ * L, channels="fd", max_batch=1, max_images=64,
                        max_intermediate=64 * L * s_ * L)
        lr = torch.tensor(lr_np.reshape(-1), device=dev)
        hr = torch.empty(64 * 512 * 512, device=dev)
        hh = np.full(64, L, np.int32)
        ss = np.full(64, s_, np.int32)
        n = max(20, steps)
        t, _ = timed(lambda: plan.upsample_2d(lr, hh, hh, ss, hr, 64), n, 3)
        ms = 1e3 * t / n
        dh = torch.tensor(hh, device=dev)
        ds = torch.tensor(ss, device=dev)
        td, _ = timed(lambda: plan.upsample_2d(lr, dh, dh, ds, hr, 64), n, 3)
        got = hr.view(64, 512, 512).cpu().numpy()
        mse = np.mean((np.clip(got, 0, 1) - hr_np) ** 2, axis=(1, 2))
        ref = oracle.upsample_2d(lr_np[0].astype(np.float64), s_, sysd)
        err = float(np.max(np.abs(got[0] - ref)) / np.sqrt(np.mean(ref ** 2)))
        bytes_ = 4 * (lr_np.size + hr_np.size)
        out[f"sisr_64x512_s{s_}"] = {
            "hr_mpixel_s": 64 * 512 * 512 / (ms / 1e3) / 1e6, "ms_per_batch": ms,
            "device_grouped_ms": 1e3 * td / n,
            "gbs_lr_plus_hr": bytes_ / (ms / 1e3) / 1e9,
            "psnr_db_mean": float(np.mean(10 * np.log10(1.0 / mse))),
            "err_vs_oracle_image0": err}
        plan.close()
    # --- the same images with mirror boundaries (mci_upsample_2d_mirror: the half-sample-
    # symmetric 2h x 2w extension interpolated as a periodic image, then cropped)
    for s_ in (2, 4):
        lr_np = synth.decimate(hr_np, s_)
        L = lr_np.shape[-1]
        plan = mci.Plan(sysd, 2 * L, 2 * s_ * L, channels="fd", max_batch=1, max_images=64,
                        max_intermediate=64 * 4 * L * s_ * L)
        lr = torch.tensor(lr_np.reshape(-1), device=dev)
        hr = torch.empty(64 * 512 * 512, device=dev)
        ext_lr = torch.empty(64 * 4 * L * L, device=dev)
        ext_hr = torch.empty(64 * 4 * 512 * 512, device=dev)
        hh = np.full(64, L, np.int32)
        ss = np.full(64, s_, np.int32)
        n = max(20, steps)
        t, _ = timed(lambda: mci.mci_upsample_2d_mirror(plan.handle, lr, hh, hh, ss, hr, 64, ext_lr, ext_hr),
                     n, 3)
        got = hr.view(64, 512, 512).cpu().numpy()
        mse = np.mean((np.clip(got, 0, 1) - hr_np) ** 2, axis=(1, 2))
        ref = oracle.upsample_2d_mirror(lr_np[0].astype(np.float64), s_, sysd)
        out[f"sisr_64x512_s{s_}_mirror"] = {
            "ms_per_batch": 1e3 * t / n, "hr_mpixel_s": 64 * 512 * 512 / (t / n) / 1e6,
            "psnr_db_mean": float(np.mean(10 * np.log10(1.0 / mse))),
            "psnr_db_mean_periodic": out[f"sisr_64x512_s{s_}"]["psnr_db_mean"],
            "err_vs_oracle_image0": float(np.max(np.abs(got[0] - ref)) / np.sqrt(np.mean(ref ** 2)))}
        plan.close()
    # --- Section 5.2 with M = 2 {f, f'} and M = 3 {f, f', f''} (centred differences), scale 3:
    # 16 synthetic 768^2 images decimated to 256^2 (P = 256, T = 768: FFT route)
    n3 = 16
    rng = synth.rng_for(2, 1)
    hr3 = np.stack([synth.synthetic_image(rng, 768) for _ in range(n3)]).astype(np.float32)
    lr3 = synth.decimate(hr3, 3)
    lr = torch.tensor(lr3.reshape(-1), device=dev)
    hr = torch.empty(n3 * 768 * 768, device=dev)
    hh = np.full(n3, 256, np.int32)
    ss = np.full(n3, 3, np.int32)
    for name, sys3 in (("m2", sysd), ("m3", sysd + [("deriv", 2)])):
        plan = mci.Plan(sys3, 256, 768, channels="fd", max_batch=1, max_images=n3,
                        max_intermediate=n3 * 256 * 768)
        n = max(20, steps)
        t, _ = timed(lambda: plan.upsample_2d(lr, hh, hh, ss, hr, n3), n, 3)
        ms = 1e3 * t / n
        got = hr.view(n3, 768, 768).cpu().numpy()
        mse = np.mean((np.clip(got, 0, 1) - hr3) ** 2, axis=(1, 2))
        ref = oracle.upsample_2d(lr3[0].astype(np.float64), 3, sys3)
        err = float(np.max(np.abs(got[0] - ref)) / np.sqrt(np.mean(ref ** 2)))
        out[f"sisr_16x768_s3_{name}"] = {
            "systems": [list(x) for x in sys3], "hr_mpixel_s": n3 * 768 * 768 / (ms / 1e3) / 1e6,
            "ms_per_batch": ms, "psnr_db_mean": float(np.mean(10 * np.log10(1.0 / mse))),
            "err_vs_oracle_image0": err}
        plan.close()
    # --- the paper's degradation (5 x 5 Gaussian, sigma 1.0, then x3) of the same images,
    # upsampled by M = 3 paper mode with the plain model and with the blur-aware channel
    # model (Wiener lambda 0.1; the true kernel, and the perturbed 7 x 7 / 1.4 of Section 5.2)
    lr3b = synth.degrade(hr3.astype(np.float64), 3, 5, 1.0).astype(np.float32)
    lr = torch.tensor(lr3b.reshape(-1), device=dev)
    sys3 = sysd + [("deriv", 2)]
    for name, blur in (("plain", None), ("aware_5x5_1.0", (5, 1.0, 0.1)), ("aware_7x7_1.4", (7, 1.4, 0.1))):
        plan = mci.Plan(sys3, 256, 768, channels="fd", max_batch=1, max_images=n3,
                        max_intermediate=n3 * 256 * 768, blur=blur)
        n = max(20, steps)
        t, _ = timed(lambda: plan.upsample_2d(lr, hh, hh, ss, hr, n3), n, 3)
        ms = 1e3 * t / n
        got = hr.view(n3, 768, 768).cpu().numpy()
        mse = np.mean((np.clip(got, 0, 1) - hr3) ** 2, axis=(1, 2))
        ref = oracle.upsample_2d(lr3b[0].astype(np.float64), 3, sys3, blur=blur)
        err = float(np.max(np.abs(got[0] - ref)) / np.sqrt(np.mean(ref ** 2)))
        out[f"sisr_blurred_16x768_s3_m3_{name}"] = {
            "degradation": "5x5 Gaussian sigma 1.0, periodic, then x3", "blur_model": blur,
            "hr_mpixel_s": n3 * 768 * 768 / (ms / 1e3) / 1e6, "ms_per_batch": ms,
            "psnr_db_mean": float(np.mean(10 * np.log10(1.0 / mse))), "err_vs_oracle_image0": err}
        plan.close()
    out.update(uneven_2d_section(mci, torch, dev, timed, steps))
    return out


def complex_section(mci, torch, dev, timed, steps):
    """Complex signals (Examples 4, 5): 4096 signals, M = 3 {f, Hf, f'}, P = 1024, T = 4P, FP32
    complex samples and outputs (no real part taken); realised error against the oracle's
    complex sum formula on 2 signals."""
    import oracle
    P, n_sig = 1024, 4096
    g = torch.Generator(device=dev)
    g.manual_seed(1802_10291 + 7)
    x = torch.randn((n_sig, 3, P, 2), generator=g, device=dev)
    y = torch.empty((n_sig, 1, 4 * P, 2), device=dev)
    plan = mci.Plan(SYSTEMS, P, 4 * P, max_batch=n_sig, complex_signal=True)
    n = max(20, steps // 4)
    t, _ = timed(lambda: plan.interp_1d(x, y, batch=n_sig), n, 3)
    ms = 1e3 * t / n
    byts = (x.numel() + y.numel()) * 4
    hbm, _ = peaks()
    xh = x[:2].double().cpu().numpy()
    ref = oracle.mci_direct_complex(SYSTEMS, xh[..., 0] + 1j * xh[..., 1], 4 * P)[:, 0]
    got = y[:2, 0].double().cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    err = float(np.max(np.abs(got - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2)))
    plan.close()
    return {"signals": n_sig, "P": P, "T": 4 * P, "ms": ms,
            "out_msamples_s": n_sig * 4 * P / (ms / 1e3) / 1e6, "gbs": byts / (ms / 1e3) / 1e9,
            "hbm_frac": byts / (ms / 1e3) / 1e9 / hbm, "fp32_err_over_rms_2_signals": err}


def mci2d_section(torch, dev, timed, steps):
    """Two-dimensional MCI (the 2-D method of the open directions of Section 5.2): 64 images,
    channels {f, f_x, f_y, f_xy} on a 2 x 2 alias lattice, 256 x 256 samples per channel, output
    768 x 768 (x3 per axis), FP32; bandlimited synthetic inputs (4 distinct images, repeated) so
    that the realised error against the exact image is known.  Inputs plus outputs (218 MB per
    batch) are larger than L2."""
    from paper_1802_10291_gb300 import mci2d, synth
    from oracle import mci2d as o2
    systems = [("identity",), ("partial", 0, 1), ("partial", 1, 0), ("partial", 1, 1)]
    grid, P, T, n_img = (2, 2), (256, 256), (768, 768), 64
    by, bx = o2.band(grid, P)
    a = synth.trig_poly_2d(synth.rng_for(16), by, bx, 4)
    g = synth.channel_samples_2d(a, by, bx, systems, P).astype(np.float32)
    x = torch.tensor(np.concatenate([g] * (n_img // 4)), device=dev)
    y = torch.empty((n_img,) + T, device=dev)
    plan = mci2d.Plan2D(systems, grid, P, T, max_batch=n_img)
    n = max(10, steps // 10)
    t, _ = timed(lambda: plan.interp(x, y), n, 3)
    ms = 1e3 * t / n
    truth = synth.sample_coeffs_2d(a[0], by, bx, T).real
    got = y[0].double().cpu().numpy()
    err = float(np.max(np.abs(got - truth)) / np.sqrt(np.mean(truth ** 2)))
    byts = (x.numel() + y.numel()) * 4
    hbm, _ = peaks()
    info = plan.info()
    plan.close()
    return {"images": n_img, "systems": [list(v) for v in systems], "P": list(P), "T": list(T), "ms": ms,
            "hr_mpixel_s": n_img * T[0] * T[1] / (ms / 1e3) / 1e6, "gbs_in_plus_out": byts / (ms / 1e3) / 1e9,
            "hbm_frac": byts / (ms / 1e3) / 1e9 / hbm, "workspace_bytes": info["workspace_bytes"],
            "fp32_err_over_rms_vs_exact": err, "launches_per_call": 3}


def exactness_section(mci, torch, dev, timed, steps):
    """One real trig polynomial on the band {-64..63}, M = 2 {f, f'}, P = 64: f and its Hilbert
    transform at T = 4096 in FP64 and FP32 -- latency of one call and the error against the
    oracle and against the exact values from the coefficients (Theorem MCIeq)."""
    from paper_1802_10291_gb300 import synth
    import oracle
    systems = [("identity",), ("deriv", 1)]
    P, T = 64, 4096
    band = synth.band_of(2, P)
    a = synth.trig_poly(synth.rng_for(0), band, 1)
    g = synth.channel_samples(a, band, systems, P)
    ref = oracle.mci_direct(systems, g, T, outputs=("f", "hilbert"))[0]
    truth = np.stack([oracle.truth_from_coeffs(a[0], band, T, o) for o in ("f", "hilbert")])
    out = {}
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        plan = mci.Plan(systems, P, T, outputs=("f", "hilbert"), precision=prec, max_batch=1)
        x = torch.tensor(g, dtype=dt, device=dev)
        y = torch.empty((1, 2, T), dtype=dt, device=dev)
        n = max(50, steps)
        t, _ = timed(lambda: plan.interp_1d(x, y), n, 3)
        got = y.cpu().double().numpy()[0]
        out[prec] = {"us_per_call": 1e6 * t / n,
                     "max_abs_err_vs_oracle": float(np.max(np.abs(got - ref))),
                     "max_abs_err_vs_truth": float(np.max(np.abs(got - truth))),
                     "rms": float(np.sqrt(np.mean(truth ** 2)))}
        plan.close()
    return {"config": "M=2 {f, f'}, P=64, band {-64..63}, outputs f and Hf at T=4096", **out}


def averaged_error_section(mci, torch, dev, timed, steps):
    """Eq. (averageerror) and the bound of Eq. (errorestimate) for 16384 signals of the
    P = 256 class of the headline systems, from 2 n_max + 1 = 6145 FP64 Fourier
    coefficients each (a(n) ~ CN(0, 1) / (1 + |n|)^1.5): HBM-bound on the coefficients."""
    import oracle
    P, n_sig = 256, 16384
    n_max = 4 * 3 * P
    L = 2 * n_max + 1
    g = torch.Generator(device=dev)
    g.manual_seed(1802_10291 + 6)
    n = torch.arange(-n_max, n_max + 1, device=dev, dtype=torch.float64)
    c = torch.randn((n_sig, L, 2), generator=g, device=dev, dtype=torch.float64)
    c = c / (1.0 + n.abs()).pow(1.5).view(1, L, 1)
    eps = torch.empty(n_sig, dtype=torch.float64, device=dev)
    bnd = torch.empty(n_sig, dtype=torch.float64, device=dev)
    plan = mci.Plan(SYSTEMS, P, 4 * P, max_batch=1)
    nrep = max(10, steps // 10)
    t, _ = timed(lambda: mci.mci_averaged_error(plan.handle, 0, c, n_max, n_sig, eps, bnd), nrep, 3)
    ms = 1e3 * t / nrep
    hbm, _ = peaks()
    gbs = c.numel() * 8 / (ms / 1e3) / 1e9
    ch = c[:2].cpu().numpy()
    rel = []
    for b in range(2):
        tab = ch[b, :, 0] + 1j * ch[b, :, 1]
        fn = lambda k, tab=tab: tab[np.asarray(k) + n_max]
        ref = oracle.averaged_error(fn, SYSTEMS, P, n_max=n_max)
        rel.append(abs(float(eps[b]) - ref) / ref)
    plan.close()
    # FP64 operations per coefficient outside the band: the Hermitian form b^H G b (M diagonal
    # terms of 4, M(M-1)/2 off-diagonal of 10), sum |b_m|^2 (3M), |a|^2 and the sums (7)
    M = len(SYSTEMS)
    outside = L - M * P
    flops = n_sig * outside * (4 * M + 10 * M * (M - 1) // 2 + 3 * M + 7)
    gflops = flops / (ms / 1e3) / 1e9
    return {"signals": n_sig, "P": P, "n_max": n_max, "ms": ms, "gbs": gbs, "hbm_frac": gbs / hbm,
            "bound": "alu (FP64)", "fp64_gflops": gflops,
            "fp64_frac_of_nominal_1250_gflops": gflops / 1250.0,
            "eps_median": float(eps.median()), "bound_over_eps_median": float((bnd / eps).median()),
            "rel_err_vs_oracle_2_signals": max(rel)}


def corrector_section(torch, dev, timed, train_steps=300, steps_per_batch=2):
    """Residual corrector on x4 MCI reconstructions of synthetic 1024^2 images: inference on
    a batch of 32, training steps on batches of 4 pairs generated on the fly (HR generated on
    the device, decimated, upsampled by MCI), PSNR of plain MCI and of the trained corrector
    on 32 held-out images."""
    from paper_1802_10291_gb300 import corrector
    size, s_, n_inf, n_tr = 1024, 4, 32, 4
    out = {}
    held = corrector.PairSource(n_inf, size, s=s_, seed=1000)
    xv, hv = held.next()
    net = corrector.Corrector(n_inf * size * size, corrector.init_params(0))
    y = torch.empty_like(xv)
    px = n_inf * size * size
    t, _ = timed(lambda: net.forward(xv, y, n_inf, size, size), 3, 1)
    ms = 1e3 * t / 3
    flop = 2 * 9 * (32 + 3 * 32 * 32 + 32) * px
    out["inference"] = {"batch": f"{n_inf}x{size}x{size}", "ms_per_batch": ms,
                        "mpixel_s": px / (ms / 1e3) / 1e6,
                        "tflop_s": flop / (ms / 1e3) / 1e12, "flop_per_batch": flop}
    src = corrector.PairSource(n_tr, size, s=s_, seed=1)
    x, hr = src.next()
    t, _ = timed(lambda: net.train_step(x, hr, n_tr, size, size, 1e-3), 5, 1)
    ms_tr = 1e3 * t / 5
    t_gen, _ = timed(src.next, 3, 1)
    ms_gen = 1e3 * t_gen / 3
    # bounded training from the identity start (last layer zero), then held-out PSNR
    net.close()
    net = corrector.Corrector(n_tr * size * size, corrector.init_params(0))
    torch.cuda.synchronize()
    t0 = time.time()
    L = torch.empty(1, device=dev)
    for it in range(train_steps):
        if it % steps_per_batch == 0:
            x, hr = src.next()
        net.train_step(x, hr, n_tr, size, size, 1e-3, loss=L)
    torch.cuda.synchronize()
    wall = time.time() - t0
    y2 = torch.empty_like(xv[:n_tr])
    psnr_c = []
    for i in range(0, n_inf, n_tr):
        net.forward(xv[i:i + n_tr], y2, n_tr, size, size)
        psnr_c.append(corrector.psnr(y2, hv[i:i + n_tr]))
    base = corrector.psnr(xv, hv)
    got = float(np.mean(psnr_c))
    pairs = train_steps * n_tr // steps_per_batch
    out["training"] = {"batch": f"{n_tr}x{size}x{size}", "ms_per_step": ms_tr,
                       "pair_generation_ms_per_batch": ms_gen,
                       "train_pairs_s": n_tr / ((ms_tr + ms_gen / steps_per_batch) / 1e3),
                       "steps": train_steps, "distinct_pairs": pairs, "lr": 1e-3, "wall_s": wall,
                       "final_loss": float(L.item())}
    out["psnr_held_out_32"] = {"mci_db": base, "corrected_db": got, "gain_db": got - base}
    net.close()
    held.plan.close()
    src.plan.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="only the FP32 step (for launch lists under a profiler)")
    ap.add_argument("--no-corrector", action="store_true")
    ap.add_argument("--pairs", type=int, default=20000,
                    help="corrector_train case: training pairs (batches of 4, one step each)")
    ap.add_argument("--case", default=None,
                    choices=["kernel4096", "corrector", "corrector_train", "corrector_small", "sisr_s2", "sisr_s4",
                             "uneven2d", "images", "mci2d", "hostlink"],
                    help="profiling case: the P=4096 size-class kernel alone on 3277 signals")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return

    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1802_10291_gb300 import mci

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    host_cpus = bind_host_to_gpu(torch, local)
    try:
        pr = torch.cuda.get_device_properties(local)
        bus_id = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
    except AttributeError:
        bus_id = None
    batch = make_batch(rank)
    n_cls = len(P_CHOICES)
    T = [S_FACTOR * p for p in P_CHOICES]
    stream = torch.cuda.current_stream()

    def setup(prec):
        dt = torch.float32 if prec == "fp32" else torch.float64
        plan = mci.Plan(SYSTEMS, P_CHOICES, T, precision=prec, max_batch=N_SIGNALS, autotune=True)
        x = torch.tensor(batch["flat"], dtype=dt, device=dev)
        y = torch.empty(batch["n_out"], dtype=dt, device=dev)
        sc = np.ascontiguousarray(batch["cls"], dtype=np.int32)   # host: host-grouped launches
        return plan, x, y, sc

    def step(plan, x, y, sc):
        mci.mci_interp_1d(plan.handle, x, None, y, None, sc, N_SIGNALS, stream)

    def timed(fn, steps, warmup, collective=True):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if collective:
            barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local, bus_id) as clk:
            torch.cuda.nvtx.range_push("timed")     # profilers can select the timed launches
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        if collective:
            barrier(world)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, clk.summary()

    def timed_local(fn, steps, warmup):
        """Rank-local timing for the sections only rank 0 runs."""
        return timed(fn, steps, warmup, collective=False)

    if args.case == "kernel4096":
        sel = np.nonzero(batch["P"] == 4096)[0]
        g4 = torch.tensor(np.stack([batch["g"][b] for b in sel]), dtype=torch.float32, device=dev)
        y4 = torch.empty((sel.size, 1, S_FACTOR * 4096), dtype=torch.float32, device=dev)
        plan4 = mci.Plan(SYSTEMS, 4096, S_FACTOR * 4096, max_batch=sel.size)
        s4, _ = timed(lambda: plan4.interp_1d(g4, y4), args.steps, args.warmup)
        print(json.dumps({"case": args.case, "signals": int(sel.size),
                          "ms_per_launch": 1e3 * s4 / args.steps}), flush=True)
        return

    if args.case == "corrector_small":
        # profiling case: forward and training steps of the corrector on 4 x 512^2 pairs
        from paper_1802_10291_gb300 import corrector
        src = corrector.PairSource(4, 512, s=4, seed=7)
        x, hr = src.next()
        net = corrector.Corrector(4 * 512 * 512, corrector.init_params(0))
        y = torch.empty_like(x)
        tf, _ = timed(lambda: net.forward(x, y, 4, 512, 512), args.steps, args.warmup)
        tt, _ = timed(lambda: net.train_step(x, hr, 4, 512, 512, 1e-3), args.steps, args.warmup)
        print(json.dumps({"case": args.case, "forward_ms": 1e3 * tf / args.steps,
                          "train_step_ms": 1e3 * tt / args.steps}), flush=True)
        return
    if args.case == "mci2d":
        # two-dimensional MCI alone (three kernels per call)
        print(json.dumps({"case": args.case, **mci2d_section(torch, dev, timed, args.steps)}), flush=True)
        return
    if args.case == "images":
        # every image workload: SISR x2/x4, x3 with M = 2 and 3, the blurred x3 set, uneven batch
        print(json.dumps({"case": args.case, **images_2d_section(mci, torch, dev, timed, args.steps)}),
              flush=True)
        return
    if args.case == "hostlink":
        # the host link alone: copy-engine rates for the end-to-end step's bytes (input host to
        # device, output device to host, both at once), page-locked host buffers
        n_in, n_out = 309187584 // 4, 411725824 // 4
        h_in = torch.empty(n_in, dtype=torch.float32).pin_memory()
        h_out = torch.empty(n_out, dtype=torch.float32).pin_memory()
        d_in = torch.empty(n_in, device=dev)
        d_out = torch.empty(n_out, device=dev)
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

        def both():
            with torch.cuda.stream(s1):
                d_in.copy_(h_in, non_blocking=True)
            with torch.cuda.stream(s2):
                h_out.copy_(d_out, non_blocking=True)
        out = {}
        for name, fn, nbytes in (("h2d", lambda: d_in.copy_(h_in, non_blocking=True), 4 * n_in),
                                 ("d2h", lambda: h_out.copy_(d_out, non_blocking=True), 4 * n_out),
                                 ("both", both, 4 * (n_in + n_out))):
            best = 1e9
            for _ in range(max(3, args.steps)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t0)
            out[name] = {"bytes": nbytes, "ms": 1e3 * best, "gb_s": nbytes / best / 1e9}
        print(json.dumps({"case": args.case, **out}), flush=True)
        return
    if args.case == "uneven2d":
        # profiling case: the uneven batch of 256 images (LR side in {128..1024}, s in {2,3,4})
        out = uneven_2d_section(mci, torch, dev, timed, args.steps)
        print(json.dumps({"case": args.case, **out}), flush=True)
        return
    if args.case in ("sisr_s2", "sisr_s4"):
        # profiling cases: 64 synthetic 512^2 images from x2 (FFT path) or x4 decimation
        # (tensor-core path)
        from paper_1802_10291_gb300 import synth
        s_ = 2 if args.case == "sisr_s2" else 4
        L = 512 // s_
        rng = synth.rng_for(2, 0)
        hr_np = np.stack([synth.synthetic_image(rng, 512) for _ in range(64)]).astype(np.float32)
        lr_np = synth.decimate(hr_np, s_)
        plan = mci.Plan([("identity",), ("deriv", 1)], L, 512, channels="fd", max_batch=1,
                        max_images=64, max_intermediate=64 * L * 512)
        lr = torch.tensor(lr_np.reshape(-1), device=dev)
        hr = torch.empty(64 * 512 * 512, device=dev)
        hh = np.full(64, L, np.int32)
        ss = np.full(64, s_, np.int32)
        t, _ = timed(lambda: plan.upsample_2d(lr, hh, hh, ss, hr, 64), args.steps, args.warmup)
        print(json.dumps({"case": args.case, "ms_per_batch": 1e3 * t / args.steps}), flush=True)
        return
    if args.case == "corrector_train":
        # the configured training: --pairs fresh pairs of 1024^2 (x4 MCI), 4 per step
        print(json.dumps({"case": args.case, **corrector_section(torch, dev, timed, args.pairs // 4, 1)}),
              flush=True)
        return
    if args.case == "corrector":
        print(json.dumps({"case": args.case, **corrector_section(torch, dev, timed, args.steps)}),
              flush=True)
        return

    # ---- FP32 headline (size classes in host memory: grouped and launched from the host)
    plan32, x32, y32, sc = setup("fp32")
    plan32_stage_bytes = 3 * 8 * N_SIGNALS
    info = plan32.info()
    secs, clocks = timed(lambda: step(plan32, x32, y32, sc), args.steps, args.warmup)
    secs = max_over_ranks(secs, world)
    out_samples = batch["n_out"] * world
    value = whole_job_rate(batch["n_out"], world, args.steps, secs) / 1e6
    st = plan32.info()
    assert st["device_status"] == 0, st
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "value": value, "unit": UNIT,
                              "ms_per_step": 1e3 * secs / args.steps}), flush=True)
        return

    # the same step with the size classes in device memory (grouped and launched on the device)
    d_sc = torch.tensor(sc, device=dev)
    secs_dev, _ = timed(lambda: step(plan32, x32, y32, d_sc), max(20, args.steps // 4), 3)
    ms_dev = 1e3 * secs_dev / max(20, args.steps // 4)
    # ... and that device-grouped step captured once in a CUDA graph and replayed
    mci.mci_interp_1d_noalloc(plan32.handle, x32, None, y32, None, d_sc, N_SIGNALS, stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        mci.mci_interp_1d_noalloc(plan32.handle, x32, None, y32, None, d_sc, N_SIGNALS)
    secs_graph, _ = timed(graph.replay, max(20, args.steps // 4), 3)
    ms_graph = 1e3 * secs_graph / max(20, args.steps // 4)

    # roofline of the step's interpolation kernels: algorithmic bytes = samples in + out
    hbm, peak_kind = peaks()
    bytes_step = 4 * (batch["n_in"] + batch["n_out"])
    achieved = bytes_step * args.steps / (secs) / 1e9

    # dominant kernel alone: the P = 4096 tiles as a uniform batch, host-launched
    sel = np.nonzero(batch["P"] == 4096)[0]
    g4 = torch.tensor(np.stack([batch["g"][b] for b in sel]), dtype=torch.float32, device=dev)
    y4 = torch.empty((sel.size, 1, S_FACTOR * 4096), dtype=torch.float32, device=dev)
    plan4 = mci.Plan(SYSTEMS, 4096, S_FACTOR * 4096, max_batch=sel.size)
    s4, _ = timed(lambda: plan4.interp_1d(g4, y4), max(20, args.steps // 4), 3)
    k_bytes = 4 * (3 * 4096 + S_FACTOR * 4096) * sel.size
    k_ms = 1e3 * s4 / max(20, args.steps // 4)
    k_achieved = k_bytes / (k_ms / 1e3) / 1e9

    # ---- image workloads (2-D)
    # single-GPU characterisations of the other workloads: at N = 1 only (under torchrun the
    # other ranks would idle while rank 0 runs them)
    solo = rank == 0 and world == 1
    images = images_2d_section(mci, torch, dev, timed_local, args.steps) if solo else None
    corr = corrector_section(torch, dev, timed_local) if solo and not args.no_corrector else None
    averr = averaged_error_section(mci, torch, dev, timed_local, args.steps) if solo else None
    exact = exactness_section(mci, torch, dev, timed_local, args.steps) if solo else None
    cplx = complex_section(mci, torch, dev, timed_local, args.steps) if solo else None
    two_d = mci2d_section(torch, dev, timed_local, args.steps) if solo else None

    # ---- FP64 on the same batch
    plan64, x64, y64, _ = setup("fp64")
    steps64 = max(3, args.steps // 20)
    secs64, _ = timed(lambda: step(plan64, x64, y64, sc), steps64, 3)
    secs64 = max_over_ranks(secs64, world)
    value64 = out_samples * steps64 / secs64 / 1e6

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timing
    h_in = torch.tensor(batch["flat"], dtype=torch.float32).pin_memory()
    h_out = torch.empty(batch["n_out"], dtype=torch.float32).pin_memory()
    def e2e_step():
        # host buffers through the C ABI: page-locked and device-mapped, so the library can
        # read and write them in place over the host link or stage them; its first three calls
        # (the warm-up) time both routes and the plan keeps the faster on this machine
        mci.mci_interp_1d_host(plan32.handle, h_in, h_out, sc, N_SIGNALS, stream)

    plan_st = mci.Plan(SYSTEMS, P_CHOICES, T, max_batch=N_SIGNALS, autotune=True, host_access="staged")

    def e2e_staged_step():
        # the same call with the buffers staged: copies in, compute and copies out pipelined in chunks
        mci.mci_interp_1d_host(plan_st.handle, h_in, h_out, sc, N_SIGNALS, stream)

    # chunks of the host-buffer call (consecutive signals up to 16 MB of input): each uploads
    # the plan's grouping block once besides its samples
    n_chunks, acc = 1, 0
    for nb in (12 * batch["P"]).tolist():
        if acc > 0 and acc + nb > (16 << 20):
            n_chunks += 1
            acc = 0
        acc += nb
    e2e_steps = max(5, args.steps // 10)
    secs_e2e, _ = timed(e2e_step, e2e_steps, 3)
    secs_e2e = max_over_ranks(secs_e2e, world)
    e2e_value = out_samples * e2e_steps / secs_e2e / 1e6
    e2e_route = plan32.info()["host_route"]   # 1 zero copy, 2 staged
    secs_st, _ = timed(e2e_staged_step, e2e_steps, 3)
    secs_st = max_over_ranks(secs_st, world)
    e2e_staged_value = out_samples * e2e_steps / secs_st / 1e6
    plan_st.close()

    # ---- realised error against the FP64 oracle (stratified sample) and the CPU baseline
    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the oracle is timed at N = 1 only
        idx = oracle_sample(batch, n_per_class=CPU_PER_CLASS)
        ref, cpu_s = run_oracle(batch, idx)
        yh = y32.cpu().double().numpy()
        yh64 = y64.cpu().numpy()
        errs, errs64 = {}, {}
        for b in idx:
            P = int(batch["P"][b])
            o0 = int(batch["out_off"][b])
            r = ref[b][0]
            rms = float(np.sqrt(np.mean(r ** 2)))
            e32 = float(np.max(np.abs(yh[o0:o0 + S_FACTOR * P] - r)))
            e64 = float(np.max(np.abs(yh64[o0:o0 + S_FACTOR * P] - r)))
            errs.setdefault(P, []).append(e32 / rms)
            errs64.setdefault(P, []).append(e64)
        err = {"fp32_max_abs_over_rms": {str(k): max(v) for k, v in errs.items()},
               "fp64_max_abs": {str(k): max(v) for k, v in errs64.items()},
               "signals": len(idx)}
        n_cpu_out = sum(S_FACTOR * int(batch["P"][b]) for b in idx)
        cpu = {"value": n_cpu_out / cpu_s / 1e6, "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"{len(idx)} signals, {CPU_PER_CLASS} of each P class (half trig, half smooth), "
                         f"FP64 direct sum formula, {cpu_s:.1f} s"}
        # the same oracle on one core, on 2 signals of each class (a few seconds)
        idx1 = oracle_sample(batch, n_per_class=2, seed=1)
        _, cpu1_s = run_oracle(batch, idx1, nthreads=1)
        n1 = sum(S_FACTOR * int(batch["P"][b]) for b in idx1)
        cpu["one_core"] = {"value": n1 / cpu1_s / 1e6, "unit": UNIT, "cores": 1,
                           "sample": f"{len(idx1)} signals, 2 of each P class, {cpu1_s:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "signals_per_gpu": N_SIGNALS, "M": 3,
                       "P_choices": P_CHOICES, "T": "4P",
                       "l2": "inputs larger than L2 (%.0f MB in, %.0f MB out per step)"
                             % (4 * batch["n_in"] / 1e6, 4 * batch["n_out"] / 1e6),
                       "parallelism": f"independent signals per GPU x{world}"},
            "clocks": clocks,
            # one persistent launch per step when every class is fused, else one per class
            "gpu_launches": (1 if info["persistent_ctas"] > 0 else n_cls) * args.steps,
            # the step is one persistent launch: its duration is taken as the step time of the
            # CUDA events (which also hold the upload of the host grouping, ~0.4 MB), so
            # `achieved` is a lower bound for the kernel
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": ROOFLINE_TRAFFIC_PER_STEP,
                         "kernel": ("mci_fast_persistent (all five classes, one launch per step)"
                                    if info["persistent_ctas"] > 0 else "per-class kernels"),
                         "bytes_per_launch": bytes_step, "ms_per_launch": 1e3 * secs / args.steps,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "class_kernel_4096": {
                             "kernel": ("mci_fast_kernel<2048, 3, 4, 1>" if plan4.info()["fused_mask"] & 1
                                        else "mci_kernel<float, 2048>") + " (P=4096 class, 3201 signals), timed alone",
                             "bytes_per_launch": k_bytes, "ms_per_launch": k_ms, "achieved": k_achieved,
                             "frac": k_achieved / hbm,
                             "traffic": CLASS4096_TRAFFIC_PER_SIGNAL * sel.size}},
            "step_roofline": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                              "bytes_per_step": bytes_step},
            "device_grouped": {"ms_per_step": ms_dev, "value": out_samples / (ms_dev / 1e3) / 1e6,
                               "unit": UNIT, "note": "size classes in device memory: grouping "
                               "kernel, then the persistent launch (two launches, no host work)",
                               "cuda_graph_ms_per_step": ms_graph},
            "fp64": {"value": value64, "unit": UNIT, "ms_per_step": 1e3 * secs64 / steps64,
                     "speedup_fp32_over_fp64": value / value64},
            "err_vs_oracle": err,
            "images_2d": images,
            "corrector": corr,
            "averaged_error": averr,
            "exactness_m2_p64": exact,
            "complex_1d": cplx,
            "mci_2d": two_d,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 4 * batch["n_in"] + (n_chunks if e2e_route == 2 else 1) * plan32_stage_bytes,
                    "d2h_bytes_per_step": 4 * batch["n_out"], "host_cpus": host_cpus,
                    "ms_per_step": 1e3 * secs_e2e / e2e_steps,
                    "mode": ("zero copy: page-locked host buffers read and written by the kernels over the "
                             "host link" if e2e_route == 1 else
                             "staged: copies in, compute, copies out pipelined in 16 MB chunks") +
                            " (mci_interp_1d_host, host_access auto: the faster route, measured on the "
                            "first calls)"},
            "e2e_staged": {"value": e2e_staged_value, "unit": UNIT,
                           "h2d_bytes_per_step": 4 * batch["n_in"] + n_chunks * plan32_stage_bytes,
                           "d2h_bytes_per_step": 4 * batch["n_out"], "chunks": n_chunks,
                           "ms_per_step": 1e3 * secs_st / e2e_steps,
                           "mode": "staged: copies in, compute, copies out pipelined in 16 MB chunks"},
            "cpu_baseline": cpu,
            "plan": {"smem_bytes": info["smem_bytes"], "signals_per_cta": info["signals_per_cta"][:n_cls],
                     "fused_mask": info["fused_mask"], "persistent_ctas": info["persistent_ctas"]},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
