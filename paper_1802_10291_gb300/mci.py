"""Python binding of the C ABI in ``include/mci.h`` (ctypes; argument marshalling only).

The functions carry the C names.  Every step of the interpolation runs in the
CUDA library ``_build/libmci.so``; this module only converts arguments.  It
raises :class:`MciError` on any non-zero status and refuses to run when the
library has not been built -- there is no CPU fallback.

Device buffers are passed as torch CUDA tensors (or raw integer addresses);
streams as ``torch.cuda.Stream`` objects, raw handles, or None for the current
torch stream.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmci.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mci.h")

MCI_OK = 0
MCI_ERR_INVALID_ARG = -1
MCI_ERR_UNSUPPORTED_SIZE = -2
MCI_ERR_SINGULAR = -3
MCI_ERR_CUDA = -4
MCI_ERR_OOM = -5
MCI_ERR_TIMEOUT = -6
MCI_ERR_DEVICE = -7

MCI_SYS_IDENTITY, MCI_SYS_DERIV, MCI_SYS_HILBERT, MCI_SYS_SHIFT, MCI_SYS_CUSTOM = range(5)
MCI_OUT_F, MCI_OUT_HILBERT, MCI_OUT_DERIV = 1, 2, 4
MCI_FP32, MCI_FP64 = 0, 1
MCI_SINGULAR_PINV, MCI_SINGULAR_ERROR, MCI_SINGULAR_ZERO = 0, 1, 2
MCI_CHANNELS_MEASURED, MCI_CHANNELS_FD = 0, 1
MCI_MAX_CHANNELS = 8
MCI_MAX_SIZES = 32

SYSTEM_KINDS = {"identity": MCI_SYS_IDENTITY, "deriv": MCI_SYS_DERIV, "hilbert": MCI_SYS_HILBERT,
                "shift": MCI_SYS_SHIFT, "custom": MCI_SYS_CUSTOM}
OUTPUTS = {"f": MCI_OUT_F, "hilbert": MCI_OUT_HILBERT, "deriv": MCI_OUT_DERIV}


class MciError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {error_string(status)} ({status})" if what else error_string(status))


class mci_system(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("order", ctypes.c_int), ("tau", ctypes.c_double),
                ("custom", ctypes.POINTER(ctypes.c_double))]


class mci_desc(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("sys", ctypes.POINTER(mci_system)), ("n_sizes", ctypes.c_int),
                ("P", ctypes.POINTER(ctypes.c_int)), ("T", ctypes.POINTER(ctypes.c_int)),
                ("N1", ctypes.POINTER(ctypes.c_int64)), ("out_flags", ctypes.c_uint),
                ("precision", ctypes.c_int), ("singular_policy", ctypes.c_int),
                ("singular_rtol", ctypes.c_double), ("channel_mode", ctypes.c_int),
                ("max_batch", ctypes.c_int64), ("max_images", ctypes.c_int64),
                ("max_intermediate", ctypes.c_int64), ("autotune", ctypes.c_int),
                ("complex_signal", ctypes.c_int), ("blur_taps", ctypes.c_int),
                ("blur_sigma", ctypes.c_double), ("blur_lambda", ctypes.c_double),
                ("host_access", ctypes.c_int)]


class mci_plan_stats(ctypes.Structure):
    _fields_ = [("n_singular", ctypes.c_int), ("max_cond", ctypes.c_double),
                ("device_status", ctypes.c_int), ("signals_per_cta", ctypes.c_int * MCI_MAX_SIZES),
                ("threads_per_cta", ctypes.c_int), ("smem_bytes", ctypes.c_int),
                ("table_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("fused_mask", ctypes.c_uint), ("persistent_ctas", ctypes.c_int),
                ("fused3_mask", ctypes.c_uint), ("host_route", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def _open(path: str):
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; build it with "
                          "paper_1802_10291_gb300.build.build() (no CPU fallback exists)")
    return ctypes.CDLL(path)


def load(path: str = LIB_PATH):
    """Open the CUDA library; raises when it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = _open(path)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.mci_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(mci_desc), vp]
        lib.mci_plan.restype = ctypes.c_int
        lib.mci_interp_1d.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
        lib.mci_interp_1d.restype = ctypes.c_int
        lib.mci_interp_1d_host.argtypes = [vp, vp, vp, vp, i64, vp]
        lib.mci_interp_1d_host.restype = ctypes.c_int
        lib.mci_upsample_2d_mirror.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.mci_upsample_2d_mirror.restype = ctypes.c_int
        lib.mci_averaged_error.argtypes = [vp, ctypes.c_int, vp, i64, i64, vp, vp, vp]
        lib.mci_averaged_error.restype = ctypes.c_int
        lib.mci_interp_1d_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
        lib.mci_interp_1d_noalloc.restype = ctypes.c_int
        lib.mci_upsample_2d.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i64, vp]
        lib.mci_upsample_2d.restype = ctypes.c_int
        lib.mci_plan_info.argtypes = [vp, ctypes.POINTER(mci_plan_stats)]
        lib.mci_plan_info.restype = ctypes.c_int
        lib.mci_destroy.argtypes = [vp]
        lib.mci_destroy.restype = ctypes.c_int
        lib.mci_tune_cache_save.argtypes = [ctypes.c_char_p]
        lib.mci_tune_cache_save.restype = ctypes.c_int
        lib.mci_tune_cache_load.argtypes = [ctypes.c_char_p]
        lib.mci_tune_cache_load.restype = ctypes.c_int
        lib.mci_debug_fail_allocation.argtypes = [ctypes.c_int]
        lib.mci_debug_fail_allocation.restype = None
        lib.mci_error_string.argtypes = [ctypes.c_int]
        lib.mci_error_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def header_functions(paths=None):
    """Names of the functions the headers under include/ declare."""
    if paths is None:
        d = os.path.dirname(HEADER)
        paths = [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".h")]
    elif isinstance(paths, str):
        paths = [paths]
    names = set()
    for path in paths:
        text = open(path).read()
        names |= set(re.findall(r"^\s*(?:mci_status|const char\*|int|void)\s+(mci\w*)\s*\(", text, re.M))
    return sorted(names)


def error_string(status: int) -> str:
    return load().mci_error_string(int(status)).decode()


def mci_error_string(status: int) -> str:
    return error_string(status)


def _check(rc: int, what: str):
    if rc != MCI_OK:
        raise MciError(rc, what)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data  # numpy array (host memory)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_desc(systems, P, T, N1=None, outputs=("f",), precision="fp32", singular="pinv",
              singular_rtol=0.0, channels="measured", max_batch=1, max_images=0,
              max_intermediate=0, autotune=False, complex_signal=False, blur=None, host_access="auto"):
    """Build an mci_desc (plus the arrays it points to, kept alive on the returned object).
    systems: list of ('identity',), ('deriv', k), ('hilbert',), ('shift', tau), ('custom', table)
    where table is a float64 array of 2*M*P_c values per size class, concatenated.
    blur: None, or (taps, sigma[, lambda]) for the blur-aware channel model.
    host_access: 'auto' (page-locked mapped host buffers accessed in place by
    mci_interp_1d_host) or 'staged' (always copied through device chunks)."""
    P = [int(p) for p in (P if hasattr(P, "__len__") else [P])]
    T = [int(t) for t in (T if hasattr(T, "__len__") else [T])]
    sysarr = (mci_system * len(systems))()
    keep = []
    for k, s in enumerate(systems):
        sysarr[k].kind = SYSTEM_KINDS[s[0]]
        sysarr[k].order = int(s[1]) if s[0] == "deriv" and len(s) > 1 else 1
        sysarr[k].tau = float(s[1]) if s[0] == "shift" else 0.0
        if s[0] == "custom":
            import numpy as np
            tab = np.ascontiguousarray(np.asarray(s[1], np.float64))
            keep.append(tab)
            sysarr[k].custom = tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    Parr = (ctypes.c_int * len(P))(*P)
    Tarr = (ctypes.c_int * len(T))(*T)
    N1arr = None
    if N1 is not None:
        N1 = [int(v) for v in (N1 if hasattr(N1, "__len__") else [N1])]
        N1arr = (ctypes.c_int64 * len(N1))(*N1)
    d = mci_desc()
    d.M = len(systems)
    d.sys = sysarr
    d.n_sizes = len(P)
    d.P = Parr
    d.T = Tarr
    d.N1 = N1arr
    d.out_flags = sum(OUTPUTS[o] for o in outputs)
    d.precision = {"fp32": MCI_FP32, "fp64": MCI_FP64}[precision]
    d.singular_policy = {"pinv": MCI_SINGULAR_PINV, "error": MCI_SINGULAR_ERROR,
                         "zero": MCI_SINGULAR_ZERO}[singular]
    d.singular_rtol = float(singular_rtol)
    d.channel_mode = {"measured": MCI_CHANNELS_MEASURED, "fd": MCI_CHANNELS_FD}[channels]
    d.max_batch = int(max_batch)
    d.max_images = int(max_images)
    d.max_intermediate = int(max_intermediate)
    d.autotune = 1 if autotune else 0
    d.complex_signal = 1 if complex_signal else 0
    d.host_access = {"auto": 0, "staged": 1}[host_access]
    if blur is not None:
        d.blur_taps = int(blur[0])
        d.blur_sigma = float(blur[1])
        d.blur_lambda = float(blur[2]) if len(blur) > 2 else 0.0
    d._keep = (sysarr, Parr, Tarr, N1arr, keep)
    return d


def mci_plan(desc: mci_desc, stream=None) -> int:
    """Create a plan; returns its handle (an int)."""
    h = ctypes.c_void_p()
    _check(load().mci_plan(ctypes.byref(h), ctypes.byref(desc), _stream(stream)), "mci_plan")
    return h.value


def mci_interp_1d(plan: int, inp, in_off, out, out_off, size_class, batch: int, stream=None):
    _check(load().mci_interp_1d(plan, _ptr(inp), _ptr(in_off), _ptr(out), _ptr(out_off),
                                _ptr(size_class), int(batch), _stream(stream)), "mci_interp_1d")


def mci_interp_1d_host(plan: int, inp, out, size_class, batch: int, stream=None):
    """mci_interp_1d on host buffers (packed), with copies pipelined against the compute."""
    _check(load().mci_interp_1d_host(plan, _ptr(inp), _ptr(out), _ptr(size_class), int(batch),
                                     _stream(stream)), "mci_interp_1d_host")


def mci_averaged_error(plan: int, size_class: int, coeffs, n_max: int, batch: int, eps, bound=None,
                       stream=None):
    """Phase-averaged error eps(f, N) and its bound from Fourier coefficients (device FP64)."""
    _check(load().mci_averaged_error(plan, int(size_class), _ptr(coeffs), int(n_max), int(batch),
                                     _ptr(eps), _ptr(bound), _stream(stream)), "mci_averaged_error")


def mci_interp_1d_noalloc(plan: int, inp, in_off, out, out_off, size_class, batch: int,
                          stream=None):
    """mci_interp_1d with its scratch in the library's static device array (no allocation)."""
    _check(load().mci_interp_1d_noalloc(plan, _ptr(inp), _ptr(in_off), _ptr(out), _ptr(out_off),
                                        _ptr(size_class), int(batch), _stream(stream)),
           "mci_interp_1d_noalloc")


MCI_NOALLOC_MAX_BATCH = 65536


def mci_tune_cache_save(path: str):
    """Write the autotuner's tile heights (process-wide) to a JSON file."""
    _check(load().mci_tune_cache_save(os.fsencode(path)), "mci_tune_cache_save")


def mci_tune_cache_load(path: str):
    """Merge a JSON file written by mci_tune_cache_save into the autotuner's entries."""
    _check(load().mci_tune_cache_load(os.fsencode(path)), "mci_tune_cache_load")


def mci_debug_fail_allocation(after: int):
    """Test hook: the library's allocations succeed `after` more times, then one is refused
    (MCI_ERR_OOM); negative: off."""
    load().mci_debug_fail_allocation(int(after))


def mci_upsample_2d(plan: int, lr, lr_off, h, w, scale, hr, hr_off, n_img: int, stream=None):
    _check(load().mci_upsample_2d(plan, _ptr(lr), _ptr(lr_off), _ptr(h), _ptr(w), _ptr(scale),
                                  _ptr(hr), _ptr(hr_off), int(n_img), _stream(stream)),
           "mci_upsample_2d")


def mci_upsample_2d_mirror(plan: int, lr, h, w, scale, hr, n_img: int, ext_lr, ext_hr, stream=None):
    """mci_upsample_2d on the mirror extension of each image (h, w, scale: host int32 arrays;
    ext_lr, ext_hr: device float scratch of sum 4 h w and sum 4 s^2 h w elements)."""
    _check(load().mci_upsample_2d_mirror(plan, _ptr(lr), _ptr(h), _ptr(w), _ptr(scale), _ptr(hr),
                                         int(n_img), _ptr(ext_lr), _ptr(ext_hr), _stream(stream)),
           "mci_upsample_2d_mirror")


def mci_plan_info(plan: int) -> dict:
    st = mci_plan_stats()
    _check(load().mci_plan_info(plan, ctypes.byref(st)), "mci_plan_info")
    return {"n_singular": st.n_singular, "max_cond": st.max_cond,
            "device_status": st.device_status, "signals_per_cta": list(st.signals_per_cta),
            "threads_per_cta": st.threads_per_cta, "smem_bytes": st.smem_bytes,
            "table_bytes": st.table_bytes, "workspace_bytes": st.workspace_bytes,
            "fused_mask": st.fused_mask, "persistent_ctas": st.persistent_ctas,
            "fused3_mask": st.fused3_mask, "host_route": st.host_route}


def mci_destroy(plan: int):
    _check(load().mci_destroy(plan), "mci_destroy")


class Plan:
    """Owns a plan handle; the same arguments as :func:`make_desc`."""

    def __init__(self, systems, P, T, stream=None, **kw):
        self.desc = make_desc(systems, P, T, **kw)
        self.systems = list(systems)
        self.P = [int(p) for p in (P if hasattr(P, "__len__") else [P])]
        self.T = [int(t) for t in (T if hasattr(T, "__len__") else [T])]
        self.outputs = kw.get("outputs", ("f",))
        self.handle = mci_plan(self.desc, stream)

    def interp_1d(self, inp, out, in_off=None, out_off=None, size_class=None, batch=None,
                  stream=None):
        if batch is None:
            batch = inp.shape[0]
        mci_interp_1d(self.handle, inp, in_off, out, out_off, size_class, batch, stream)
        return out

    def upsample_2d(self, lr, h, w, scale, hr, n_img, lr_off=None, hr_off=None, stream=None):
        mci_upsample_2d(self.handle, lr, lr_off, h, w, scale, hr, hr_off, n_img, stream)
        return hr

    def info(self):
        return mci_plan_info(self.handle)

    def close(self):
        if self.handle:
            mci_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
