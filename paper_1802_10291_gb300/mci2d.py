"""Python binding of include/mci2d.h (ctypes; argument marshalling only): two-dimensional
multichannel interpolation of real images with 2-D channel systems."""
from __future__ import annotations

import ctypes

from . import mci

MCI2_SYS = {"identity": 0, "partial": 1, "laplacian": 2, "shift": 3, "riesz": 4}


class mci2_system(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("order_y", ctypes.c_int), ("order_x", ctypes.c_int),
                ("tau_y", ctypes.c_double), ("tau_x", ctypes.c_double)]


class mci2_desc(ctypes.Structure):
    _fields_ = [("My", ctypes.c_int), ("Mx", ctypes.c_int), ("sys", ctypes.POINTER(mci2_system)),
                ("P1", ctypes.c_int), ("P2", ctypes.c_int), ("T1", ctypes.c_int), ("T2", ctypes.c_int),
                ("N1", ctypes.POINTER(ctypes.c_int64)), ("precision", ctypes.c_int),
                ("singular_policy", ctypes.c_int), ("singular_rtol", ctypes.c_double),
                ("max_batch", ctypes.c_int64)]


_bound = False


def _lib():
    global _bound
    lib = mci.load()
    if not _bound:
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.mci2_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(mci2_desc), vp]
        lib.mci2_interp.argtypes = [vp, vp, vp, i64, vp]
        lib.mci2_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(i64)]
        lib.mci2_destroy.argtypes = [vp]
        for f in ("mci2_plan", "mci2_interp", "mci2_plan_info", "mci2_destroy"):
            getattr(lib, f).restype = ctypes.c_int
        _bound = True
    return lib


def make_desc(systems, grid, P, T, N1=None, precision="fp32", singular="pinv", singular_rtol=0.0,
              max_batch=1):
    """systems: My * Mx tuples ('identity',), ('partial', a, b) = (i ny)^a (i nx)^b,
    ('laplacian',), ('shift', tau_y, tau_x), ('riesz', axis); grid = (My, Mx);
    P = (P1, P2) samples per channel; T = (T1, T2) output grid."""
    arr = (mci2_system * len(systems))()
    for k, s in enumerate(systems):
        arr[k].kind = MCI2_SYS[s[0]]
        if s[0] == "partial":
            arr[k].order_y, arr[k].order_x = int(s[1]), int(s[2])
        elif s[0] == "riesz":
            arr[k].order_y = int(s[1])
        elif s[0] == "shift":
            arr[k].tau_y, arr[k].tau_x = float(s[1]), float(s[2])
    d = mci2_desc()
    d.My, d.Mx = int(grid[0]), int(grid[1])
    d.sys = arr
    d.P1, d.P2 = int(P[0]), int(P[1])
    d.T1, d.T2 = int(T[0]), int(T[1])
    n1 = None
    if N1 is not None:
        n1 = (ctypes.c_int64 * 2)(int(N1[0]), int(N1[1]))
    d.N1 = n1
    d.precision = {"fp32": mci.MCI_FP32, "fp64": mci.MCI_FP64}[precision]
    d.singular_policy = {"pinv": mci.MCI_SINGULAR_PINV, "error": mci.MCI_SINGULAR_ERROR,
                         "zero": mci.MCI_SINGULAR_ZERO}[singular]
    d.singular_rtol = float(singular_rtol)
    d.max_batch = int(max_batch)
    d._keep = (arr, n1)
    return d


class Plan2D:
    """Owns an mci2 plan; arguments as :func:`make_desc`."""

    def __init__(self, systems, grid, P, T, stream=None, **kw):
        self.desc = make_desc(systems, grid, P, T, **kw)
        h = ctypes.c_void_p()
        mci._check(_lib().mci2_plan(ctypes.byref(h), ctypes.byref(self.desc), mci._stream(stream)),
                   "mci2_plan")
        self.handle = h.value
        self.grid, self.P, self.T = tuple(grid), tuple(P), tuple(T)

    def interp(self, inp, out, batch=None, stream=None):
        """inp [batch][M][P1][P2] -> out [batch][T1][T2] (device tensors of the plan's precision)."""
        if batch is None:
            batch = inp.shape[0]
        mci._check(_lib().mci2_interp(self.handle, mci._ptr(inp), mci._ptr(out), int(batch),
                                      mci._stream(stream)), "mci2_interp")
        return out

    def info(self):
        ns, mc, ws = ctypes.c_int(), ctypes.c_double(), ctypes.c_int64()
        mci._check(_lib().mci2_plan_info(self.handle, ctypes.byref(ns), ctypes.byref(mc), ctypes.byref(ws)),
                   "mci2_plan_info")
        return {"n_singular": ns.value, "max_cond": mc.value, "workspace_bytes": ws.value}

    def close(self):
        if self.handle:
            mci._check(_lib().mci2_destroy(self.handle), "mci2_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
