"""Python binding of include/mci_corrector.h (ctypes; argument marshalling only) and
the training loop that drives it: synthetic HR images generated on the device,
decimated, upsampled by MCI (mci_upsample_2d), then the residual corrector trained
on (MCI reconstruction, HR) pairs.  Every numerical step runs in the CUDA library."""
from __future__ import annotations

import ctypes

import numpy as np

from . import mci
from . import synth

_bound = False


def _lib():
    global _bound
    lib = mci.load()
    if not _bound:
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.mci_corrector_num_params.restype = ctypes.c_int
        lib.mci_corrector_create.argtypes = [ctypes.POINTER(vp), i64, vp, vp]
        lib.mci_corrector_forward.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.mci_corrector_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                vp, vp, vp]
        lib.mci_corrector_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_float, vp, vp]
        lib.mci_corrector_get_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
        lib.mci_corrector_set_state.argtypes = [vp, vp, ctypes.c_int]
        lib.mci_corrector_destroy.argtypes = [vp]
        lib.mci_corrector_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.mci_generate_images.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.mci_decimate.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        lib.mci_degrade.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, vp]
        for f in ("mci_corrector_create", "mci_corrector_forward", "mci_corrector_loss_grad",
                  "mci_corrector_train_step", "mci_corrector_get_state", "mci_corrector_set_state",
                  "mci_corrector_destroy", "mci_corrector_status", "mci_generate_images", "mci_decimate",
                  "mci_degrade"):
            getattr(lib, f).restype = ctypes.c_int
        _bound = True
    return lib


def num_params() -> int:
    return _lib().mci_corrector_num_params()


LAYERS = [(1, 32), (32, 32), (32, 32), (32, 32), (32, 1)]   # (cin, cout)


def init_params(seed: int = 0, zero_last: bool = True) -> np.ndarray:
    """He-initialised weights (seeded), zero biases; the last layer zero so that the
    untrained corrector returns the MCI reconstruction unchanged."""
    rng = np.random.default_rng([synth.SEED_BASE, 5, seed])
    out = []
    for l, (ci, co) in enumerate(LAYERS):
        w = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        if zero_last and l == len(LAYERS) - 1:
            w[:] = 0
        out += [w.ravel(), np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


def split_params(flat):
    """Flat parameter vector -> list of (w [co][ci][3][3], b [co])."""
    out, k = [], 0
    for ci, co in LAYERS:
        w = np.asarray(flat[k:k + co * ci * 9]).reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = np.asarray(flat[k:k + co])
        k += co
        out.append((w, b))
    return out


def _stream(stream):
    return mci._stream(stream)


class Corrector:
    def __init__(self, max_pixels: int, params=None, stream=None):
        h = ctypes.c_void_p()
        p = None if params is None else np.ascontiguousarray(params, np.float32)
        rc = _lib().mci_corrector_create(ctypes.byref(h), int(max_pixels),
                                         None if p is None else p.ctypes.data, _stream(stream))
        mci._check(rc, "mci_corrector_create")
        self.handle = h.value
        self.n = num_params()

    def forward(self, x, out, batch, h, w, stream=None):
        mci._check(_lib().mci_corrector_forward(self.handle, mci._ptr(x), mci._ptr(out), batch, h, w,
                                                _stream(stream)), "mci_corrector_forward")
        return out

    def loss_grad(self, x, hr, batch, h, w, grad=None, loss=None, stream=None):
        mci._check(_lib().mci_corrector_loss_grad(self.handle, mci._ptr(x), mci._ptr(hr), batch, h, w,
                                                  mci._ptr(grad), mci._ptr(loss), _stream(stream)),
                   "mci_corrector_loss_grad")

    def train_step(self, x, hr, batch, h, w, lr, loss=None, stream=None):
        mci._check(_lib().mci_corrector_train_step(self.handle, mci._ptr(x), mci._ptr(hr), batch, h, w,
                                                   float(lr), mci._ptr(loss), _stream(stream)),
                   "mci_corrector_train_step")

    def get_state(self):
        buf = np.zeros(3 * self.n, np.float32)
        step = ctypes.c_int()
        mci._check(_lib().mci_corrector_get_state(self.handle, buf.ctypes.data, ctypes.byref(step)),
                   "mci_corrector_get_state")
        return buf, step.value

    def status(self) -> int:
        """Device error word since the last call (0 = no error); synchronises."""
        st = ctypes.c_int()
        mci._check(_lib().mci_corrector_status(self.handle, ctypes.byref(st)), "mci_corrector_status")
        return st.value

    def set_state(self, buf, step):
        buf = np.ascontiguousarray(buf, np.float32)
        mci._check(_lib().mci_corrector_set_state(self.handle, buf.ctypes.data, int(step)),
                   "mci_corrector_set_state")

    def save(self, path):
        """Checkpoint: master weights, Adam moments and step count (numpy .npz)."""
        buf, step = self.get_state()
        np.savez(path, state=buf, step=step, n=self.n)

    def load(self, path):
        d = np.load(path)
        assert int(d["n"]) == self.n
        self.set_state(d["state"], int(d["step"]))

    def close(self):
        if self.handle:
            mci._check(_lib().mci_corrector_destroy(self.handle), "mci_corrector_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate_images(params_dev, img_dev, n, h, w, stream=None):
    mci._check(_lib().mci_generate_images(mci._ptr(params_dev), mci._ptr(img_dev), n, h, w,
                                          _stream(stream)), "mci_generate_images")


def decimate(hr_dev, lr_dev, n, h, w, s, stream=None):
    mci._check(_lib().mci_decimate(mci._ptr(hr_dev), mci._ptr(lr_dev), n, h, w, s, _stream(stream)),
               "mci_decimate")


def degrade(hr_dev, lr_dev, n, h, w, s, taps=5, sigma=1.0, stream=None):
    """Gaussian blur (taps x taps, periodic) then decimation by s, on the device."""
    mci._check(_lib().mci_degrade(mci._ptr(hr_dev), mci._ptr(lr_dev), n, h, w, s, int(taps),
                                  float(sigma), _stream(stream)), "mci_degrade")


class PairSource:
    """(MCI reconstruction, HR) pairs of n images of size x size, scale s, on the device."""

    def __init__(self, n, size, s=4, seed=0):
        import torch
        self.n, self.size, self.s = n, size, s
        lo = size // s
        self.plan = mci.Plan([("identity",), ("deriv", 1)], lo, size, channels="fd", max_batch=1,
                             max_images=n, max_intermediate=n * lo * size)
        self.rng = synth.rng_for(5, seed)
        self.hr = torch.empty((n, size, size), device="cuda")
        self.lr = torch.empty((n, lo, lo), device="cuda")
        self.mci = torch.empty((n, size, size), device="cuda")
        self.sizes = np.full(n, lo, np.int32)
        self.scales = np.full(n, s, np.int32)

    def next(self):
        import torch
        prm = torch.tensor(synth.image_params(self.rng, self.n, self.size), device="cuda")
        generate_images(prm, self.hr, self.n, self.size, self.size)
        decimate(self.hr, self.lr, self.n, self.size, self.size, self.s)
        self.plan.upsample_2d(self.lr, self.sizes, self.sizes, self.scales, self.mci, self.n)
        return self.mci, self.hr


def psnr(x, ref):
    """Mean PSNR (dB) over images of x clamped to [0, 1] against ref (torch tensors [n, h, w])."""
    import torch
    mse = ((x.clamp(0, 1) - ref) ** 2).mean(dim=(1, 2))
    return float((10 * torch.log10(1.0 / mse)).mean())
