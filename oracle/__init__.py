"""FP64 CPU oracle for FFT multichannel interpolation (MCI).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path: the heavy sums live in ``mci_oracle.c`` (plain C, built
with gcc), the rest is numpy written straight from the paper's definitions.

Notation follows Cheng & Kou, "FFT multichannel interpolation and application
to image super-resolution": M channels, P samples per channel (the paper's L),
band {N1 .. N1 + M P - 1} (Section 3), output grid t_j = 2 pi j / T.

Functions and the passage each follows:

* :func:`q_table` -- Eq. (defH) and its inverse; Remark (aequal0) for singular
  residues (pseudo-inverse, zero, or error).
* :func:`interp_functions` -- Eq. (defrm) and Eq. (ym), with an output
  operator applied to y_m as in Example 6.
* :func:`mci_direct` -- Theorem (MCIeq), Eq. (drictexpression); the
  approximation operator T_N of Eq. (appxi operator) for non-bandlimited f.
* :func:`mci_bruteforce` -- a second, independent route for tiny sizes: solve
  the mu x mu sampling system sum_n a(n) b_m(n) e^{i n t_p} = g_m(t_p) of
  Section 3 directly (minimum-norm least squares).
* :func:`fd_channels` -- the three-point centred differences of Section 5.2.
* :func:`upsample_2d` -- rows then columns, Section 5.2.
* :func:`upsample_2d_mirror` -- the same on the half-sample-symmetric extension
  of the image (mirror boundaries instead of the periodic wrap of Section 2).
* :func:`blur_factor`, :func:`blur_systems` -- the blur-aware channel model that
  Section 5.2 lists as an open extension: every channel is the system response
  blurred by a periodic Gaussian on the output grid, so each b_m(n) carries the
  blur's multiplier beta(n); optionally Wiener-regularised (a reading: the paper
  gives no formula).
* :func:`averaged_error` -- Eq. (averageerror), Theorem (error).
* :func:`truth_from_coeffs` -- evaluates a trigonometric polynomial and its
  Hilbert transform from coefficients, Eq. (bandsignal) and Section 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "mci_oracle.c")
_lock = threading.Lock()
_lib = None

SYS_KINDS = {"identity": 0, "deriv": 1, "hilbert": 2, "shift": 3, "custom": 4}
OUT_OPS = {"f": 0, "hilbert": 1, "deriv": 2}
POLICIES = {"pinv": 0, "error": 1, "zero": 2}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, dp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
            lib.oracle_q_table.argtypes = [ctypes.c_int, ip, ip, dp, dp, i64, i64, ctypes.c_int,
                                           ctypes.c_double, dp, ip]
            lib.oracle_mci_direct.argtypes = [ctypes.c_int, ip, ip, dp, dp, i64, i64, i64,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_int, ip, dp,
                                              i64, ip, i64, dp, ctypes.c_int, ip]
            lib.oracle_interp_functions.argtypes = [ctypes.c_int, ip, ip, dp, dp, i64, i64, i64,
                                                    ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                    dp, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _sys_arrays(systems, P=None, N1=None):
    """systems: list of tuples ('identity',), ('deriv', k), ('hilbert',), ('shift', tau),
    ('custom', table) -- table: complex array of b(n) for n in the band."""
    M = len(systems)
    kind = np.zeros(M, np.int32)
    order = np.ones(M, np.int32)
    tau = np.zeros(M, np.float64)
    custom = None
    for k, s in enumerate(systems):
        kind[k] = SYS_KINDS[s[0]]
        if s[0] == "deriv":
            order[k] = int(s[1]) if len(s) > 1 else 1
        elif s[0] == "shift":
            tau[k] = float(s[1])
        elif s[0] == "custom":
            if custom is None:
                custom = np.zeros((M, M * P, 2), np.float64)
            tab = np.asarray(s[1], np.complex128)
            custom[k, :, 0] = tab.real
            custom[k, :, 1] = tab.imag
    if custom is not None:
        custom = np.ascontiguousarray(custom)
    return M, kind, order, tau, custom


def default_n1(M: int, P: int) -> int:
    """Band start for an even-length band read as {-mu/2 .. mu/2 - 1} (mu = M P)."""
    return -((M * P) // 2)


def q_table(systems, P, N1=None, policy="pinv", rtol=1e-13):
    """Q_r = H_r^{-1} (or pseudo-inverse) for r < P; returns (Q[P, M, M] complex, n_singular).
    Q[r, m, j] = q_{m, j+1}(N1 + r): row m = channel, column j = alias block."""
    M = len(systems)
    N1 = default_n1(M, P) if N1 is None else N1
    M, kind, order, tau, custom = _sys_arrays(systems, P, N1)
    Q = np.zeros((P, M, M, 2), np.float64)
    ns = np.zeros(1, np.int32)
    rc = _load().oracle_q_table(M, _ptr(kind), _ptr(order), _ptr(tau), _ptr(custom), P, N1,
                                POLICIES[policy], rtol, _ptr(Q), _ptr(ns))
    if rc == -3:
        raise OracleError("singular system matrix")
    if rc:
        raise OracleError(f"oracle_q_table failed ({rc})")
    return Q[..., 0] + 1j * Q[..., 1], int(ns[0])


def interp_functions(systems, P, T, N1=None, op="f", policy="pinv", rtol=1e-13, nthreads=0):
    """y_m(2 pi l / T) for l < T (with output operator op applied): complex [M, T]."""
    M = len(systems)
    N1 = default_n1(M, P) if N1 is None else N1
    M, kind, order, tau, custom = _sys_arrays(systems, P, N1)
    Y = np.zeros((M, T, 2), np.float64)
    rc = _load().oracle_interp_functions(M, _ptr(kind), _ptr(order), _ptr(tau), _ptr(custom), P,
                                         N1, T, POLICIES[policy], rtol, OUT_OPS[op], _ptr(Y),
                                         nthreads)
    if rc:
        raise OracleError(f"oracle_interp_functions failed ({rc})")
    return Y[..., 0] + 1j * Y[..., 1]


def mci_direct(systems, g, T, N1=None, outputs=("f",), policy="pinv", rtol=1e-13, idx=None,
               nthreads=0):
    """Direct sum formula.  g: real [batch, M, P] (or [M, P]).
    Returns [batch, n_out, T] (or [batch, n_out, len(idx)] when idx is given)."""
    g = np.asarray(g, np.float64)
    squeeze = g.ndim == 2
    if squeeze:
        g = g[None]
    g = np.ascontiguousarray(g)
    batch, M, P = g.shape
    if M != len(systems):
        raise ValueError("g has %d channels, %d systems given" % (M, len(systems)))
    N1 = default_n1(M, P) if N1 is None else N1
    M, kind, order, tau, custom = _sys_arrays(systems, P, N1)
    ops = np.array([OUT_OPS[o] for o in outputs], np.int32)
    if idx is not None:
        idx = np.ascontiguousarray(np.asarray(idx, np.int64))
        npts = idx.size
    else:
        npts = T
    out = np.zeros((batch, len(ops), npts), np.float64)
    ns = np.zeros(1, np.int32)
    rc = _load().oracle_mci_direct(M, _ptr(kind), _ptr(order), _ptr(tau), _ptr(custom), P, N1, T,
                                   POLICIES[policy], rtol, len(ops), _ptr(ops), _ptr(g), batch,
                                   _ptr(idx), npts if idx is not None else 0, _ptr(out), nthreads,
                                   _ptr(ns))
    if rc == -3:
        raise OracleError("singular system matrix")
    if rc:
        raise OracleError(f"oracle_mci_direct failed ({rc})")
    return out[0] if squeeze else out


# ---------------------------------------------------------------------------
# numpy parts
# ---------------------------------------------------------------------------

def multiplier(system, n, P=None, N1=None):
    """b(n) of one system (Eq. (sysfunction); Examples 2, 3, 5)."""
    n = np.asarray(n)
    kind = system[0]
    if kind == "identity":
        return np.ones(n.shape, np.complex128)
    if kind == "deriv":
        k = int(system[1]) if len(system) > 1 else 1
        return (1j * n.astype(np.float64)) ** k
    if kind == "hilbert":
        return -1j * np.sign(n).astype(np.float64)
    if kind == "shift":
        return np.exp(1j * n.astype(np.float64) * float(system[1]))
    if kind == "custom":
        tab = np.asarray(system[1], np.complex128)
        return tab[n - N1]
    raise ValueError(kind)


def out_operator(op, n):
    n = np.asarray(n, np.float64)
    if op == "f":
        return np.ones(n.shape, np.complex128)
    if op == "hilbert":
        return -1j * np.sign(n)
    if op == "deriv":
        return 1j * n
    raise ValueError(op)


def mci_bruteforce(systems, g, T, N1=None, outputs=("f",), rcond=1e-13):
    """Independent route for tiny P: solve the mu x mu system
    sum_{n in band} a(n) b_m(n) e^{i n t_p} = g_m(t_p)  (Section 3, Eq. (sumformgm)
    before the residue split) in the minimum-norm least-squares sense, then evaluate
    Re sum_n a(n) o(n) e^{i n t_j} on the T-grid."""
    g = np.asarray(g, np.float64)
    M, P = g.shape
    N1 = default_n1(M, P) if N1 is None else N1
    band = np.arange(N1, N1 + M * P)
    tp = 2 * np.pi * np.arange(P) / P
    rows = []
    for m, s in enumerate(systems):
        rows.append(multiplier(s, band, P, N1)[None, :] * np.exp(1j * np.outer(tp, band)))
    A = np.concatenate(rows, axis=0)
    a, *_ = np.linalg.lstsq(A, g.reshape(-1).astype(np.complex128), rcond=rcond)
    tj = 2 * np.pi * np.arange(T) / T
    E = np.exp(1j * np.outer(tj, band))
    return np.stack([(E @ (a * out_operator(o, band))).real for o in outputs])


def truth_from_coeffs(coeffs, band, T, op="f"):
    """Re sum_n c(n) o(n) e^{2 pi i n j / T}, j < T, for given coefficients over a band."""
    band = np.asarray(band)
    j = np.arange(T)
    ph = np.exp(2j * np.pi * np.outer(j, band) / T)
    return (ph @ (np.asarray(coeffs) * out_operator(op, band))).real


def samples_from_coeffs(coeffs, band, systems, P):
    """Channel samples g_m(t_p) = sum_n a(n) b_m(n) e^{i n t_p} (Eq. (sumformgm))."""
    band = np.asarray(band)
    tp = 2 * np.pi * np.arange(P) / P
    E = np.exp(1j * np.outer(tp, band))
    return np.stack([(E @ (np.asarray(coeffs) * multiplier(s, band))).real for s in systems])


def samples_from_coeffs_complex(coeffs, band, systems, P):
    """Complex channel samples g_m(t_p) = sum_n a(n) b_m(n) e^{i n t_p} of a complex signal."""
    band = np.asarray(band)
    tp = 2 * np.pi * np.arange(P) / P
    E = np.exp(1j * np.outer(tp, band))
    return np.stack([E @ (np.asarray(coeffs) * multiplier(s, band)) for s in systems])


def truth_from_coeffs_complex(coeffs, band, T, op="f"):
    """sum_n c(n) o(n) e^{2 pi i n j / T}, j < T (complex signal, no real part taken)."""
    band = np.asarray(band)
    j = np.arange(T)
    ph = np.exp(2j * np.pi * np.outer(j, band) / T)
    return ph @ (np.asarray(coeffs) * out_operator(op, band))


def mci_direct_complex(systems, g, T, N1=None, outputs=("f",), policy="pinv", rtol=1e-13):
    """Sum formula of Theorem MCIeq for complex signals (Examples 4, 5: no real part):
    out(t_j) = (1/P) sum_m sum_p g_m(t_p) y_m(t_j - t_p), y_m from interp_functions.
    g: complex [batch, M, P] (or [M, P]); T a multiple of P (t_j - t_p on the T-grid).
    Returns complex [batch, n_out, T]."""
    g = np.asarray(g, np.complex128)
    squeeze = g.ndim == 2
    if squeeze:
        g = g[None]
    batch, M, P = g.shape
    if T % P:
        raise ValueError("T must be a multiple of P")
    s = T // P
    out = np.zeros((batch, len(outputs), T), np.complex128)
    j = np.arange(T)
    for oi, o in enumerate(outputs):
        Y = interp_functions(systems, P, T, N1=N1, op=o, policy=policy, rtol=rtol)   # [M, T]
        for m in range(M):
            for p in range(P):
                out[:, oi, :] += g[:, m, p:p + 1] * Y[m, (j - p * s) % T][None, :]
    out /= P
    return out[0] if squeeze else out


def mci_bruteforce_complex(systems, g, T, N1=None, outputs=("f",), rcond=1e-13):
    """Tiny-P route for complex signals: minimum-norm least-squares solve of
    sum_{n in band} a(n) b_m(n) e^{i n t_p} = g_m(t_p), then sum_n a(n) o(n) e^{i n t_j}."""
    g = np.asarray(g, np.complex128)
    M, P = g.shape
    N1 = default_n1(M, P) if N1 is None else N1
    band = np.arange(N1, N1 + M * P)
    tp = 2 * np.pi * np.arange(P) / P
    A = np.concatenate([multiplier(sy, band, P, N1)[None, :] * np.exp(1j * np.outer(tp, band))
                        for sy in systems], axis=0)
    a, *_ = np.linalg.lstsq(A, g.reshape(-1), rcond=rcond)
    tj = 2 * np.pi * np.arange(T) / T
    E = np.exp(1j * np.outer(tj, band))
    return np.stack([E @ (a * out_operator(o, band)) for o in outputs])


def fd_channels(x, systems):
    """Derived channels of Section 5.2: identity -> x, first derivative -> three-point centred
    difference (x[p+1] - x[p-1]) / (2h), second derivative -> (x[p+1] - 2x[p] + x[p-1]) / h^2,
    h = 2 pi / P, periodic wrap along the last axis."""
    x = np.asarray(x, np.float64)
    P = x.shape[-1]
    h = 2 * np.pi / P
    xp, xm = np.roll(x, -1, axis=-1), np.roll(x, 1, axis=-1)
    chans = []
    for s in systems:
        if s[0] == "identity":
            chans.append(x)
        elif s[0] == "deriv" and (len(s) == 1 or int(s[1]) == 1):
            chans.append((xp - xm) / (2 * h))
        elif s[0] == "deriv" and int(s[1]) == 2:
            chans.append((xp - 2 * x + xm) / (h * h))
        else:
            raise ValueError("no finite-difference form for %r" % (s,))
    return np.stack(chans, axis=-2)


def blur_factor(n, T, taps, sigma):
    """Multiplier beta(n) = sum_{k=-K..K} w_k e^{-2 pi i n k / T} of the circular convolution
    y(t) = sum_k w_k x(t - 2 pi k / T) on the T-point output grid, where w is the normalised
    Gaussian w_k = exp(-k^2 / (2 sigma^2)) / sum_j exp(-j^2 / (2 sigma^2)), K = taps // 2."""
    K = taps // 2
    k = np.arange(-K, K + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    w /= w.sum()
    n = np.asarray(n, np.float64)
    return np.exp(-2j * np.pi * np.multiply.outer(n, k) / T) @ w


def blur_systems(systems, P, T, taps, sigma, lam=0.0, N1=None):
    """Blur-aware channel model: custom systems b_m(n) gamma(n) over the band.
    lam = 0: gamma = beta, i.e. every measured channel is the blurred system response, and MCI
    then recovers the unblurred signal where the blurred band is recoverable.
    lam > 0 (Wiener-type regularisation, normalised to 1 at n = 0):
    gamma = (|beta|^2 + lam) / ((1 + lam) conj beta), i.e. the reconstruction of the plain
    channel model multiplied by (1 + lam) conj beta / (|beta|^2 + lam)."""
    M = len(systems)
    N1 = default_n1(M, P) if N1 is None else N1
    band = np.arange(N1, N1 + M * P, dtype=np.int64)
    beta = blur_factor(band, T, taps, sigma)
    gamma = beta if lam == 0 else (np.abs(beta) ** 2 + lam) / ((1.0 + lam) * np.conj(beta))
    return [("custom", multiplier(sy, band, P, N1) * gamma) for sy in systems]


def upsample_2d(img, scale, systems, policy="pinv", nthreads=0, blur=None):
    """Separable 2-D MCI of Section 5.2: every row (length w) is interpolated to s*w samples
    from its FD-derived channels, then every column (length h) of that result to s*h.
    Pixel p of a row sits at t_p = 2 pi p / w; output pixel j at 2 pi j / (s w).
    blur = (taps, sigma, lam): each pass uses the blur-aware model of :func:`blur_systems`
    for a taps-tap Gaussian along its axis (the 2-D Gaussian is the outer product)."""
    img = np.asarray(img, np.float64)
    h, w = img.shape

    def model(P, T):
        if blur is None:
            return systems
        return blur_systems(systems, P, T, blur[0], blur[1], blur[2] if len(blur) > 2 else 0.0)

    rows = mci_direct(model(w, scale * w), fd_channels(img, systems), scale * w, policy=policy,
                      nthreads=nthreads)[:, 0, :]                      # h x sw
    cols = mci_direct(model(h, scale * h), fd_channels(rows.T, systems), scale * h,
                      policy=policy, nthreads=nthreads)[:, 0, :]       # sw x sh
    return cols.T


def upsample_2d_mirror(img, scale, systems, policy="pinv", nthreads=0):
    """Separable 2-D MCI with mirror (half-sample-symmetric) image boundaries in place of the
    periodic wrap that the method assumes (Section 2: 2 pi-periodic signals): the h x w image
    is reflected about its edges to 2h x 2w (sample P + n repeats sample P - 1 - n), that
    extension is interpolated as a periodic image by :func:`upsample_2d`, and the s h x s w
    block over the original image is kept."""
    img = np.asarray(img, np.float64)
    h, w = img.shape
    ext = np.pad(img, ((0, h), (0, w)), mode="symmetric")
    return upsample_2d(ext, scale, systems, policy, nthreads)[: scale * h, : scale * w]


def error_bound(coeff_fn, systems, P, N1=None, n_max=None, policy="pinv", rtol=1e-13):
    """Bound of Eq. (errorestimate) on eps(f, N) by the Cauchy-Schwarz inequality:
    bound^2 = sum_{n not in band} |a(n)|^2 + M (sum_m Omega_m) sum_{n not in band} sum_m |a(n) b_m(n)|^2,
    Omega_m = sup over the band of |r_m|^2 (the printed square on Omega read as a slip)."""
    M = len(systems)
    N1 = default_n1(M, P) if N1 is None else N1
    mu = M * P
    Q, _ = q_table(systems, P, N1, policy, rtol)
    omega = np.max(np.abs(Q) ** 2, axis=(0, 2))      # Omega_m: sup over residues r and aliases j
    if n_max is None:
        n_max = 8 * mu
    n = np.arange(-n_max, n_max + 1)
    a = np.asarray(coeff_fn(n), np.complex128)
    outside = (n < N1) | (n >= N1 + mu)
    bm = np.stack([multiplier(s, n) for s in systems])
    s_out = np.sum(np.abs(a[outside]) ** 2)
    s_ab = np.sum(np.abs(a[outside]) ** 2 * np.sum(np.abs(bm[:, outside]) ** 2, axis=0))
    return float(np.sqrt(s_out + M * np.sum(omega) * s_ab))


def averaged_error(coeff_fn, systems, P, N1=None, n_max=None, policy="pinv", rtol=1e-13):
    """Phase-averaged error eps(f, N) of Eq. (averageerror):
    eps^2 = sum_{n not in band} |a(n)|^2
          + sum_{k not in 1..M} sum_{n in I_k} |a(n)|^2 sum_{l=1}^M |sum_m r_m(n + (l-k)P) b_m(n)|^2
    coeff_fn(n) gives a(n); the sums over n outside the band run over |n| <= n_max."""
    M = len(systems)
    N1 = default_n1(M, P) if N1 is None else N1
    mu = M * P
    Q, _ = q_table(systems, P, N1, policy, rtol)
    r = np.zeros((M, mu), np.complex128)         # r_m(N1 + i)
    for m in range(M):
        for j in range(M):
            r[m, j * P:(j + 1) * P] = Q[:, m, j]
    if n_max is None:
        n_max = 8 * mu
    n = np.arange(-n_max, n_max + 1)
    a = np.asarray(coeff_fn(n), np.complex128)
    outside = (n < N1) | (n >= N1 + mu)
    e2 = np.sum(np.abs(a[outside]) ** 2)
    # block index k (1-based) of every n: I_k = {N1 + (k-1)P .. N1 + kP - 1}
    k = np.floor_divide(n - N1, P) + 1
    bm = np.stack([multiplier(s, n) for s in systems])  # M x len(n)
    for i in np.nonzero(outside)[0]:
        tot = 0.0
        for l in range(1, M + 1):
            idx = n[i] + (l - k[i]) * P - N1         # position of n + (l-k)P inside the band
            tot += abs(np.sum(r[:, idx] * bm[:, i])) ** 2
        e2 += abs(a[i]) ** 2 * tot
    return float(np.sqrt(e2))
