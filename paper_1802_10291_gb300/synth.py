"""Seeded synthetic inputs for multichannel interpolation (MCI).

This module produces signals, their exact channel samples and images.  It holds
none of the interpolation method itself: every value here is the definition of
a test signal (a trigonometric polynomial, a smooth periodic function, a
synthetic image) together with the exact responses of the linear systems the
channels model (identity, derivative, circular Hilbert transform, shift --
Section 2 and Eq. (sysfunction) of Cheng & Kou).  Both the CUDA path's tests
and the CPU oracle's tests draw their inputs from here, so the two sides see
the same numbers.

Recipes (seed = 1802_10291 + workload index unless a test passes its own):

* ``trig_poly``: real trigonometric polynomial over the band {N1 .. N1+mu-1}.
  For n > 0 in the band, Re a(n) and Im a(n) ~ N(0,1)/(1+|n|) independently,
  a(-n) = conj a(n), a(0) ~ N(0,1); a frequency whose mirror image is outside
  the band gets 0 so that f is real.
* ``smooth_periodic``: f(t) = exp(alpha cos(t - phi)), alpha ~ U(0.5, 3),
  phi ~ U(0, 2 pi).  Its Fourier coefficients are alpha-Bessel values
  I_n(alpha) e^{-i n phi}; they are taken from a 256-point FP64 DFT of f, whose
  aliasing error is below 1e-100 for alpha <= 3.
* ``table1_function``: f(t) = Re phi(e^{it}) of Section 5.1 with phi as printed
  there; its Taylor coefficients come from partial fractions.
* ``synthetic_image``: 0.5 + 20 anisotropic Gaussian blobs + 10 straight edges
  + low-passed noise of standard deviation 0.02, clipped to [0, 1].
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1802_10291

_KINDS = ("identity", "deriv", "hilbert", "shift")


def rng_for(index: int, extra: int = 0) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + index, extra])


# ---------------------------------------------------------------------------
# channel responses of a coefficient set (exact definitions, Section 2)
# ---------------------------------------------------------------------------

def response(system, n):
    """Fourier multiplier of a linear system at integer frequencies n:
    identity 1, k-th derivative (i n)^k, circular Hilbert transform -i sgn(n),
    shift by tau e^{i n tau}."""
    n = np.asarray(n, np.float64)
    kind = system[0]
    if kind == "identity":
        return np.ones(n.shape, np.complex128)
    if kind == "deriv":
        k = int(system[1]) if len(system) > 1 else 1
        return (1j * n) ** k
    if kind == "hilbert":
        return -1j * np.sign(n)
    if kind == "shift":
        return np.exp(1j * n * float(system[1]))
    raise ValueError(kind)


def sample_coeffs(coeffs, freqs, npts):
    """Exact values of sum_n c(n) e^{i n t} at t = 2 pi p / npts, p < npts.
    Frequencies are folded modulo npts (exact aliasing) before one inverse FFT."""
    coeffs = np.asarray(coeffs, np.complex128)
    freqs = np.asarray(freqs, np.int64)
    lead = coeffs.shape[:-1]
    L = freqs.size
    if L and np.all(np.diff(freqs) == 1):
        # contiguous range: place at (start mod npts) + i, then sum the npts-long rows
        off = int(np.mod(freqs[0], npts))
        nrow = -(-(off + L) // npts)
        buf = np.zeros(lead + (nrow * npts,), np.complex128)
        buf[..., off:off + L] = coeffs
        bins = buf.reshape(lead + (nrow, npts)).sum(axis=-2)
    else:
        bins = np.zeros(lead + (npts,), np.complex128)
        idx = np.mod(freqs, npts)
        flat = bins.reshape(-1, npts)
        cf = coeffs.reshape(-1, L)
        for r in range(flat.shape[0]):
            np.add.at(flat[r], idx, cf[r])
    return np.fft.ifft(bins, axis=-1) * npts


def channel_samples(coeffs, freqs, systems, P):
    """Real samples g_m(t_p) of every system's response, shape [..., M, P]."""
    chans = [sample_coeffs(np.asarray(coeffs) * response(s, freqs), freqs, P).real
             for s in systems]
    return np.stack(chans, axis=-2)


def response_2d(system, ny, nx):
    """Fourier multiplier of a 2-D linear system at integer frequencies (ny, nx) (rows y,
    columns x): identity 1; partial derivative ('partial', a, b) (i ny)^a (i nx)^b;
    Laplacian -(ny^2 + nx^2); shift ('shift', ty, tx) e^{i (ny ty + nx tx)}; Riesz transform
    ('riesz', axis) -i n_axis / |n| (0 at n = 0), axis 0 = y, 1 = x."""
    ny = np.asarray(ny, np.float64)
    nx = np.asarray(nx, np.float64)
    ny, nx = np.broadcast_arrays(ny, nx)
    kind = system[0]
    if kind == "identity":
        return np.ones(ny.shape, np.complex128)
    if kind == "partial":
        return (1j * ny) ** int(system[1]) * (1j * nx) ** int(system[2])
    if kind == "laplacian":
        return -(ny * ny + nx * nx) + 0j
    if kind == "shift":
        return np.exp(1j * (ny * float(system[1]) + nx * float(system[2])))
    if kind == "riesz":
        r = np.hypot(ny, nx)
        n_ax = ny if int(system[1]) == 0 else nx
        return np.where(r > 0, -1j * n_ax / np.where(r > 0, r, 1.0), 0.0)
    raise ValueError(kind)


def sample_coeffs_2d(coeffs, band_y, band_x, shape):
    """Exact values of sum_n c(n) e^{i (ny t1 + nx t2)} on the grid t = (2 pi l1 / T1,
    2 pi l2 / T2), l < shape = (T1, T2); coeffs [..., len(band_y), len(band_x)].
    Frequencies are folded modulo the grid (exact aliasing) before one inverse FFT."""
    T1, T2 = shape
    coeffs = np.asarray(coeffs, np.complex128)
    lead = coeffs.shape[:-2]
    bins = np.zeros(lead + (T1, T2), np.complex128)
    iy = np.mod(np.asarray(band_y, np.int64), T1)
    ix = np.mod(np.asarray(band_x, np.int64), T2)
    for a, ya in enumerate(iy):
        np.add.at(bins[..., ya, :], (Ellipsis, ix), coeffs[..., a, :])
    return np.fft.ifft2(bins, axes=(-2, -1)) * (T1 * T2)


def channel_samples_2d(coeffs, band_y, band_x, systems, P):
    """Real samples of every 2-D system's response on the P = (P1, P2) grid: [..., M, P1, P2]."""
    ny, nx = np.meshgrid(band_y, band_x, indexing="ij")
    return np.stack([sample_coeffs_2d(np.asarray(coeffs) * response_2d(s, ny, nx), band_y, band_x, P).real
                     for s in systems], axis=-3)


def trig_poly_2d(rng, band_y, band_x, batch=None):
    """Real 2-D trigonometric polynomial over band_y x band_x: for each pair n, -n both in the
    band, Re and Im of a(n) ~ N(0,1) / (1 + |ny| + |nx|) with a(-n) = conj a(n); a(0) ~ N(0,1);
    frequencies whose mirror image is outside the band get 0.  Both bands are contiguous."""
    by, bx = np.asarray(band_y, np.int64), np.asarray(band_x, np.int64)
    lead = () if batch is None else (batch,)
    a = np.zeros(lead + (by.size, bx.size), np.complex128)
    Y, X = np.meshgrid(by, bx, indexing="ij")
    iy, ix = -Y - by[0], -X - bx[0]                      # index of the mirror frequency -n
    has = (iy >= 0) & (iy < by.size) & (ix >= 0) & (ix < bx.size)
    first = has & ((Y > 0) | ((Y == 0) & (X > 0)))       # one of each pair {n, -n}, n != 0
    yy, xx = np.nonzero(first)
    scale = 1.0 / (1.0 + np.abs(Y[yy, xx]) + np.abs(X[yy, xx]))
    z = (rng.standard_normal(lead + (yy.size,)) + 1j * rng.standard_normal(lead + (yy.size,))) * scale
    a[..., yy, xx] = z
    a[..., iy[yy, xx], ix[yy, xx]] = np.conj(z)
    if by[0] <= 0 <= by[-1] and bx[0] <= 0 <= bx[-1]:
        a[..., -by[0], -bx[0]] = rng.standard_normal(lead)
    return a


# ---------------------------------------------------------------------------
# signals
# ---------------------------------------------------------------------------

def band_of(M: int, P: int, N1: int | None = None):
    mu = M * P
    N1 = -(mu // 2) if N1 is None else N1
    return np.arange(N1, N1 + mu, dtype=np.int64)


def trig_poly(rng, band, batch=None):
    """Real trigonometric polynomial coefficients over ``band`` (law above)."""
    band = np.asarray(band, np.int64)
    shape = (band.size,) if batch is None else (batch, band.size)
    a = np.zeros(shape, np.complex128)
    bset = {int(n): i for i, n in enumerate(band)}
    pos = [int(n) for n in band if n > 0 and -n in bset]
    pos_i = np.array([bset[n] for n in pos], np.int64)
    neg_i = np.array([bset[-n] for n in pos], np.int64)
    scale = 1.0 / (1.0 + np.asarray(pos, np.float64))
    lead = () if batch is None else (batch,)
    re = rng.standard_normal(lead + (len(pos),)) * scale
    im = rng.standard_normal(lead + (len(pos),)) * scale
    a[..., pos_i] = re + 1j * im
    a[..., neg_i] = re - 1j * im
    if 0 in bset:
        a[..., bset[0]] = rng.standard_normal(lead)
    return a


def smooth_periodic_coeffs(alpha, phi, nmax=128):
    """Fourier coefficients c(n), |n| <= nmax, of exp(alpha cos(t - phi)) from a
    2*nmax-point FP64 DFT (aliasing below 1e-100 for alpha <= 3)."""
    alpha = np.atleast_1d(np.asarray(alpha, np.float64))
    phi = np.atleast_1d(np.asarray(phi, np.float64))
    K = 2 * nmax
    t = 2 * np.pi * np.arange(K) / K
    vals = np.exp(alpha[:, None] * np.cos(t[None, :] - phi[:, None]))
    c = np.fft.fft(vals, axis=-1) / K
    freqs = np.arange(-nmax, nmax + 1)
    coeffs = c[:, np.mod(freqs, K)]
    coeffs[:, 0] *= 0.5        # n = -nmax and n = nmax share one DFT bin
    coeffs[:, -1] *= 0.5
    return freqs, coeffs


def table1_coeffs(nmax=600):
    """Taylor coefficients c_n, n = 0..nmax, of the Section 5.1 test function
    phi(z) = (0.08 z^2 + 0.06 z^10)/((1.3 - z)(1.5 - z)) + (0.05 z^3 + 0.09 z^10)/((1.2 + z)(1.3 + z)),
    by partial fractions: 1/((u - z)(v - z)) = (1/(v - u)) (1/(u - z) - 1/(v - z))."""
    n = np.arange(nmax + 1)
    s1 = (1 / 0.2) * (1 / 1.3 ** (n + 1) - 1 / 1.5 ** (n + 1))
    s2 = (1 / 0.1) * ((-1.0) ** n / 1.2 ** (n + 1) - (-1.0) ** n / 1.3 ** (n + 1))
    c = np.zeros(nmax + 1)
    for k, w in ((2, 0.08), (10, 0.06)):
        c[k:] += w * s1[: nmax + 1 - k]
    for k, w in ((3, 0.05), (10, 0.09)):
        c[k:] += w * s2[: nmax + 1 - k]
    return c


def table1_fourier(nmax=600):
    """Fourier coefficients a(n), |n| <= nmax, of f(t) = Re phi(e^{it}) (real, even in n)."""
    c = table1_coeffs(nmax)
    freqs = np.arange(-nmax, nmax + 1)
    a = np.where(freqs == 0, c[0], c[np.abs(freqs)] / 2).astype(np.complex128)
    return freqs, a


def signal_batch_1d(rng, P, count, systems, kind="trig", T=None):
    """count signals with P samples per channel.  kind 'trig': bandlimited in the default band
    {-3P/2 .. 3P/2 - 1}-style band of M = len(systems) blocks; 'smooth': exp(alpha cos(t - phi)).
    Returns (g [count, M, P], freqs, coeffs) -- coeffs give the exact signal."""
    M = len(systems)
    if kind == "trig":
        freqs = band_of(M, P)
        coeffs = trig_poly(rng, freqs, count)
    elif kind == "smooth":
        alpha = rng.uniform(0.5, 3.0, count)
        phi = rng.uniform(0.0, 2 * np.pi, count)
        freqs, coeffs = smooth_periodic_coeffs(alpha, phi)
    else:
        raise ValueError(kind)
    g = channel_samples(coeffs, freqs, systems, P)
    return g, freqs, coeffs


def uneven_batch_1d(rng, n_signals, P_choices, systems, smooth_fraction=0.5):
    """Signals whose P is drawn uniformly from P_choices; the first half (by draw order)
    trigonometric polynomials, the rest smooth periodic functions.
    Returns dict with per-signal P, kind and channel samples (list of [M, P] float64)."""
    P_of = rng.choice(np.asarray(P_choices), size=n_signals)
    kind_of = np.where(rng.random(n_signals) < smooth_fraction, "smooth", "trig")
    g = [None] * n_signals
    for P in np.unique(P_of):
        for kind in ("trig", "smooth"):
            sel = np.nonzero((P_of == P) & (kind_of == kind))[0]
            if sel.size == 0:
                continue
            gs, _, _ = signal_batch_1d(rng, int(P), sel.size, systems, kind)
            for i, b in enumerate(sel):
                g[b] = gs[i]
    return {"P": P_of.astype(np.int64), "kind": kind_of, "g": g}


# ---------------------------------------------------------------------------
# images
# ---------------------------------------------------------------------------

def synthetic_image(rng, H, W=None):
    """Grayscale test image in [0, 1] (recipe in the module docstring)."""
    W = H if W is None else W
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    img = np.full((H, W), 0.5)
    side = float(max(H, W))
    for _ in range(20):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        s_major = rng.uniform(side / 64, side / 8)
        s_minor = s_major / rng.uniform(1, 4)
        ang = rng.uniform(0, np.pi)
        amp = rng.uniform(-0.4, 0.4)
        dy, dx = yy - cy, xx - cx
        u = dx * np.cos(ang) + dy * np.sin(ang)
        v = -dx * np.sin(ang) + dy * np.cos(ang)
        img += amp * np.exp(-0.5 * ((u / s_major) ** 2 + (v / s_minor) ** 2))
    for _ in range(10):
        py, px = rng.uniform(0, H), rng.uniform(0, W)
        ang = rng.uniform(0, np.pi)
        step = rng.uniform(0.1, 0.3) * rng.choice([-1.0, 1.0])
        side_of = (xx - px) * np.sin(ang) - (yy - py) * np.cos(ang) > 0
        img += np.where(side_of, step, 0.0)
    noise = rng.standard_normal((H, W))
    F = np.fft.fft2(noise)
    fy = np.abs(np.fft.fftfreq(H))[:, None]
    fx = np.abs(np.fft.fftfreq(W))[None, :]
    F[(fy > 0.125) | (fx > 0.125)] = 0.0          # a quarter of the Nyquist frequency 0.5
    noise = np.fft.ifft2(F).real
    noise *= 0.02 / max(noise.std(), 1e-30)
    return np.clip(img + noise, 0.0, 1.0)


def decimate(img, s):
    """Pure decimation: LR pixel p is HR pixel s p (no blur, offset 0)."""
    return np.ascontiguousarray(np.asarray(img)[..., ::s, ::s])


def gaussian_kernel_1d(taps, sigma):
    """Normalised 1-D Gaussian of ``taps`` (odd) samples at integer offsets -K..K, K = taps // 2:
    w_k = exp(-k^2 / (2 sigma^2)) / sum_j exp(-j^2 / (2 sigma^2)).  The square taps x taps
    Gaussian of the paper's degradation (5 x 5, standard deviation 1.0, Section 5.2) is the
    outer product of two of these."""
    if taps < 1 or taps % 2 == 0 or not sigma > 0:
        raise ValueError("taps must be odd and positive, sigma positive")
    k = np.arange(-(taps // 2), taps // 2 + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    return w / w.sum()


def blur_periodic(x, taps, sigma, axes=(-1,)):
    """Circular convolution of x with the normalised Gaussian along each of ``axes``
    (periodic images, as MCI assumes): y[i] = sum_k w_k x[i - k], indices wrapped."""
    w = gaussian_kernel_1d(taps, sigma)
    K = taps // 2
    y = np.asarray(x, np.float64)
    for ax in axes:
        acc = np.zeros_like(y)
        for j, wk in enumerate(w):
            acc += wk * np.roll(y, j - K, axis=ax)
        y = acc
    return y


def degrade(img, s, taps=5, sigma=1.0):
    """The degradation of the paper's super-resolution experiment (Section 5.2): blur by a
    taps x taps Gaussian (periodic boundary), then keep every s-th pixel (offset 0)."""
    return decimate(blur_periodic(img, taps, sigma, axes=(-2, -1)), s)


def image_params(rng, n, size):
    """Parameters of n synthetic size x size images for the device generator (192 floats per
    image): 20 blobs (cy, cx, 1/s_major, 1/s_minor, angle, amp) with s_major ~ U(size/64, size/8),
    aspect ~ U(1, 4), amp ~ U(-0.4, 0.4); 10 edges (py, px, angle, step +-U(0.1, 0.3));
    8 waves (cycles_y, cycles_x ~ U{-12..12}, phase, amplitude 0.01)."""
    out = np.zeros((n, 192), np.float32)
    for i in range(n):
        q = out[i]
        for k in range(20):
            sm = rng.uniform(size / 64, size / 8)
            sn = sm / rng.uniform(1, 4)
            q[6 * k:6 * k + 6] = [rng.uniform(0, size), rng.uniform(0, size), 1 / sm, 1 / sn,
                                  rng.uniform(0, np.pi), rng.uniform(-0.4, 0.4)]
        for k in range(10):
            q[120 + 4 * k:124 + 4 * k] = [rng.uniform(0, size), rng.uniform(0, size),
                                          rng.uniform(0, np.pi),
                                          rng.uniform(0.1, 0.3) * rng.choice([-1.0, 1.0])]
        for k in range(8):
            q[160 + 4 * k:164 + 4 * k] = [rng.integers(-12, 13), rng.integers(-12, 13),
                                          rng.uniform(0, 2 * np.pi), 0.01]
    return out
