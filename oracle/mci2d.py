"""FP64 CPU oracle for two-dimensional multichannel interpolation.

TEST INFRASTRUCTURE ONLY (as the rest of ``oracle/``): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.  It
shares no code with the CUDA path.

Section 5.2 of Cheng & Kou names, as the first limitation of MCI in image
super-resolution, that rows and columns are treated separately, and proposes a
2-D MCI.  This module is that method written out on the lattice Z^2 with the
definitions of Section 3 carried over axis by axis:

* a 2-D real signal f(t) = sum_n a(n) e^{i n.t}, t in [0, 2 pi)^2, bandlimited to
  the rectangle I = {N1y .. N1y + My P1 - 1} x {N1x .. N1x + Mx P2 - 1};
* M = My Mx channels g_m = h_m * f with Fourier multipliers b_m(n) (Eq.
  (sysfunction) on Z^2), each sampled on the P1 x P2 grid t_p = 2 pi (p1/P1, p2/P2);
* for every residue r = (r1, r2) the M frequencies n_j = n0 + (jy P1, jx P2),
  j = jy Mx + jx, of I that alias onto one DFT bin give the M x M matrix
  H_r[j][k] = b_k(n_j) (Eq. (defH)); Q_r = H_r^{-1} (or its pseudo-inverse, Remark
  (aequal0)) gives r_m(n_j) = Q_r[m][j] (Eq. (defrm));
* y_m(t) = sum_{n in I} r_m(n) e^{i n.t} (Eq. (ym)) and the sum formula of Theorem
  (MCIeq): f(t) = (1 / (P1 P2)) sum_m sum_p g_m(t_p) y_m(t - t_p); with real
  channels the real part is taken (the 1-D convention for an asymmetric band).

Systems are tuples: ('identity',), ('partial', a, b) = (i ny)^a (i nx)^b,
('laplacian',) = -(ny^2 + nx^2), ('shift', ty, tx) = e^{i (ny ty + nx tx)},
('riesz', axis) = -i n_axis / |n| (0 at n = 0).
"""
from __future__ import annotations

import numpy as np


def multiplier(system, ny, nx):
    """b(n) of one 2-D system at frequencies (ny, nx)."""
    ny = np.asarray(ny, np.float64)
    nx = np.asarray(nx, np.float64)
    ny, nx = np.broadcast_arrays(ny, nx)
    kind = system[0]
    if kind == "identity":
        return np.ones(ny.shape, np.complex128)
    if kind == "partial":
        return (1j * ny) ** int(system[1]) * (1j * nx) ** int(system[2])
    if kind == "laplacian":
        return -(ny ** 2 + nx ** 2) + 0j
    if kind == "shift":
        return np.exp(1j * ny * float(system[1])) * np.exp(1j * nx * float(system[2]))
    if kind == "riesz":
        norm = np.sqrt(ny ** 2 + nx ** 2)
        comp = ny if int(system[1]) == 0 else nx
        out = np.zeros(ny.shape, np.complex128)
        nz = norm > 0
        out[nz] = -1j * comp[nz] / norm[nz]
        return out
    raise ValueError(kind)


def default_n1(grid, P):
    """Band start per axis: -floor(M_axis P_axis / 2)."""
    return tuple(-((m * p) // 2) for m, p in zip(grid, P))


def band(grid, P, N1=None):
    N1 = default_n1(grid, P) if N1 is None else N1
    return (np.arange(N1[0], N1[0] + grid[0] * P[0], dtype=np.int64),
            np.arange(N1[1], N1[1] + grid[1] * P[1], dtype=np.int64))


def q_table(systems, grid, P, N1=None, policy="pinv", rtol=1e-13):
    """Q[r1, r2, m, j] for every residue (Eq. (defH) inverted per residue) and the number of
    singular residues (sigma_min < rtol sigma_max)."""
    My, Mx = grid
    P1, P2 = P
    M = My * Mx
    if len(systems) != M:
        raise ValueError("need My * Mx systems")
    N1 = default_n1(grid, P) if N1 is None else N1
    Q = np.zeros((P1, P2, M, M), np.complex128)
    n_sing = 0
    for r1 in range(P1):
        for r2 in range(P2):
            ny = np.array([N1[0] + r1 + (j // Mx) * P1 for j in range(M)])
            nx = np.array([N1[1] + r2 + (j % Mx) * P2 for j in range(M)])
            H = np.stack([multiplier(s, ny, nx) for s in systems], axis=1)   # H[j][k]
            sv = np.linalg.svd(H, compute_uv=False)
            if not sv[0] > 0 or sv[-1] < rtol * sv[0]:
                n_sing += 1
                if policy == "error":
                    raise np.linalg.LinAlgError("singular system matrix")
                if policy == "zero" or not sv[0] > 0:
                    continue
                Q[r1, r2] = np.linalg.pinv(H, rcond=rtol)
            else:
                Q[r1, r2] = np.linalg.inv(H)
    return Q, n_sing


def interp_functions(systems, grid, P, T, N1=None, policy="pinv", rtol=1e-13):
    """y_m(2 pi l1 / T1, 2 pi l2 / T2) for l < T: complex [M, T1, T2] (Eq. (ym) on Z^2)."""
    My, Mx = grid
    P1, P2 = P
    T1, T2 = T
    M = My * Mx
    N1 = default_n1(grid, P) if N1 is None else N1
    Q, _ = q_table(systems, grid, P, N1, policy, rtol)
    by, bx = band(grid, P, N1)
    # r_m over the band: r_m(N1y + r1 + jy P1, N1x + r2 + jx P2) = Q[r1, r2, m, jy Mx + jx]
    R = np.zeros((M, by.size, bx.size), np.complex128)
    for j in range(M):
        jy, jx = divmod(j, Mx)
        R[:, jy * P1:(jy + 1) * P1, jx * P2:(jx + 1) * P2] = np.moveaxis(Q[:, :, :, j], 2, 0)
    # e^{i n t} with the phase n l reduced modulo T in integers
    Ey = np.exp(2j * np.pi * np.mod(np.outer(np.arange(T1), by), T1) / T1)    # T1 x |by|
    Ex = np.exp(2j * np.pi * np.mod(np.outer(np.arange(T2), bx), T2) / T2)    # T2 x |bx|
    return np.stack([Ey @ R[m] @ Ex.T for m in range(M)])


def mci2_direct(systems, grid, g, T, N1=None, policy="pinv", rtol=1e-13):
    """Sum formula of Theorem (MCIeq) on Z^2.  g: real [batch, M, P1, P2] (or [M, P1, P2]);
    returns the real part of the interpolant on the T1 x T2 grid, [batch, T1, T2]."""
    g = np.asarray(g, np.float64)
    squeeze = g.ndim == 3
    if squeeze:
        g = g[None]
    batch, M, P1, P2 = g.shape
    T1, T2 = T
    if T1 % P1 or T2 % P2:
        raise ValueError("T must be a multiple of P per axis")
    s1, s2 = T1 // P1, T2 // P2
    Y = interp_functions(systems, grid, (P1, P2), T, N1, policy, rtol)
    out = np.zeros((batch, T1, T2), np.complex128)
    for m in range(M):
        for p1 in range(P1):
            for p2 in range(P2):
                # y_m(t_j - t_p): shift the tabulated y_m by (s1 p1, s2 p2) grid points
                out += g[:, m, p1, p2, None, None] * np.roll(Y[m], (s1 * p1, s2 * p2), axis=(0, 1))[None]
    out /= P1 * P2
    return out.real[0] if squeeze else out.real


def mci2_bruteforce(systems, grid, g, T, N1=None, rcond=1e-13):
    """Second route for tiny sizes: solve the sampling equations
    sum_{n in I} a(n) b_m(n) e^{i n.t_p} = g_m(t_p) for all m, p (minimum-norm least squares),
    then evaluate Re sum_n a(n) e^{i n.t} on the T grid.  g: real [M, P1, P2]."""
    g = np.asarray(g, np.float64)
    M, P1, P2 = g.shape
    by, bx = band(grid, (P1, P2), N1)
    ny, nx = np.meshgrid(by, bx, indexing="ij")
    ny, nx = ny.ravel(), nx.ravel()
    p1, p2 = np.meshgrid(np.arange(P1), np.arange(P2), indexing="ij")
    t1 = 2 * np.pi * p1.ravel() / P1
    t2 = 2 * np.pi * p2.ravel() / P2
    E = np.exp(1j * (np.outer(t1, ny) + np.outer(t2, nx)))                  # samples x band
    A = np.concatenate([E * multiplier(s, ny, nx)[None, :] for s in systems], axis=0)
    a, *_ = np.linalg.lstsq(A, g.reshape(-1).astype(np.complex128), rcond=rcond)
    T1, T2 = T
    l1, l2 = np.meshgrid(np.arange(T1), np.arange(T2), indexing="ij")
    Et = np.exp(1j * (np.outer(2 * np.pi * l1.ravel() / T1, ny) + np.outer(2 * np.pi * l2.ravel() / T2, nx)))
    return (Et @ a).real.reshape(T1, T2)
