/*
 * mci2d.h -- two-dimensional multichannel interpolation (MCI) of real images.
 *
 * Section 5.2 of Cheng & Kou names, as the first limitation of MCI for images,
 * that rows and columns are interpolated separately, and proposes a 2-D MCI.
 * This interface is the method of Section 3 carried to Z^2 axis by axis:
 *
 *   - a real signal f(t) = sum_n a(n) e^{i (ny t1 + nx t2)}, t in [0, 2 pi)^2,
 *     bandlimited to the rectangle I = {N1y .. N1y + My P1 - 1} x
 *     {N1x .. N1x + Mx P2 - 1};
 *   - M = My * Mx channels g_m with 2-D Fourier multipliers b_m(n) (Eq.
 *     (sysfunction) on Z^2), each sampled on the P1 x P2 grid
 *     t_p = 2 pi (p1 / P1, p2 / P2);
 *   - per 2-D residue the M frequencies n_j = n0 + (jy P1, jx P2), j = jy Mx + jx,
 *     give H_r[j][k] = b_k(n_j) (Eq. (defH)); its inverse (pseudo-inverse where
 *     singular, Remark (aequal0)) solves for a(n_j) from the channels' DFT bins
 *     (Eq. (matrixeqn1)), and the interpolant is evaluated on the T1 x T2 grid
 *     t_j = 2 pi (j1 / T1, j2 / T2) by inverse DFTs (Eq. (DFTexpression)).  As in
 *     the 1-D real mode the real part is returned.
 *
 * With a product channel set, e.g. {1, i nx} x {1, i ny} (f, f_x, f_y, f_xy), the
 * result equals 1-D MCI along x then along y with the real part taken once at the
 * end; other sets (shifts, Riesz transforms, mixed derivatives) are not separable.
 *
 * Computation (all in this library's kernels): row FFTs of every channel (two real
 * rows per complex FFT), then per column of the half spectrum the column FFTs, the
 * per-residue solve and the T1/P1 x T2/P2 output phases with their inverse column
 * FFTs, then inverse real row FFTs per output row and phase, interleaved.
 *
 * Buffers are DEVICE pointers unless stated; calls are stream-ordered; status codes
 * as in mci.h.
 */
#ifndef MCI2D_H
#define MCI2D_H

#include "mci.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mci2_plan_s* mci2_plan_t;

/* 2-D linear systems: Fourier multiplier b(ny, nx). */
enum {
    MCI2_SYS_IDENTITY = 0,  /* 1                                                  */
    MCI2_SYS_PARTIAL = 1,   /* (i ny)^order_y (i nx)^order_x, orders >= 0        */
    MCI2_SYS_LAPLACIAN = 2, /* -(ny^2 + nx^2)                                     */
    MCI2_SYS_SHIFT = 3,     /* e^{i (ny tau_y + nx tau_x)}                         */
    MCI2_SYS_RIESZ = 4      /* -i n_a / |n| (0 at n = 0), a = y if order_y == 0 else x
                               (the 2-D counterpart of the Hilbert transform)     */
};

typedef struct {
    int kind;               /* MCI2_SYS_*                                          */
    int order_y, order_x;   /* PARTIAL: derivative orders; RIESZ: order_y = axis  */
    double tau_y, tau_x;    /* SHIFT                                               */
} mci2_system;

typedef struct {
    int My, Mx;             /* alias blocks along y (rows) and x (columns); M = My * Mx
                               channels, 1 .. 8                                     */
    const mci2_system* sys; /* M systems (host, read during mci2_plan only)         */
    int P1, P2;             /* samples per channel along y and x: each 2^a or 3 * 2^a,
                               4 .. 1024                                            */
    int T1, T2;             /* output grid: positive multiples of P1, P2 (T / P <= 16) */
    const int64_t* N1;      /* host {N1y, N1x}, or NULL for {-floor(My P1 / 2),
                               -floor(Mx P2 / 2)}                                   */
    int precision;          /* MCI_FP32 or MCI_FP64: type of samples and outputs     */
    int singular_policy;    /* MCI_SINGULAR_* as in mci.h                           */
    double singular_rtol;   /* <= 0 selects 1e-13                                   */
    int64_t max_batch;      /* most images per mci2_interp call (>= 1)              */
} mci2_desc;

/* Build a plan: FP64 per-residue inverses on the host (P1 * P2 Jacobi SVDs of M x M),
 * stored with the output phase factors and FFT roots in device memory, plus a workspace
 * for max_batch images (mci2_plan_info reports its size).  Synchronises.
 * Errors: MCI_ERR_INVALID_ARG (null pointers, bad enums or counts),
 * MCI_ERR_UNSUPPORTED_SIZE (P, T outside the ranges above, or a kernel's shared memory
 * above the per-CTA limit), MCI_ERR_SINGULAR (singular H_r under MCI_SINGULAR_ERROR),
 * MCI_ERR_OOM, MCI_ERR_CUDA. */
mci_status mci2_plan(mci2_plan_t* plan, const mci2_desc* d, mci_stream_t stream);

/* Interpolate batch images: in [batch][M][P1][P2] (channel planes of each image,
 * row-major), out [batch][T1][T2], both of the plan's precision, device, 16-byte
 * aligned.  0 <= batch <= max_batch (batch 0 is a no-op).  Asynchronous. */
mci_status mci2_interp(mci2_plan_t plan, const void* in, void* out, int64_t batch, mci_stream_t stream);

/* Singular residues, largest sigma_max / sigma_min over the others, workspace bytes
 * (any pointer may be NULL). */
mci_status mci2_plan_info(mci2_plan_t plan, int* n_singular, double* max_cond, int64_t* workspace_bytes);

/* Free the plan (NULL is a no-op); synchronises. */
mci_status mci2_destroy(mci2_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* MCI2D_H */
