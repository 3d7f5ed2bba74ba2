// Internal interface between the 2-D MCI plan code (mci2d_host.cpp) and its kernels (mci2d.cu).
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

#include "mci2d.h"

namespace mci2 {

constexpr int kThreads2 = 256;
constexpr int kSmemMax = 227 * 1024;   // dynamic + static shared memory per CTA

struct Dims2 {
    int M, My, Mx, P1, P2, H2, T1, T2, s1, s2;
    int N1y_mod, N1x_mod;   // N1 reduced modulo P1, P2 (non-negative)
    int G1, G3, chunk;      // rows per rowfwd CTA, output rows per rowinv CTA, phases per col pass
    int lgG1, lgG3;         // log2 of G1, G3 (powers of two)
};

// Device tables and workspace of a plan (precision-typed complex arrays).
struct Tables {
    const void* Qt;       // [r2][r1][m][j]: Q_r / (2 P1 P2)
    const void* Fy;       // [u1][r1]: e^{2 pi i (N1y + r1) u1 / T1}
    const void* Oy;       // [u1][jy]: e^{2 pi i jy u1 / s1} (alias block jy of the y axis)
    const void* Fx;       // [u2][jx][r2]: e^{2 pi i n_x u2 / T2}
    const void* roots1;   // e^{-2 pi i k / P1}
    const void* roots2;   // e^{-2 pi i k / P2}
    void* X;              // [b][m][k2][p1] row half spectra
    void* Zw;             // [b][u2][k2][j1] column-inverted sub-grid spectra
};

// Opt the three kernels of one precision into their dynamic shared memory sizes.
mci_status set_smem(int precision, size_t smem1, size_t smem2, size_t smem3);

// The three passes for batch images on stream st.
mci_status launch(int precision, const Dims2& d, const Tables& t, size_t smem1, size_t smem2, size_t smem3,
                  const void* in, void* out, int64_t batch, cudaStream_t st);

}  // namespace mci2
