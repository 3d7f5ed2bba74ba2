// Phase-averaged approximation error of MCI for signals given by their Fourier
// coefficients (Section 4): Eq. (averageerror)
//     eps^2 = sum_{n outside I} |a(n)|^2 (1 + sum_{l=1..M} |sum_m r_m(n + (l - k) P) b_m(n)|^2),
// k the (1-based) block of n, I_k = {N1 + (k-1) P .. N1 + k P - 1}, and the bound of
// Eq. (errorestimate) from the Cauchy-Schwarz inequality,
//     eps^2 <= sum_{n outside I} |a(n)|^2 + M (sum_m Omega_m) sum_{n outside I} sum_m |a(n) b_m(n)|^2,
// Omega_m = sup_i |r_m(i)|^2.  The inner sum is evaluated as the Hermitian form
// b(n)^H G_r b(n), G_r[m][m'] = sum_l conj(r_m(N1 + l P + r)) r_m'(N1 + l P + r), r the
// residue of n (tabulated by the plan).  One CTA per signal, threads over n, FP64.
#include <cuda_runtime.h>

#include "mci_internal.h"

namespace mci {
namespace {

constexpr int kErrThreads = 256;

__device__ __forceinline__ double2 cmul64(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// b_m(n) of the systems with a closed form (Eq. (sysfunction))
__device__ double2 multiplier(int kind, int order, double tau, int n)
{
    if (kind == MCI_SYS_DERIV) {
        double2 v = make_double2(1.0, 0.0);
        for (int i = 0; i < order; ++i) v = cmul64(v, make_double2(0.0, (double)n));
        return v;
    }
    if (kind == MCI_SYS_HILBERT) return make_double2(0.0, -(double)((n > 0) - (n < 0)));
    if (kind == MCI_SYS_SHIFT) {
        double s, c;
        sincos((double)n * tau, &s, &c);
        return make_double2(c, s);
    }
    return make_double2(1.0, 0.0);
}

__global__ void __launch_bounds__(kErrThreads) averaged_error_kernel(const ErrArgs a)
{
    __shared__ double red[3][kErrThreads / 32];
    const int64_t b = blockIdx.x;
    const int64_t len = 2 * a.n_max + 1;
    const double2* c = a.coeffs + b * len;
    double e2 = 0.0, out2 = 0.0, ab2 = 0.0;
    // 32-bit index arithmetic (the host checks that n_max and the band fit in 2^30)
    const int len32 = (int)len, nmax = (int)a.n_max, n1 = (int)a.N1, mu = (int)a.mu, P = a.P;
    for (int i = threadIdx.x; i < len32; i += blockDim.x) {
        const int n = i - nmax;
        const int d = n - n1;
        if (d >= 0 && d < mu) continue;                      // inside the band
        const double2 an = c[i];
        const double a2 = an.x * an.x + an.y * an.y;
        const int kb = d >= 0 ? d / P : -((-d + P - 1) / P);   // floor(d / P) = k - 1
        const int rr = d - kb * P;                           // position inside its block
        double2 bm[MCI_MAX_CHANNELS];
        double sb2 = 0.0;
        for (int m = 0; m < a.M; ++m) {
            bm[m] = multiplier(a.kind[m], a.order[m], a.tau[m], n);
            sb2 += bm[m].x * bm[m].x + bm[m].y * bm[m].y;
        }
        // tot = b^H G b = sum_m G_mm |b_m|^2 + 2 Re sum_{m < m'} conj(b_m) G_mm' b_m'
        const double2* G = a.G + (int64_t)rr * a.M * a.M;
        double tot = 0.0;
        for (int m = 0; m < a.M; ++m) {
            tot += G[m * a.M + m].x * (bm[m].x * bm[m].x + bm[m].y * bm[m].y);
            for (int m2 = m + 1; m2 < a.M; ++m2) {
                const double2 cb = make_double2(bm[m].x * bm[m2].x + bm[m].y * bm[m2].y,
                                                bm[m].x * bm[m2].y - bm[m].y * bm[m2].x);   // conj(b_m) b_m'
                const double2 g = G[m * a.M + m2];
                tot += 2.0 * (g.x * cb.x - g.y * cb.y);
            }
        }
        e2 += a2 * (1.0 + tot);
        out2 += a2;
        ab2 += a2 * sb2;
    }
    for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_down_sync(0xffffffffu, e2, o);
        out2 += __shfl_down_sync(0xffffffffu, out2, o);
        ab2 += __shfl_down_sync(0xffffffffu, ab2, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = e2;
        red[1][w] = out2;
        red[2][w] = ab2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < kErrThreads / 32; ++i) {
            s0 += red[0][i];
            s1 += red[1][i];
            s2 += red[2][i];
        }
        a.eps[b] = sqrt(s0);
        if (a.bound) a.bound[b] = sqrt(s1 + (double)a.M * a.omega_sum * s2);
    }
}

}  // namespace

int launch_averaged_error(const ErrArgs& a, void* stream)
{
    if (a.batch <= 0) return 0;
    averaged_error_kernel<<<(unsigned)a.batch, kErrThreads, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace mci
