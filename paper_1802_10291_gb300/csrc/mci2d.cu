// Two-dimensional multichannel interpolation (include/mci2d.h): plan construction in
// FP64 on the host and three kernels.
//
//   mci2_rowfwd   forward FFT of every channel row (two real rows per complex FFT),
//                 half spectrum stored column-major per channel: X[b][m][k2][p1]
//   mci2_col      per half-spectrum column k2: forward column FFTs of the M channels,
//                 per-residue solve (Eq. (matrixeqn1) on Z^2) for the M aliases of bin k
//                 and of bin -k, then for every output phase (u1, u2) the Hermitian-
//                 symmetrised sub-grid spectrum and its inverse column FFT:
//                 Z[b][u2][k2][j1], j1 = s1 p1 + u1
//   mci2_rowinv   per output row j1 and phase u2: inverse real FFT over k2 (two real
//                 outputs per complex FFT), interleaved into out[b][j1][s2 p2 + u2]
//
// The FFTs are shared-memory Stockham transforms of runtime length (radix 4, then 2,
// then one radix-3 pass), all threads of the CTA working on several sequences.
#include <cuda_runtime.h>

#include "mci2d_internal.h"

using mci2::Dims2;
using mci2::kThreads2;

namespace {

template <typename R>
struct alignas(2 * sizeof(R)) zc {
    R re, im;
};

template <typename R>
__device__ __forceinline__ zc<R> zmul(zc<R> a, zc<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ zc<R> zadd(zc<R> a, zc<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ zc<R> zsub(zc<R> a, zc<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ zc<R> zconj(zc<R> a) { return {a.re, -a.im}; }
// a * (+i) when s > 0, a * (-i) when s < 0
template <typename R>
__device__ __forceinline__ zc<R> zrot(zc<R> a, bool plus_i) { return plus_i ? zc<R>{-a.im, a.re} : zc<R>{a.im, -a.re}; }

// n / d for n d < 2^32 by a multiply-high with m = ceil(2^32 / d) (d = 1 passes n through).
struct FDiv {
    unsigned d, m;
};
__device__ __forceinline__ FDiv fdiv_make(unsigned d)
{
    return {d, d == 1 ? 0u : 0xFFFFFFFFu / d + 1u};   // = ceil(2^32 / d) for d > 1
}
__device__ __forceinline__ int fdiv(int n, FDiv f) { return f.d == 1 ? n : (int)__umulhi((unsigned)n, f.m); }

// One radix-RAD Stockham pass over `count` sequences of length N (stride N): butterfly i of a
// sequence reads x_j = src[i + j N/RAD], multiplies by w^{j k} (k = i mod p, w = e^{-+2 pi i /
// (p RAD)}), and writes the RAD-point DFT to dst[(i / p) p RAD + k + j p].  p is a power of two
// (2^lp).  N / RAD = 2^nb_shift * (nb_three ? 3 : 1).
template <typename R, int RAD>
__device__ __forceinline__ void fft_pass(const zc<R>* src, zc<R>* dst, int N, int count, int ld, int p, int lp,
                                         int nb_shift, bool nb_three, const zc<R>* __restrict__ roots, bool inv)
{
    const int nb = N / RAD, step = N / (p * RAD);
    for (int idx = threadIdx.x; idx < count * nb; idx += blockDim.x) {
        // idx / nb: a shift, then floor(x / 3) = (x * 0xAAAAAAAB) >> 33 for 32-bit x
        const int hi = idx >> nb_shift;
        const int sq = nb_three ? (int)(__umulhi((unsigned)hi, 0xAAAAAAABu) >> 1) : hi;
        const int i = idx - sq * nb;
        const int k = i & (p - 1);
        const zc<R>* s = src + sq * ld + i;
        zc<R>* d = dst + sq * ld + ((i >> lp) * p * RAD + k);
        zc<R> x[RAD];
#pragma unroll
        for (int j = 0; j < RAD; ++j) x[j] = s[j * nb];
        if (k > 0) {
#pragma unroll
            for (int j = 1; j < RAD; ++j) {
                zc<R> w = roots[j * k * step];
                if (inv) w.im = -w.im;
                x[j] = zmul(x[j], w);
            }
        }
        if constexpr (RAD == 4) {
            const zc<R> t0 = zadd(x[0], x[2]), t1 = zsub(x[0], x[2]);
            const zc<R> t2 = zadd(x[1], x[3]), t3 = zsub(x[1], x[3]);
            // forward: X1 = t1 - i t3, X3 = t1 + i t3; inverse the other way round
            const zc<R> it3 = zrot(t3, inv);
            d[0] = zadd(t0, t2);
            d[p] = zadd(t1, it3);
            d[2 * p] = zsub(t0, t2);
            d[3 * p] = zsub(t1, it3);
        } else if constexpr (RAD == 2) {
            d[0] = zadd(x[0], x[1]);
            d[p] = zsub(x[0], x[1]);
        } else {
            const R h = (R)0.86602540378443864676;   // sin(2 pi / 3)
            const zc<R> t1 = zadd(x[1], x[2]), t2 = zsub(x[1], x[2]);
            const zc<R> m = {x[0].re - (R)0.5 * t1.re, x[0].im - (R)0.5 * t1.im};
            const zc<R> it2 = zrot(zc<R>{h * t2.re, h * t2.im}, inv);   // forward: -i h t2
            d[0] = zadd(x[0], t1);
            d[p] = zadd(m, it2);
            d[2 * p] = zsub(m, it2);
        }
    }
}

// Stockham FFT of `count` sequences of length N stored at stride ld (>= N; N + 1 keeps
// accesses that run across sequences off a single bank) in a; b is scratch of the same size.  Forward: X_k = sum_p x_p e^{-2 pi i k p / N}; inverse: the
// conjugate kernel, unnormalised.  roots[k] = e^{-2 pi i k / N}.  Radix 4 while 4 | rem, then
// 2, then 3, so the stride p before every pass is a power of two.  Returns the buffer holding
// the result.  All threads of the block must call it, after the input is visible to all.
template <typename R>
__device__ zc<R>* fft_seq(zc<R>* a, zc<R>* b, int N, int count, int ld, const zc<R>* __restrict__ roots, bool inv)
{
    zc<R>* src = a;
    zc<R>* dst = b;
    const bool three = N % 3 == 0;
    const int a2 = 31 - __clz(three ? N / 3 : N);   // N = 2^a2 (3 if three)
    int p = 1, lp = 0, rem = N;
    while (rem > 1) {
        const int r = rem % 4 == 0 ? 4 : (rem % 2 == 0 ? 2 : 3);
        if (r == 4) fft_pass<R, 4>(src, dst, N, count, ld, p, lp, a2 - 2, three, roots, inv);
        else if (r == 2) fft_pass<R, 2>(src, dst, N, count, ld, p, lp, a2 - 1, three, roots, inv);
        else fft_pass<R, 3>(src, dst, N, count, ld, p, lp, a2, false, roots, inv);
        __syncthreads();
        zc<R>* t = src;
        src = dst;
        dst = t;
        p *= r;
        lp += (r == 4) ? 2 : (r == 2 ? 1 : 0);
        rem /= r;
    }
    return src;
}

// -------------------------------------------------------------------------------------------
// pass 1: row FFTs of every channel plane, two real rows per complex FFT
template <typename R>
__global__ void __launch_bounds__(kThreads2) mci2_rowfwd(const R* __restrict__ in, zc<R>* __restrict__ X,
                                                         const zc<R>* __restrict__ roots2, const Dims2 d)
{
    extern __shared__ __align__(16) unsigned char smem2d[];
    const int G = d.G1, P2 = d.P2, H2 = d.H2, P1 = d.P1;
    zc<R>* A = reinterpret_cast<zc<R>*>(smem2d);
    const int ld = P2 + 1;
    zc<R>* B = A + (size_t)(G / 2) * ld;
    zc<R>* tw = B + (size_t)(G / 2) * ld;   // P2 FFT roots
    for (int p = threadIdx.x; p < P2; p += blockDim.x) tw[p] = roots2[p];
    const int b = blockIdx.z, m = blockIdx.y, p0 = blockIdx.x * G;
    const R* src = in + ((int64_t)b * d.M + m) * P1 * P2 + (int64_t)p0 * P2;
    const FDiv fp2 = fdiv_make(P2);
    for (int idx = threadIdx.x; idx < (G / 2) * P2; idx += blockDim.x) {
        const int q = fdiv(idx, fp2), c = idx - q * P2;
        A[q * ld + c] = zc<R>{src[(int64_t)(2 * q) * P2 + c], src[(int64_t)(2 * q + 1) * P2 + c]};
    }
    __syncthreads();
    const zc<R>* res = fft_seq(A, B, P2, G / 2, ld, tw, false);
    zc<R>* dst = X + ((int64_t)b * d.M + m) * (H2 + 1) * P1 + p0;
    for (int idx = threadIdx.x; idx < (H2 + 1) * G; idx += blockDim.x) {
        const int k2 = idx >> d.lgG1, g = idx & (G - 1);
        const zc<R>* seq = res + (size_t)(g >> 1) * ld;
        const zc<R> z = seq[k2];
        const zc<R> zc_ = zconj(seq[k2 == 0 ? 0 : P2 - k2]);
        // even row: (z + conj z(-k)) / 2; odd row: (z - conj z(-k)) / (2 i)
        const zc<R> v = (g & 1) ? zc<R>{(R)0.5 * (z.im - zc_.im), (R)-0.5 * (z.re - zc_.re)}
                                : zc<R>{(R)0.5 * (z.re + zc_.re), (R)0.5 * (z.im + zc_.im)};
        dst[(int64_t)k2 * P1 + g] = v;
    }
}

// -------------------------------------------------------------------------------------------
// pass 2: column FFTs, per-residue solve, output phases, inverse column FFTs
// (one instantiation per channel count M, so the per-bin M x M products unroll fully)
template <typename R, int M>
__global__ void __launch_bounds__(kThreads2, sizeof(R) == 4 ? 4 : 2)
    mci2_col(const zc<R>* __restrict__ X, zc<R>* __restrict__ Z, const zc<R>* __restrict__ Qt,
             const zc<R>* __restrict__ Fy, const zc<R>* __restrict__ Oy, const zc<R>* __restrict__ Fx,
             const zc<R>* __restrict__ roots1, const Dims2 d)
{
    extern __shared__ __align__(16) unsigned char smem2d[];
    const int P1 = d.P1, P2 = d.P2, H2 = d.H2, Mx = d.Mx, s1 = d.s1;
    const int nph = s1 * d.s2;                           // output phases q = u2 s1 + u1
    const int k2 = blockIdx.x, b = blockIdx.y;
    const int ld = P1 + 1;                               // sequence stride in shared memory
    zc<R>* bufA = reinterpret_cast<zc<R>*>(smem2d);     // M sequences
    zc<R>* bufB = bufA + (size_t)M * ld;                 // M sequences
    zc<R>* Yb = bufB + (size_t)M * ld;                   // chunk sequences
    zc<R>* Sb = Yb + (size_t)d.chunk * ld;               // chunk sequences
    zc<R>* tw = Sb + (size_t)d.chunk * ld;               // P1 FFT roots
    // phase factors of the batch per (phase, alias j): e^{2 pi i (jy u1 / s1 + n_x(j) u2 / T2)}
    // for bin k (ph) and for bin -k (phn); the r1-dependent part Fy[u1][r1] is applied per bin
    zc<R>* ph = tw + P1;                                 // chunk * M
    zc<R>* phn = ph + (size_t)d.chunk * M;               // chunk * M

    const zc<R>* src = X + (int64_t)b * M * (H2 + 1) * P1 + (int64_t)k2 * P1;
#pragma unroll
    for (int m = 0; m < M; ++m)
        for (int p = threadIdx.x; p < P1; p += blockDim.x) bufA[m * ld + p] = src[(int64_t)m * (H2 + 1) * P1 + p];
    for (int p = threadIdx.x; p < P1; p += blockDim.x) tw[p] = roots1[p];
    // residues of the column: r2 for k2, r2n for -k2
    int r2 = k2 - d.N1x_mod;
    if (r2 < 0) r2 += P2;
    int r2n = (k2 == 0 ? 0 : P2 - k2) - d.N1x_mod;
    if (r2n < 0) r2n += P2;
    __syncthreads();
    zc<R>* Xs = fft_seq(bufA, bufB, P1, M, ld, tw, false);
    zc<R>* As = Xs == bufA ? bufB : bufA;   // A' (aliases of -k) go to the other buffer
    // per bin k1: A_j(k) = sum_m X_m(k) Q_r(k)[m][j] (in place over X), A'_j(k) = sum_m conj X_m(k) Q_r(-k)[m][j];
    // Q is stored [r2][m][j][r1]: consecutive bins read consecutive entries
    const zc<R>* Qc = Qt + (int64_t)r2 * M * M * P1;
    const zc<R>* Qn = Qt + (int64_t)r2n * M * M * P1;
    for (int k1 = threadIdx.x; k1 < P1; k1 += blockDim.x) {
        zc<R> x[M];
#pragma unroll
        for (int m = 0; m < M; ++m) x[m] = Xs[m * ld + k1];
        int r1 = k1 - d.N1y_mod;
        if (r1 < 0) r1 += P1;
        int r1n = (k1 == 0 ? 0 : P1 - k1) - d.N1y_mod;
        if (r1n < 0) r1n += P1;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            zc<R> a{0, 0}, an{0, 0};
#pragma unroll
            for (int m = 0; m < M; ++m) {
                a = zadd(a, zmul(x[m], Qc[(int64_t)(m * M + j) * P1 + r1]));
                an = zadd(an, zmul(zconj(x[m]), Qn[(int64_t)(m * M + j) * P1 + r1n]));
            }
            Xs[j * ld + k1] = a;
            As[j * ld + k1] = an;
        }
    }
    zc<R>* out = Z + (int64_t)b * d.s2 * (H2 + 1) * d.T1 + (int64_t)k2 * d.T1;
    for (int q0 = 0; q0 < nph; q0 += d.chunk) {
        const int cnt = min(d.chunk, nph - q0);
        for (int idx = threadIdx.x; idx < cnt * M; idx += blockDim.x) {
            const int c = idx / M, j = idx - c * M;
            const int q = q0 + c, u2 = q / s1, u1 = q - u2 * s1;
            const int jy = j / Mx, jx = j - jy * Mx;
            const zc<R> oy = Oy[u1 * d.My + jy];
            ph[idx] = zmul(oy, Fx[((int64_t)u2 * Mx + jx) * P2 + r2]);
            phn[idx] = zmul(oy, Fx[((int64_t)u2 * Mx + jx) * P2 + r2n]);
        }
        __syncthreads();   // also orders the A, A' writes before the first batch
        // Y_q(k1) = Fy[u1][r1] sum_j A_j ph_j + conj(Fy[u1][r1n] sum_j A'_j phn_j)
        // (1 / (2 P1 P2) is folded into Q)
        for (int c = 0; c < cnt; ++c) {
            const int u1 = (q0 + c) % s1;
            const zc<R>* f = Fy + (int64_t)u1 * P1;
            const zc<R>* pc = ph + c * M;
            const zc<R>* pn = phn + c * M;
            for (int k1 = threadIdx.x; k1 < P1; k1 += blockDim.x) {
                int r1 = k1 - d.N1y_mod;
                if (r1 < 0) r1 += P1;
                int r1n = (k1 == 0 ? 0 : P1 - k1) - d.N1y_mod;
                if (r1n < 0) r1n += P1;
                zc<R> y{0, 0}, yn{0, 0};
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    y = zadd(y, zmul(Xs[j * ld + k1], pc[j]));
                    yn = zadd(yn, zmul(As[j * ld + k1], pn[j]));
                }
                Yb[c * ld + k1] = zadd(zmul(f[r1], y), zconj(zmul(f[r1n], yn)));
            }
        }
        __syncthreads();
        const zc<R>* ys = fft_seq(Yb, Sb, P1, cnt, ld, tw, true);
        // j1 = s1 p1 + u1 of phase column u2; within one u2, consecutive threads take consecutive j1
        const FDiv fcnt = fdiv_make(cnt);
        for (int idx = threadIdx.x; idx < cnt * P1; idx += blockDim.x) {
            const int p1 = fdiv(idx, fcnt), c = idx - p1 * cnt;
            const int q = q0 + c, u2 = q / s1, u1 = q - u2 * s1;
            out[((int64_t)u2 * (H2 + 1)) * d.T1 + (int64_t)p1 * s1 + u1] = ys[(size_t)c * ld + p1];
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------------------------------
// pass 3: inverse real FFTs along rows, two real outputs (rows j1, j1 + 1) per complex FFT
template <typename R>
__global__ void __launch_bounds__(kThreads2) mci2_rowinv(const zc<R>* __restrict__ Z, R* __restrict__ out,
                                                         const zc<R>* __restrict__ roots2, const Dims2 d)
{
    extern __shared__ __align__(16) unsigned char smem2d[];
    const int G = d.G3, P2 = d.P2, H2 = d.H2, T1 = d.T1, s2 = d.s2;
    const int nseq = s2 * (G / 2);
    const int ld = P2 + 1;
    zc<R>* A = reinterpret_cast<zc<R>*>(smem2d);
    zc<R>* B = A + (size_t)nseq * ld;
    zc<R>* tw = B + (size_t)nseq * ld;   // P2 FFT roots
    for (int p = threadIdx.x; p < P2; p += blockDim.x) tw[p] = roots2[p];
    const int b = blockIdx.y, j0 = blockIdx.x * G;
    const zc<R>* zb = Z + (int64_t)b * s2 * (H2 + 1) * T1;
    // sequence q = u2 * (G/2) + gp holds rows (j0 + 2 gp, j0 + 2 gp + 1) of phase u2:
    // W(k) = S_a(k) + i S_b(k) and W(P2 - k) = conj S_a(k) + i conj S_b(k), S = Z for k <= H2.
    // The two rows' values are adjacent in Z (j1 contiguous): one 2-element read per stored bin.
    const FDiv fs2 = fdiv_make(s2);
    for (int idx = threadIdx.x; idx < nseq * (H2 + 1); idx += blockDim.x) {
        const int gp = idx & (G / 2 - 1);
        const int rest = idx >> (d.lgG3 - 1);
        const int k = fdiv(rest, fs2), u2 = rest - k * s2;
        const zc<R>* e = zb + ((int64_t)u2 * (H2 + 1) + k) * T1 + j0 + 2 * gp;
        zc<R> sa, sb;
        if constexpr (sizeof(R) == 4) {
            const float4 v = *reinterpret_cast<const float4*>(e);   // 16-byte aligned: j0 + 2 gp and T1 even
            sa = zc<R>{v.x, v.y};
            sb = zc<R>{v.z, v.w};
        } else {
            sa = e[0];
            sb = e[1];
        }
        zc<R>* q = A + (size_t)(u2 * (G / 2) + gp) * ld;
        q[k] = zc<R>{sa.re - sb.im, sa.im + sb.re};
        if (k > 0 && k < H2) q[P2 - k] = zc<R>{sa.re + sb.im, -sa.im + sb.re};
    }
    __syncthreads();
    const zc<R>* res = fft_seq(A, B, P2, nseq, ld, tw, true);
    for (int g = 0; g < G; ++g) {
        R* row = out + ((int64_t)b * T1 + j0 + g) * d.T2;
        for (int j2 = threadIdx.x; j2 < d.T2; j2 += blockDim.x) {
            const int p2 = fdiv(j2, fs2), u2 = j2 - p2 * s2;
            const zc<R> v = res[(size_t)(u2 * (G / 2) + (g >> 1)) * ld + p2];
            row[j2] = (g & 1) ? v.im : v.re;
        }
    }
}

template <typename R>
bool set_col_smem(size_t smem2)
{
    bool ok = true;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(mci2_col<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) == cudaSuccess;
    return ok;
}

template <typename R, int M>
void launch_col(const Dims2& D, const mci2::Tables& t, size_t smem2, int64_t batch, cudaStream_t st)
{
    mci2_col<R, M><<<dim3(D.H2 + 1, (unsigned)batch), dim3(kThreads2), smem2, st>>>(
        static_cast<const zc<R>*>(t.X), static_cast<zc<R>*>(t.Zw), static_cast<const zc<R>*>(t.Qt),
        static_cast<const zc<R>*>(t.Fy), static_cast<const zc<R>*>(t.Oy), static_cast<const zc<R>*>(t.Fx),
        static_cast<const zc<R>*>(t.roots1), D);
}

template <typename R>
mci_status set_smem_t(size_t smem1, size_t smem2, size_t smem3)
{
    if (cudaFuncSetAttribute(mci2_rowfwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1) != cudaSuccess ||
        !set_col_smem<R>(smem2) ||
        cudaFuncSetAttribute(mci2_rowinv<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3) != cudaSuccess)
        return MCI_ERR_CUDA;
    return MCI_OK;
}

template <typename R>
mci_status launch_t(const Dims2& D, const mci2::Tables& t, size_t smem1, size_t smem2, size_t smem3, const void* in,
                    void* out, int64_t batch, cudaStream_t st)
{
    const dim3 blk(kThreads2);
    mci2_rowfwd<R><<<dim3(D.P1 / D.G1, D.M, (unsigned)batch), blk, smem1, st>>>(
        static_cast<const R*>(in), static_cast<zc<R>*>(t.X), static_cast<const zc<R>*>(t.roots2), D);
    switch (D.M) {
    case 1: launch_col<R, 1>(D, t, smem2, batch, st); break;
    case 2: launch_col<R, 2>(D, t, smem2, batch, st); break;
    case 3: launch_col<R, 3>(D, t, smem2, batch, st); break;
    case 4: launch_col<R, 4>(D, t, smem2, batch, st); break;
    case 5: launch_col<R, 5>(D, t, smem2, batch, st); break;
    case 6: launch_col<R, 6>(D, t, smem2, batch, st); break;
    case 7: launch_col<R, 7>(D, t, smem2, batch, st); break;
    default: launch_col<R, 8>(D, t, smem2, batch, st); break;
    }
    mci2_rowinv<R><<<dim3(D.T1 / D.G3, (unsigned)batch), blk, smem3, st>>>(
        static_cast<const zc<R>*>(t.Zw), static_cast<R*>(out), static_cast<const zc<R>*>(t.roots2), D);
    return cudaGetLastError() == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

}  // namespace

namespace mci2 {

mci_status set_smem(int precision, size_t smem1, size_t smem2, size_t smem3)
{
    return precision == MCI_FP64 ? set_smem_t<double>(smem1, smem2, smem3) : set_smem_t<float>(smem1, smem2, smem3);
}

mci_status launch(int precision, const Dims2& d, const Tables& t, size_t smem1, size_t smem2, size_t smem3,
                  const void* in, void* out, int64_t batch, cudaStream_t st)
{
    return precision == MCI_FP64 ? launch_t<double>(d, t, smem1, smem2, smem3, in, out, batch, st)
                                 : launch_t<float>(d, t, smem1, smem2, smem3, in, out, batch, st);
}

}  // namespace mci2
