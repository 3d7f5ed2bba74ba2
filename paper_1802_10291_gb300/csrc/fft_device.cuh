// Shared-memory FFTs for the interpolation kernels.
//
// A length-N complex transform is computed by a group of N/E threads, each
// holding E elements in registers.  Every pass is one radix-R step of the
// Stockham autosort formulation (each butterfly reads R elements N/R apart,
// applies the twiddles w_{Ns R}^{(j mod Ns) r}, does an R-point DFT and
// writes R elements Ns apart at (j div Ns) Ns R + (j mod Ns)); the data stay
// in one shared-memory buffer because every thread loads its inputs before a
// barrier and stores after it.  Each transform length is its own compile-time
// instantiation with a fixed radix sequence (16/8/4/2 on the power-of-two
// part, one radix-3 pass last where N has a factor 3).  Twiddles come from a
// per-size table of e^{-2 pi i q / (2N)} computed in FP64 on the host.
#pragma once
#include <cuda_runtime.h>

#include "mci_internal.h"

namespace mci {

template <typename R>
struct alignas(2 * sizeof(R)) cpx {
    R x, y;
};

template <typename R>
struct vec2_of;
template <>
struct vec2_of<float> { using type = float2; };
template <>
struct vec2_of<double> { using type = double2; };

template <typename R>
__device__ __forceinline__ cpx<R> mk(R x, R y) { return cpx<R>{x, y}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename R>
__device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b)
{
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename R>
__device__ __forceinline__ cpx<R> conjc(cpx<R> a) { return {a.x, -a.y}; }
template <typename R>
__device__ __forceinline__ cpx<R> scale(cpx<R> a, R s) { return {a.x * s, a.y * s}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename R>
__device__ __forceinline__ cpx<R> rot90(cpx<R> a)
{
    return INV ? cpx<R>{-a.y, a.x} : cpx<R>{a.y, -a.x};
}
// multiply by the constant twiddle (c, s) for the forward sign, (c, -s) conjugated for INV:
// forward uses e^{-i theta} = (cos, -sin); pass c = cos theta, s = sin theta.
template <bool INV, typename R>
__device__ __forceinline__ cpx<R> twc(cpx<R> a, R c, R s)
{
    // forward: a * (c - i s); inverse: a * (c + i s)
    return INV ? cpx<R>{a.x * c - a.y * s, a.x * s + a.y * c}
               : cpx<R>{a.x * c + a.y * s, a.y * c - a.x * s};
}

// ---------------------------------------------------------------------------
// in-register DFTs, natural order in and out; forward sign e^{-2 pi i nk/R}
// ---------------------------------------------------------------------------
template <bool INV, typename R>
__device__ __forceinline__ void dft2(cpx<R>* v)
{
    cpx<R> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}

template <bool INV, typename R>
__device__ __forceinline__ void dft4(cpx<R>& x0, cpx<R>& x1, cpx<R>& x2, cpx<R>& x3)
{
    cpx<R> a = x0 + x2, b = x0 - x2, c = x1 + x3, d = rot90<INV>(x1 - x3);
    x0 = a + c;
    x2 = a - c;
    x1 = b + d;
    x3 = b - d;
}

template <bool INV, typename R>
__device__ __forceinline__ void dft4(cpx<R>* v) { dft4<INV>(v[0], v[1], v[2], v[3]); }

template <bool INV, typename R>
__device__ __forceinline__ void dft3(cpx<R>* v)
{
    const R h = R(0.86602540378443864676372317075294);  // sin(2 pi / 3)
    cpx<R> t = v[1] + v[2];
    cpx<R> m = v[0] - scale(t, R(0.5));
    cpx<R> d = v[1] - v[2];
    // forward: X1 = m - i h d, X2 = m + i h d
    cpx<R> ihd = INV ? cpx<R>{-h * d.y, h * d.x} : cpx<R>{h * d.y, -h * d.x};  // (-/+ i) h d
    v[0] = v[0] + t;
    v[1] = m + ihd;
    v[2] = m - ihd;
}

// 8 = 2 x 4: n = n1 + 2 n2, k = k2 + 4 k1
template <bool INV, typename R>
__device__ __forceinline__ void dft8(cpx<R>* v)
{
    const R r2 = R(0.70710678118654752440084436210485);
    cpx<R> a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6];
    cpx<R> b0 = v[1], b1 = v[3], b2 = v[5], b3 = v[7];
    dft4<INV>(a0, a1, a2, a3);
    dft4<INV>(b0, b1, b2, b3);
    b1 = twc<INV>(b1, r2, r2);
    b2 = rot90<INV>(b2);
    b3 = twc<INV>(b3, -r2, r2);
    v[0] = a0 + b0; v[4] = a0 - b0;
    v[1] = a1 + b1; v[5] = a1 - b1;
    v[2] = a2 + b2; v[6] = a2 - b2;
    v[3] = a3 + b3; v[7] = a3 - b3;
}

// 16 = 4 x 4: n = n1 + 4 n2, k = k2 + 4 k1; twiddle w16^{n1 k2} between the stages
template <bool INV, typename R>
__device__ __forceinline__ void dft16(cpx<R>* v)
{
    const R c1 = R(0.92387953251128675612818318939679);  // cos(pi/8)
    const R s1 = R(0.38268343236508977172845998403040);  // sin(pi/8)
    const R r2 = R(0.70710678118654752440084436210485);
    cpx<R> y[16];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        cpx<R> a = v[n1], b = v[n1 + 4], c = v[n1 + 8], d = v[n1 + 12];
        dft4<INV>(a, b, c, d);
        y[n1 * 4 + 0] = a;
        y[n1 * 4 + 1] = b;
        y[n1 * 4 + 2] = c;
        y[n1 * 4 + 3] = d;
    }
    // n1 = 1: w^{k2}, k2 = 1,2,3 -> angles pi/8, pi/4, 3pi/8
    y[5] = twc<INV>(y[5], c1, s1);
    y[6] = twc<INV>(y[6], r2, r2);
    y[7] = twc<INV>(y[7], s1, c1);
    // n1 = 2: w^{2 k2} -> pi/4, pi/2, 3pi/4
    y[9] = twc<INV>(y[9], r2, r2);
    y[10] = rot90<INV>(y[10]);
    y[11] = twc<INV>(y[11], -r2, r2);
    // n1 = 3: w^{3 k2} -> 3pi/8, 3pi/4, 9pi/8
    y[13] = twc<INV>(y[13], s1, c1);
    y[14] = twc<INV>(y[14], -r2, r2);
    y[15] = twc<INV>(y[15], -c1, -s1);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        cpx<R> a = y[k2], b = y[4 + k2], c = y[8 + k2], d = y[12 + k2];
        dft4<INV>(a, b, c, d);
        v[k2] = a;
        v[k2 + 4] = b;
        v[k2 + 8] = c;
        v[k2 + 12] = d;
    }
}

template <int RAD, bool INV, typename R>
__device__ __forceinline__ void dft(cpx<R>* v)
{
    if constexpr (RAD == 2) dft2<INV>(v);
    else if constexpr (RAD == 3) dft3<INV>(v);
    else if constexpr (RAD == 4) dft4<INV>(v);
    else if constexpr (RAD == 8) dft8<INV>(v);
    else dft16<INV>(v);
}

// ---------------------------------------------------------------------------
// transforms of length N = 2^a (E = min(16, N) elements per thread, radices
// 16/8/4/2) and N = 3 * 2^a (E = min(12, N), radices 4/2 then one radix-3
// pass last).  Because the radix-3 pass comes last, every Ns before it is a
// power of two, so all index arithmetic is shifts and masks.
// ---------------------------------------------------------------------------
// Returns x through an opaque move, so index arithmetic derived from it is
// recomputed where it is used instead of being hoisted out of loops and kept
// live in registers across them.
__device__ __forceinline__ int opaque(int x)
{
    int y;
    asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

// Thread index laundered through an opaque move.  Index arithmetic of the tile
// code derives from it, so the compiler cannot hoist that arithmetic out of the
// persistent tile loop and keep it live across iterations (which made every
// kernel spill).
__device__ __forceinline__ int ltid() { return opaque((int)threadIdx.x); }

// Padded shared-memory positions of a butterfly: when the offsets pad16(x + c_r) -
// pad16(x) of a pass's R reads (or writes) do not depend on the butterfly's base x,
// they are compile-time constants and every access is base + immediate.
//   reads  x = j (< N / RAD), c_r = r * N / RAD: constant when N / RAD is a multiple of
//          32 or a power of two (no carry into bit 5 from the low part);
//   writes x = (j div NS) NS RAD + j mod NS, c_r = r * NS: constant when NS is a power of
//          two and NS >= 32, or NS * RAD divides 32, or 32 divides NS * RAD.
__host__ __device__ constexpr bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
__host__ __device__ constexpr bool read_offsets_const(int N, int RAD)
{
    return (N / RAD) % 32 == 0 || is_pow2(N / RAD);
}
__host__ __device__ constexpr bool write_offsets_const(int NS, int RAD)
{
    return is_pow2(NS) && (NS >= 32 || 32 % (NS * RAD) == 0 || (NS * RAD) % 32 == 0);
}

// One Stockham pass of radix RAD over nfft length-N buffers (buffer f at
// sm + base_of(f)); E elements per thread, groups of N/E threads per buffer.
// Butterfly j needs w^r, r < RAD, w = e^{-2 pi i (j mod NS) / (NS RAD)}: w is read
// from this pass's shared-memory twiddle row stw (built at tile start), its
// powers come from a product tree of depth <= 4.  With GIN the pass reads its
// input from global memory (src_of(f), natural order, first pass only) and runs
// hook() (all threads, once) while those loads are in flight.
template <typename R, int N, int NS, int E, int RAD, bool INV, bool GIN, typename BaseFn, typename SrcFn,
          typename Hook>
__device__ __forceinline__ void fft_pass_many(cpx<R>* sm, int nfft, BaseFn base_of, SrcFn src_of,
                                              const cpx<R>* stw, Hook hook)
{
    constexpr int NB = E / RAD;
    constexpr int TPF = N / E;
    constexpr int STRIDE = N / RAD;
    constexpr bool RD_CONST = read_offsets_const(N, RAD);
    constexpr bool WR_CONST = write_offsets_const(NS, RAD);
    const int tix = ltid();
    const int groups = blockDim.x / TPF;
    const int gi = tix / TPF;
    const int lt = tix - gi * TPF;
#pragma unroll 1
    for (int f0 = 0; f0 < nfft; f0 += groups) {
        const int f = f0 + gi;
        const bool active = gi < groups && f < nfft;
        cpx<R>* buf = sm + (active ? base_of(f) : 0);
        const int ltr = opaque(lt);
        cpx<R> v[NB * RAD];
        cpx<R> w1[NB];
        if (active && NS > 1) {
#pragma unroll
            for (int i = 0; i < NB; ++i) w1[i] = stw[(ltr + i * TPF) & (NS - 1)];
        }
        if (active) {
            if constexpr (GIN) {
                const cpx<R>* src = src_of(f);
#pragma unroll
                for (int i = 0; i < NB; ++i)
#pragma unroll
                    for (int r = 0; r < RAD; ++r) v[i * RAD + r] = src[ltr + i * TPF + r * STRIDE];
            } else {
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int j = ltr + i * TPF;
                    if constexpr (RD_CONST) {
                        const cpx<R>* b = buf + pad16(j);
#pragma unroll
                        for (int r = 0; r < RAD; ++r) v[i * RAD + r] = b[pad16(r * STRIDE)];
                    } else {
#pragma unroll
                        for (int r = 0; r < RAD; ++r) v[i * RAD + r] = buf[pad16(j + r * STRIDE)];
                    }
                }
            }
        }
        if constexpr (!GIN) __syncthreads();
        if constexpr (GIN) {
            if (f0 == 0) hook();
        }
        if (active) {
            const int lts = opaque(lt);
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int j = lts + i * TPF;
                const int jm = j & (NS - 1);
                if constexpr (NS > 1) {
                    cpx<R> w[RAD];
                    w[1] = w1[i];
#pragma unroll
                    for (int r = 2; r < RAD; ++r)
                        w[r] = (r & 1) ? cmul(w[r - 1], w[1]) : cmul(w[r / 2], w[r / 2]);
#pragma unroll
                    for (int r = 1; r < RAD; ++r)
                        v[i * RAD + r] = INV ? cmulc(v[i * RAD + r], w[r]) : cmul(v[i * RAD + r], w[r]);
                }
                dft<RAD, INV>(&v[i * RAD]);
                const int d = (j - jm) * RAD + jm;
                if constexpr (WR_CONST) {
                    cpx<R>* b = buf + pad16(d);
#pragma unroll
                    for (int r = 0; r < RAD; ++r) b[pad16(r * NS)] = v[i * RAD + r];
                } else {
#pragma unroll
                    for (int r = 0; r < RAD; ++r) buf[pad16(d + r * NS)] = v[i * RAD + r];
                }
            }
        }
        __syncthreads();
    }
}

struct NoSrc {
    template <typename T>
    __device__ __forceinline__ const T* operator()(int) const { return nullptr; }
};

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Compile-time radix sequence of a length-N transform with E elements per thread
// (pick_radix); stw is the shared-memory twiddle table (smem_twiddle_offset).
template <typename R, int N, int E, int NS, bool INV, bool GIN, typename BaseFn, typename SrcFn,
          typename Hook>
__device__ __forceinline__ void fft_passes_ct(cpx<R>* sm, int nfft, BaseFn base_of, SrcFn src_of,
                                              const cpx<R>* stw, Hook hook)
{
    if constexpr (NS < N) {
        constexpr int RAD = pick_radix(N / NS, E);
        fft_pass_many<R, N, NS, E, RAD, INV, GIN && NS == 1>(sm, nfft, base_of, src_of,
                                                               stw + smem_twiddle_offset(N, NS), hook);
        fft_passes_ct<R, N, E, NS * RAD, INV, GIN>(sm, nfft, base_of, src_of, stw, hook);
    }
}

// nfft transforms of length N held in shared memory (GIN: read from global memory).
template <typename R, int N, bool INV, bool GIN = false, typename BaseFn, typename SrcFn = NoSrc,
          typename Hook = NoHook>
__device__ __forceinline__ void fft_many_ct(cpx<R>* sm, int nfft, BaseFn base_of, const cpx<R>* stw,
                                            SrcFn src_of = SrcFn(), Hook hook = Hook())
{
    fft_passes_ct<R, N, elems_per_thread(N), 1, INV, GIN>(sm, nfft, base_of, src_of, stw, hook);
}

// e^{-2 pi i num / den}
template <typename R>
__device__ __forceinline__ cpx<R> cis_neg(int num, int den);
template <>
__device__ __forceinline__ cpx<float> cis_neg<float>(int num, int den)
{
    float s, c;
    sincospif(2.0f * (float)num / (float)den, &s, &c);
    return {c, -s};
}
template <>
__device__ __forceinline__ cpx<double> cis_neg<double>(int num, int den)
{
    double s, c;
    sincospi(2.0 * (double)num / (double)den, &s, &c);
    return {c, -s};
}

// e^{-pi i x} for x = 2 num / den given as num * (2 / den) (the caller hoists 2 / den)
template <typename R>
__device__ __forceinline__ cpx<R> cis_neg_pi(R x);
template <>
__device__ __forceinline__ cpx<float> cis_neg_pi<float>(float x)
{
    float s, c;
    sincospif(x, &s, &c);
    return {c, -s};
}
template <>
__device__ __forceinline__ cpx<double> cis_neg_pi<double>(double x)
{
    double s, c;
    sincospi(x, &s, &c);
    return {c, -s};
}

// Fill the shared-memory twiddle table of a length-N transform (all threads call;
// the caller's barrier follows).
template <typename R, int N, int E, int NS>
__device__ __forceinline__ void fill_twiddles_ct(cpx<R>* stw)
{
    if constexpr (NS < N) {
        constexpr int RAD = pick_radix(N / NS, E);
        if constexpr (NS > 1) {
            for (int jm = ltid(); jm < NS; jm += blockDim.x)
                stw[smem_twiddle_offset(N, NS) + jm] = cis_neg<R>(jm, NS * RAD);
        }
        fill_twiddles_ct<R, N, E, NS * RAD>(stw);
    }
}

}  // namespace mci
