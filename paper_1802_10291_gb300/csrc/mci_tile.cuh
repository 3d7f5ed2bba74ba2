// The fused per-tile interpolation pipeline (Eq. (DFTexpression) of Cheng & Kou).
//
// A tile holds G signals of one size class in shared memory.  For every signal:
//   1. its M_in real channels (P samples each) are read as N = P/2 complex
//      values (even sample = real part, odd sample = imaginary part);
//   2. forward FFT of length N per channel;
//   3. per bin pair (k, N-k), k = 0..N/2: the real-input spectrum X_m[k] of
//      every channel (the even/odd split of a length-P real DFT), then
//      Y_q[k] = sum_m X_m[k] W[k][m][q] for every output phase q = (o, u), and
//      the packing of the Hermitian spectrum Y_q into N complex values whose
//      inverse FFT gives the real output samples 2l, 2l+1 of phase q;
//   4. inverse FFT of length N per phase;
//   5. phase u of output o holds the samples j = s l + u of the T-grid.
// W[k][m][q] already contains the per-residue inverse system matrix
// (Eq. (matrixeqn1)), the output operator, the phase e^{i n 2 pi u / T} of
// sub-grid u, the 1/P of the DFT, and the Hermitian symmetrisation that makes
// the output the real part of the interpolant; it is built in FP64 by the
// plan.  The spectrum never leaves shared memory.
#pragma once
#include "fft_device.cuh"

namespace mci {

// Combine of one bin pair (k, N - k), 0 <= k <= N/2, of one signal (buffers at base):
// the real-input spectrum X_m of every channel from its packed FFT Z_m, then
// Y_q = sum_m X_m W_m,q for both bins of the pair and every phase q, packed for the
// real inverse FFT.  W is stored as planes: W_m,q[k] at W[(m Q + q)(N + 1) + k].
// MIN, Q > 0 fix the channel and phase counts at compile time (all weight loads of
// the pair are independent and issued together); MIN = 0 takes them from c.
// Read-only cached load of one weight.
__device__ __forceinline__ cpx<float> ldw(const cpx<float>* p)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cpx<double> ldw(const cpx<double>* p)
{
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}

// SPLIT (runtime counts only): the caller spreads the phases of one pair over several
// threads, each with phases q0 .. q1 - 1; since phase buffer q shares its storage with
// channel buffer q, all threads read their channels, then a barrier, then write (every
// thread of the CTA calls it once; threads with act = false only take the barrier).
template <typename R, int MIN, int QC, bool SPLIT = false>
__device__ __forceinline__ void combine_pair(cpx<R>* base, const ClassDev& c, int k,
                                             const cpx<R>* __restrict__ W, cpx<R> w, int q0 = 0,
                                             int q1 = 1 << 30, bool act = true)
{
    const int npad = c.npad, N = c.N, NH = N / 2;
    const int Min = MIN > 0 ? MIN : c.M_in, Q = MIN > 0 ? QC : c.Q;
    const int ws = N + 1;
    const int kk = k == 0 ? 0 : N - k;   // mirror bin (k = 0 pairs with bin N == 0 of Z)
    const int pk = pad16(k), pkk = pad16(kk);
    // pack: Z'[k] = A + iC, Z'[N-k] = conj(A) + i conj(C),
    // A = Y[k] + conj Y[N-k], C = e^{2 pi i k / P} (Y[k] - conj Y[N-k])
    auto emit = [&](int q, cpx<R> ya, cpx<R> yb) {
        const cpx<R> A = ya + conjc(yb);
        const cpx<R> C = cmulc(ya - conjc(yb), w);
        base[q * npad + pk] = mk<R>(A.x - C.y, A.y + C.x);
        if (k != 0 && k != NH) base[q * npad + pkk] = mk<R>(A.x + C.y, C.x - A.y);
    };
    auto spectrum = [&](int m, cpx<R>& xa, cpx<R>& xb) {
        const cpx<R> zk = base[m * npad + pk];
        const cpx<R> zn = base[m * npad + pkk];
        if (k == 0) {
            xa = mk<R>(zk.x + zk.y, R(0));  // X[0]
            xb = mk<R>(zk.x - zk.y, R(0));  // X[N]
        } else {
            const cpx<R> e = scale(zk + conjc(zn), R(0.5));
            const cpx<R> d = zk - conjc(zn);
            const cpx<R> o = mk<R>(R(0.5) * d.y, R(-0.5) * d.x);  // d / (2i)
            const cpx<R> wo = cmul(w, o);
            xa = e + wo;                 // X[k]
            xb = conjc(e - wo);          // X[N-k]
        }
    };
    if constexpr (MIN > 0) {
        // FP32: every weight of the pair is loaded up front; FP64 (twice the registers):
        // one channel's weights at a time
        constexpr int MH = sizeof(R) == 4 ? MIN : 1;
        cpx<R> wa[MH][QC], wb[MH][QC];
        auto load = [&](int m, int slot) {
#pragma unroll
            for (int q = 0; q < QC; ++q) {
                wa[slot][q] = ldw(&W[(m * QC + q) * ws + k]);
                wb[slot][q] = ldw(&W[(m * QC + q) * ws + (N - k)]);
            }
        };
        if constexpr (MH == MIN) {
#pragma unroll
            for (int m = 0; m < MIN; ++m) load(m, m);
        }
        cpx<R> ya[QC], yb[QC];
#pragma unroll
        for (int m = 0; m < MIN; ++m) {
            const int sl = MH == MIN ? m : 0;
            if constexpr (MH != MIN) load(m, 0);
            cpx<R> xa, xb;
            spectrum(m, xa, xb);
#pragma unroll
            for (int q = 0; q < QC; ++q) {
                ya[q] = m == 0 ? cmul(xa, wa[sl][q]) : ya[q] + cmul(xa, wa[sl][q]);
                yb[q] = m == 0 ? cmul(xb, wb[sl][q]) : yb[q] + cmul(xb, wb[sl][q]);
            }
        }
#pragma unroll
        for (int q = 0; q < QC; ++q) emit(q, ya[q], yb[q]);
    } else {
        cpx<R> Xa[MCI_MAX_CHANNELS], Xb[MCI_MAX_CHANNELS];
#pragma unroll
        for (int m = 0; m < MCI_MAX_CHANNELS; ++m)
            if (act && m < Min) spectrum(m, Xa[m], Xb[m]);
        if constexpr (SPLIT) __syncthreads();
        for (int q = q0; act && q < min(Q, q1); ++q) {   // runtime counts: phases q0 .. q1 - 1
            cpx<R> ya = mk<R>(0, 0), yb = mk<R>(0, 0);
#pragma unroll
            for (int m = 0; m < MCI_MAX_CHANNELS; ++m) {
                if (m < Min) {
                    ya = ya + cmul(Xa[m], ldw(&W[(m * Q + q) * ws + k]));
                    yb = yb + cmul(Xb[m], ldw(&W[(m * Q + q) * ws + (N - k)]));
                }
            }
            emit(q, ya, yb);
        }
    }
}

template <typename R, int MIN, int QC>
__device__ __forceinline__ void combine_loop(cpx<R>* sm, const ClassDev& c, int gcount,
                                             const cpx<R>* __restrict__ W, int q0 = 0, int q1 = 1 << 30)
{
    const int total = (c.N / 2 + 1) * gcount;
    const R two_over_p = R(2) / R(c.P);
    const int sst = c.sstride;
    // item it = k * gcount + g; (k, g) advance incrementally (no division in the loop)
    const int it0 = ltid();
    const int step = blockDim.x;
    const int dk = step / gcount, dg = step - dk * gcount;
    int k = it0 / gcount, g = it0 - k * gcount;
    for (int it = it0; it < total; it += step) {
        const cpx<R> w = cis_neg_pi<R>(R(k) * two_over_p);  // e^{-2 pi i k / P}
        combine_pair<R, MIN, QC>(sm + g * sst, c, k, W, w, q0, q1);
        k += dk;
        g += dg;
        if (g >= gcount) {
            g -= gcount;
            ++k;
        }
    }
}

// Runtime channel/phase counts when the bin pairs of the tile cannot fill the CTA (a few
// short signals with many output phases, e.g. P = 64 evaluated at T = 4096): items are
// (bin pair, signal, chunk of phases), so the phases of one pair spread over threads.
template <typename R>
__device__ __forceinline__ void combine_loop_split(cpx<R>* sm, const ClassDev& c, int gcount,
                                                   const cpx<R>* __restrict__ W, int qa = 0, int qb = 1 << 30)
{
    qb = min(qb, c.Q);                          // phases qa .. qb - 1
    const int units = (c.N / 2 + 1) * gcount;   // at most blockDim.x / 2 (the caller's test)
    const int chunks = max(1, min(qb - qa, (int)blockDim.x / units));
    const int per = (qb - qa + chunks - 1) / chunks;
    const int it = ltid();                         // one item per thread at most
    const bool act = it < units * chunks;
    const int u = act ? it / chunks : 0, ch = act ? it - u * chunks : 0;
    const int k = u / gcount, g = u - k * gcount;
    const cpx<R> w = cis_neg_pi<R>(R(k) * (R(2) / R(c.P)));  // e^{-2 pi i k / P}
    combine_pair<R, 0, 0, true>(sm + g * c.sstride, c, k, W, w, qa + ch * per, min(qb, qa + (ch + 1) * per), act);
}

// Channel/phase counts with a compile-time combine: M = 3 measured channels with
// s = 4 phases (batched 1-D), and one channel with s = 2, 3, 4 (image rows and
// columns with derivative channels formed from the samples).
template <typename R>
__device__ __forceinline__ void combine_tile(cpx<R>* sm, const ClassDev& c, int gcount,
                                             const cpx<R>* __restrict__ W, int q0 = 0, int q1 = 1 << 30)
{
    if (q0 > 0 || q1 < c.Q) {   // this CTA's share of the phases (runtime counts)
        if (2 * (c.N / 2 + 1) * gcount <= (int)blockDim.x) combine_loop_split<R>(sm, c, gcount, W, q0, q1);
        else combine_loop<R, 0, 0>(sm, c, gcount, W, q0, q1);
        return;
    }
    if (c.M_in == 3 && c.Q == 4) combine_loop<R, 3, 4>(sm, c, gcount, W);
    else if (c.M_in == 1 && c.Q == 2) combine_loop<R, 1, 2>(sm, c, gcount, W);
    else if (c.M_in == 1 && c.Q == 3) combine_loop<R, 1, 3>(sm, c, gcount, W);
    else if (c.M_in == 1 && c.Q == 4) combine_loop<R, 1, 4>(sm, c, gcount, W);
    else if (c.Q > 4 && 2 * (c.N / 2 + 1) * gcount <= (int)blockDim.x) combine_loop_split<R>(sm, c, gcount, W);
    else combine_loop<R, 0, 0>(sm, c, gcount, W);
}

// Complex signals (Examples 4, 5): every bin k < P is its own residue class, so
// Y_q[k] = sum_m X_m[k] W_m,q[k] with the weights as planes of P bins (no real-input
// unpacking and no Hermitian packing).  Items (k, g), g fastest.
template <typename R>
__device__ __forceinline__ void combine_complex(cpx<R>* sm, const ClassDev& c, int gcount,
                                                const cpx<R>* __restrict__ W)
{
    const int N = c.N, npad = c.npad, sst = c.sstride, Min = c.M_in, Q = c.Q;
    const int total = N * gcount;
    const int it0 = ltid();
    const int step = blockDim.x;
    const int dk = step / gcount, dg = step - dk * gcount;
    int k = it0 / gcount, g = it0 - k * gcount;
    for (int it = it0; it < total; it += step) {
        cpx<R>* base = sm + g * sst;
        const int pk = pad16(k);
        cpx<R> X[MCI_MAX_CHANNELS];
#pragma unroll
        for (int m = 0; m < MCI_MAX_CHANNELS; ++m)
            if (m < Min) X[m] = base[m * npad + pk];
        for (int q = 0; q < Q; ++q) {
            cpx<R> y = mk<R>(0, 0);
#pragma unroll
            for (int m = 0; m < MCI_MAX_CHANNELS; ++m)
                if (m < Min) y = y + cmul(X[m], ldw(&W[(m * Q + q) * N + k]));
            base[q * npad + pk] = y;
        }
        k += dk;
        g += dg;
        if (g >= gcount) {
            g -= gcount;
            ++k;
        }
    }
}

// Buffer f of a tile with `cnt` transforms per signal: signal f / cnt, slot f % cnt.
struct SlotBase {
    int cnt, sstride, npad;
    uint64_t mag;   // fastdiv_magic(cnt)
    __device__ __forceinline__ int operator()(int f) const
    {
        const int g = fastdiv(f, mag);
        return g * sstride + (f - g * cnt) * npad;
    }
};

// Channel f % M_in of tile signal f / M_in, read in place from global memory as
// N complex values (even sample = real part).
template <typename R>
struct SrcContig {
    const R* in;
    const int64_t* off;
    int Min, P;
    uint64_t mag;   // fastdiv_magic(Min)
    __device__ __forceinline__ const cpx<R>* operator()(int f) const
    {
        const int g = fastdiv(f, mag);
        return reinterpret_cast<const cpx<R>*>(in + off[g] + (int64_t)(f - g * Min) * P);   // P: reals per channel
    }
};

// gin != nullptr: the tile's signals are read by the first forward pass directly
// from gin + s_in[g] (8-byte aligned); otherwise they are already in shared memory.
// The FFT twiddles live after the tile's buffers (smem_twiddle_offset); they are
// filled here, before or during the first pass, which needs none and ends with a barrier.
template <typename R, int N>
// q0, q1: a CTA that serves only phases q0 .. q1 - 1 of its signals (real signals with many
// output phases, spread over several CTAs); by default all of them.
__device__ __forceinline__ void compute_tile(cpx<R>* sm, const ClassDev& c, int gcount,
                                             const cpx<R>* __restrict__ W, const R* gin = nullptr,
                                             const int64_t* s_in = nullptr, int q0 = 0, int q1 = 1 << 30)
{
    q1 = min(q1, c.Q);
    cpx<R>* stw = sm + c.G * c.sstride;
    auto fill = [stw] { fill_twiddles_ct<R, N, elems_per_thread(N), 1>(stw); };
    if (gin) {
        // the twiddles are computed while the first pass's global loads are in flight
        fft_many_ct<R, N, false, true>(sm, gcount * c.M_in, SlotBase{c.M_in, c.sstride, c.npad, c.mag_min}, stw,
                                       SrcContig<R>{gin, s_in, c.M_in, c.chan_len, c.mag_min}, fill);
    } else {
        fill();
        fft_many_ct<R, N, false>(sm, gcount * c.M_in, SlotBase{c.M_in, c.sstride, c.npad, c.mag_min}, stw);
    }
    if (c.cplx) combine_complex<R>(sm, c, gcount, W);
    else combine_tile<R>(sm, c, gcount, W, q0, q1);
    __syncthreads();
    if (q0 > 0 || q1 < c.Q) {   // inverse transforms of phases q0 .. q1 - 1 only
        const int nq = q1 - q0;
        fft_many_ct<R, N, true>(sm + q0 * c.npad, gcount * nq, SlotBase{nq, c.sstride, c.npad, fastdiv_magic(nq)}, stw);
        return;
    }
    fft_many_ct<R, N, true>(sm, gcount * c.Q, SlotBase{c.Q, c.sstride, c.npad, c.mag_q}, stw);
}

// ---------------------------------------------------------------------------
// loads and stores
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Contiguous signals: signal g's M_in x P samples start at in + off[g].  Aligned
// signals are copied with asynchronous 16-byte copies (all in flight at once);
// the caller's barrier follows.  Threads run over (signal, vector) pairs of the
// whole tile, so short signals keep every thread busy.
template <typename R>
__device__ __forceinline__ void load_contig(cpx<R>* sm, const ClassDev& c, const R* __restrict__ in,
                                            const int64_t* off, int gcount)
{
    const int P = c.chan_len, Min = c.M_in, npad = c.npad, sst = c.sstride;   // P: reals per channel
    const int per = Min * P;
    constexpr int VW = sizeof(R) == 4 ? 4 : 2;  // reals per 16-byte copy
    bool vec = (P % VW) == 0;
    for (int g = 0; g < gcount; ++g) vec = vec && ((reinterpret_cast<uintptr_t>(in + off[g]) & 15) == 0);
    if (vec) {
        const int nv = per / VW;
        for (int t = ltid(); t < gcount * nv; t += blockDim.x) {
            const int g = t / nv, v = t - g * nv;
            const int i = v * VW;
            const int m = i / P, p = (i - m * P) >> 1;
            cp_async16(&sm[g * sst + m * npad + pad16(p)], in + off[g] + i);
        }
        cp_async_wait_all();
    } else {
        for (int t = ltid(); t < gcount * per; t += blockDim.x) {
            const int g = t / per, i = t - g * per;
            const int m = i / P, pp = i - m * P;
            R* d = reinterpret_cast<R*>(&sm[g * sst + m * npad + pad16(pp >> 1)]);
            d[pp & 1] = in[off[g] + i];
        }
    }
}

// Contiguous outputs: output o of signal g at out + off[g] + o * T, T = s P samples.
// Complex element l of phase buffer (o, u) holds samples s (2l) + u (real part) and
// s (2l + 1) + u (imaginary part), so one thread per (g, o, l) gathers the s phases
// and writes the 2s consecutive samples [2ls, 2ls + 2s): consecutive threads write
// consecutive runs.  Runs are written as 16-byte vectors when s is even (FP64) or a
// multiple of 4 (FP32) and the outputs are 16-byte aligned, as 8-byte pairs for
// FP32 with s even, else as scalars.
template <typename R, int N>
__device__ __forceinline__ void store_contig(const cpx<R>* sm, const ClassDev& c, R* __restrict__ out,
                                             const int64_t* off, int gcount, int q0 = 0, int q1 = 1 << 30)
{
    q1 = min(q1, c.Q);
    if (q0 > 0 || q1 < c.Q) {
        // phases q0 .. q1 - 1 only: phase q = o s + u, element l -> samples s (2l) + u, s (2l + 1) + u
        const int nq = q1 - q0, total = gcount * nq * N;
        for (int t = ltid(); t < total; t += blockDim.x) {
            const int gq = t / N, l = t - gq * N;
            const int g = gq / nq, q = q0 + (gq - g * nq);
            const int o = q / c.s, u = q - o * c.s;
            const cpx<R> z = sm[g * c.sstride + q * c.npad + pad16(l)];
            R* dst = out + off[g] + (int64_t)o * c.T;
            dst[(int64_t)2 * l * c.s + u] = z.x;
            dst[(int64_t)(2 * l + 1) * c.s + u] = z.y;
        }
        return;
    }
    const int T = c.T, s = c.s, npad = c.npad, sst = c.sstride, nout = c.n_out;
    constexpr int VR = 16 / sizeof(R);     // reals per 16-byte vector
    bool vec = (s % VR) == 0 && (T % VR) == 0, vec2 = sizeof(R) == 4 && (s % 2) == 0;
    for (int g = 0; g < gcount; ++g) {
        vec = vec && ((reinterpret_cast<uintptr_t>(out + off[g]) & 15) == 0);
        vec2 = vec2 && ((reinterpret_cast<uintptr_t>(out + off[g]) & 7) == 0);
    }
    const int total = gcount * nout * N;
    if constexpr (sizeof(R) == 4 && N % 32 == 0) {
        // s = 4: a warp writes the 256 samples of 32 consecutive l as two fully contiguous
        // 512-byte stores; lane 2i + e of store h takes component e of l = l0 + 16 h + i
        // (lanes 2i and 2i + 1 read the same shared-memory words: broadcast)
        if (vec && s == 4) {
            const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
            for (int base = (ltid() >> 5) * 32; base < total; base += nwarp * 32) {
                const int go = base / N;
                const int l0 = base - go * N;
                const int g = fastdiv(go, c.mag_nout), o = go - g * nout;
                const cpx<R>* src0 = sm + g * sst + o * 4 * npad;
                float* dst = out + off[g] + (int64_t)o * T + (int64_t)8 * l0;
                const int e = lane & 1;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const cpx<R>* src = src0 + pad16(l0 + 16 * h + (lane >> 1));
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const cpx<R> z = src[u * npad];
                        v[u] = e ? z.y : z.x;
                    }
                    reinterpret_cast<float4*>(dst)[32 * h + lane] = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
            return;
        }
    }
    for (int t = ltid(); t < total; t += blockDim.x) {
        const int go = t / N;                    // compile-time N: shift or multiply
        const int l = t - go * N;
        const int g = fastdiv(go, c.mag_nout), o = go - g * nout;
        const cpx<R>* src = sm + g * sst + o * s * npad + pad16(l);
        R* dst = out + off[g] + (int64_t)o * T + (int64_t)2 * l * s;
        if (vec) {
            for (int u = 0; u < s; u += VR) {
                cpx<R> z[VR];
#pragma unroll
                for (int e = 0; e < VR; ++e) z[e] = src[(u + e) * npad];
                if constexpr (sizeof(R) == 4) {
                    *reinterpret_cast<float4*>(dst + u) = make_float4(z[0].x, z[1].x, z[2].x, z[3].x);
                    *reinterpret_cast<float4*>(dst + s + u) = make_float4(z[0].y, z[1].y, z[2].y, z[3].y);
                } else {
                    *reinterpret_cast<double2*>(dst + u) = make_double2(z[0].x, z[1].x);
                    *reinterpret_cast<double2*>(dst + s + u) = make_double2(z[0].y, z[1].y);
                }
            }
        } else if (vec2) {      // FP32, s even: 8-byte pairs
            for (int u = 0; u < s; u += 2) {
                const cpx<R> z0 = src[u * npad], z1 = src[(u + 1) * npad];
                *reinterpret_cast<float2*>(dst + u) = make_float2(z0.x, z1.x);
                *reinterpret_cast<float2*>(dst + s + u) = make_float2(z0.y, z1.y);
            }
        } else {
            for (int u = 0; u < s; ++u) {
                const cpx<R> z = src[u * npad];
                dst[u] = z.x;
                dst[s + u] = z.y;
            }
        }
    }
}

// Complex outputs: output o of signal g at out + off[g] + 2 o T (interleaved re, im);
// sample j = s l + u is element l of phase buffer (o, u), so one thread per (g, o, l)
// writes the s consecutive complex samples [s l, s l + s).
template <typename R, int N>
__device__ __forceinline__ void store_contig_complex(const cpx<R>* sm, const ClassDev& c, R* __restrict__ out,
                                                     const int64_t* off, int gcount)
{
    const int T = c.T, s = c.s, npad = c.npad, sst = c.sstride, nout = c.n_out;
    bool vec = true;   // complex values as 8-byte (FP32) or 16-byte (FP64) stores
    for (int g = 0; g < gcount; ++g)
        vec = vec && ((reinterpret_cast<uintptr_t>(out + off[g]) & (2 * sizeof(R) - 1)) == 0);
    const int total = gcount * nout * N;
    for (int t = ltid(); t < total; t += blockDim.x) {
        const int go = t / N;
        const int l = t - go * N;
        const int g = fastdiv(go, c.mag_nout), o = go - g * nout;
        const cpx<R>* src = sm + g * sst + o * s * npad + pad16(l);
        R* dst = out + off[g] + 2 * ((int64_t)o * T + (int64_t)s * l);
        for (int u = 0; u < s; ++u) {
            const cpx<R> z = src[u * npad];
            if (vec) {
                *reinterpret_cast<cpx<R>*>(dst + 2 * u) = z;
            } else {
                dst[2 * u] = z.x;
                dst[2 * u + 1] = z.y;
            }
        }
    }
}

// Strided signals (image columns): signal g's sample p at in[base + g + p * ld]
// (one channel).  Consecutive g are adjacent in memory, so threads run over g fastest:
// thread t takes column g = t % gcount and samples p = t / gcount + j * per, per =
// blockDim / gcount, so the loop itself has no division.
template <typename R>
__device__ __forceinline__ void load_cols(cpx<R>* sm, const ClassDev& c, const R* __restrict__ in,
                                          int64_t base, int64_t ld, int gcount)
{
    const int P = c.P, sst = c.sstride;
    const int t = ltid(), per = blockDim.x / gcount;
    if (t < per * gcount) {
        const int g = t % gcount;
        R* col = reinterpret_cast<R*>(sm + g * sst);
        const R* src = in + base + g;
        for (int p = t / gcount; p < P; p += per) col[2 * pad16(p >> 1) + (p & 1)] = __ldg(src + (int64_t)p * ld);
    }
}

// Output sample x = s l + u of column g is component l & 1 of element l >> 1 of phase
// buffer u; (l, u) advance with x (no division in the loop).
template <typename R>
__device__ __forceinline__ void store_cols(const cpx<R>* sm, const ClassDev& c, R* __restrict__ out,
                                           int64_t base, int64_t ld, int gcount)
{
    const int T = c.T, s = c.s, npad = c.npad, sst = c.sstride;
    const int t = ltid(), per = blockDim.x / gcount;
    if (t < per * gcount) {
        const int g = t % gcount;
        int x = t / gcount;
        int l = x / s, u = x - l * s;
        const int dl = per / s, du = per - dl * s;
        const cpx<R>* col = sm + g * sst;
        R* dst = out + base + g;
        for (; x < T; x += per) {
            const cpx<R> z = col[u * npad + pad16(l >> 1)];
            dst[(int64_t)x * ld] = (l & 1) ? z.y : z.x;
            l += dl;
            u += du;
            if (u >= s) {
                u -= s;
                ++l;
            }
        }
    }
}

}  // namespace mci
