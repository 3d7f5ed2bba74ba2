// Fused radix-8 interpolation kernel for real FP32 signals (Eq. (DFTexpression) of
// Cheng & Kou) in size classes whose FFT length N = P/2 is a power of two.
//
// A tile holds G = 2048/N signals and N/8 threads serve one signal.  Thread j of a
// signal computes butterfly j (and j + (N/8) i where a pass has radix below 8) of every
// pass, for all M_in channels of the forward transforms and all Q = s n_out phases of
// the inverse ones, so each twiddle is formed once and applied to every channel or phase.
//   forward:  M_in length-N complex FFTs of the packed channels (even sample = real part,
//             odd sample = imaginary part), Stockham passes through shared memory; the
//             first pass reads global memory;
//   junction: the last forward pass leaves bins k = j + (N/8) r, r < 8, in registers, and
//             those are the elements the first inverse pass reads.  In between, each thread
//             forms the real-input spectra X_m[k] (even/odd split of the packed FFT), the
//             phase spectra Y_q[k] = sum_m X_m[k] W_m,q[k] (Eq. (matrixeqn1) per residue,
//             through the plan's folded weights) and their packing for the real inverse
//             transforms.  Both steps need the mirror bin N - k; a lane permutation puts the
//             thread holding it in the same warp (lane ^ HALF), so it moves by warp shuffles;
//   inverse:  Q length-N inverse FFTs; the last pass leaves output elements l = j + (N/8) t
//             of every phase in the thread, i.e. all samples [2 s l, 2 s l + 2 s) of each
//             output, which go to global memory directly (16-byte stores for s = 2, 4).
// Shared memory holds M_in (forward) or Q (inverse) buffers of N complex values per signal,
// without padding: every pass writes through an XOR swizzle of the low four index bits,
// keyed by higher bits and chosen per (stride, radix) so that the strided writes of the pass
// and the reads of the next pass are free of bank conflicts.  The spectra never leave the SM.
#include "fft_device.cuh"
#include "mci_kernels.cuh"

namespace mci {
namespace {

using C = cpx<float>;

// Element e of a buffer written by a pass of stride NS and radix R.
template <int NS, int R>
__device__ __forceinline__ int swz(int e)
{
    if constexpr (NS == 1) return e ^ ((e >> 4) & (R - 1));
    else if constexpr (NS == 2) return e ^ (((e >> 4) & 7) << 1);
    else if constexpr (NS < 16) return e ^ (((e >> 5) & 3) << 2);
    else return e;
}

__device__ __forceinline__ C ldc(const C* p)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}

__device__ __forceinline__ C shfl_xor_c(C v, int m)
{
    return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}

// w^r for 1 <= r < R from w (forward sign; conjugated for the inverse)
template <int R, bool INV>
__device__ __forceinline__ void powers(C w, C (&wp)[R])
{
    wp[0] = mk<float>(1.f, 0.f);
    wp[1] = INV ? conjc(w) : w;
#pragma unroll
    for (int r = 2; r < R; ++r) wp[r] = (r & 1) ? cmul(wp[r - 1], wp[1]) : cmul(wp[r / 2], wp[r / 2]);
}

// Pass PS of a transform (INV: inverse) on V buffers of N complex at sm + v N.  Butterfly b
// reads elements b + r N / R and writes element r at (b div NS) NS R + b mod NS + r NS.
template <int N, int PS, bool INV>
struct Pass {
    static constexpr int R = fast_radix(N, INV, PS);
    static constexpr int NS = fast_ns(N, INV, PS);
    static constexpr int NB = 8 / R;      // butterflies per thread
    static constexpr int TPS = N / 8;
    static constexpr int ST = N / R;

    // element (i, r) of thread j: butterfly j + TPS i, input r
    // fx: XORed into every element index (a per-signal layout; 0 on the radix-8 kernels)
    template <int V>
    static __device__ __forceinline__ void load(const C* sm, int j, C (&v)[V][8], int fx = 0)
    {
        constexpr int PNS = fast_ns(N, INV, PS - 1), PR = fast_radix(N, INV, PS - 1);
#pragma unroll
        for (int x = 0; x < V; ++x)
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int r = 0; r < R; ++r) v[x][i * R + r] = sm[x * N + (swz<PNS, PR>(j + TPS * i + r * ST) ^ fx)];
    }

    template <int V>
    static __device__ __forceinline__ void compute(C (&v)[V][8], int j, const C* tab)
    {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            if constexpr (NS > 1) {
                const int b = j + TPS * i;
                C wp[R];
                powers<R, INV>(ldc(tab + fast_tw_offset(N, INV, PS) + (b & (NS - 1))), wp);
#pragma unroll
                for (int x = 0; x < V; ++x)
#pragma unroll
                    for (int r = 1; r < R; ++r) v[x][i * R + r] = cmul(v[x][i * R + r], wp[r]);
            }
#pragma unroll
            for (int x = 0; x < V; ++x) dft<R, INV>(&v[x][i * R]);
        }
    }

    template <int V>
    static __device__ __forceinline__ void store(C* sm, int j, const C (&v)[V][8], int fx = 0)
    {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int b = j + TPS * i;
            const int d = (b & ~(NS - 1)) * R + (b & (NS - 1));
#pragma unroll
            for (int x = 0; x < V; ++x)
#pragma unroll
                for (int r = 0; r < R; ++r) sm[x * N + (swz<NS, R>(d + r * NS) ^ fx)] = v[x][i * R + r];
        }
    }
};

// Barrier among the N/8 threads of signal g of a tile.  Between the tile's loads and its
// stores the signals share nothing, so each waits only for its own threads: its warp when it
// fits in one, else named barrier 1 + g (barrier 0 stays the CTA-wide one).
template <int N>
__device__ __forceinline__ void sig_sync(int g)
{
    constexpr int TPS = N / 8;
    if constexpr (TPS >= 256) __syncthreads();
    else if constexpr (TPS <= 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(TPS) : "memory");
}

// Passes PS .. L-2 of a transform, each: load, barrier, twiddles and DFTs, store, barrier.
template <int N, int V, int PS, bool INV>
__device__ __forceinline__ void middle_passes(C* sm, int j, const C* tab, int g, int fx = 0)
{
    if constexpr (PS < fast_passes(N) - 1) {
        using PP = Pass<N, PS, INV>;
        C v[V][8];
        PP::template load<V>(sm, j, v, fx);
        sig_sync<N>(g);
        PP::template compute<V>(v, j, tab);
        PP::template store<V>(sm, j, v, fx);
        sig_sync<N>(g);
        middle_passes<N, V, PS + 1, INV>(sm, j, tab, g, fx);
    }
}

// One tile of the fused path: its signals and where their data live.
struct FastTile {
    const C* W;              // the class's bin weights
    const C* tab;            // the class's fused-path table
    const float* in;
    float* out;
    const int64_t* s_in;     // per signal of the tile (shared memory); image columns: the
    const int64_t* s_out;    // offsets of their first samples, consecutive columns
    int cnt;                 // signals in the tile
    int64_t ld;              // image columns: the row pitch of input and output (else 0)
};

// Image columns: the G = 2048/N columns of a tile are staged through shared memory so that
// every global access is a row segment of the G columns.  Column g's words start rotated by
// (32/G) g, which keeps the row-wise staging accesses and the column-wise FFT accesses free of
// bank conflicts (G columns x 32/G rows of a warp cover the 32 banks).
template <int N>
__device__ __forceinline__ int col_rot(int g)
{
    return (32 / (2048 / N)) * g;
}

// The whole pipeline for one tile (all threads of the CTA; smem_raw holds the buffers).
// COLS: the signals are G consecutive image columns (one channel, one output).
template <int N, int MIN, int S, int NOUT, bool COLS = false>
__device__ __forceinline__ void fast_tile(const FastTile& ft, unsigned char* smem_raw)
{
    constexpr int Q = S * NOUT, QM = MIN > Q ? MIN : Q;
    constexpr int TPS = N / 8, L = fast_passes(N), P = 2 * N, T = S * P;
    constexpr int HALF = TPS >= 32 ? 16 : TPS / 2;   // lane distance of mirror partners
    static_assert(N >= kFastMinN && N <= kFastMaxN && (N & (N - 1)) == 0, "fused path length");
    const int tid = threadIdx.x, g = tid / TPS, t = tid - g * TPS;
    const bool active = g < ft.cnt;
    C* sm = reinterpret_cast<C*>(smem_raw) + g * QM * N;
    const C* W = ft.W;
    const C* tab = ft.tab;
    // natural butterfly index, and the permuted one of the junction: within each run of
    // 2 HALF threads, the first half takes a = w HALF + i, the second half N/8 - a (N/16
    // for a = 0), so that bins k and N - k sit on lanes l and l ^ HALF
    const int jn = t;
    int jm;
    {
        const int w = t / (2 * HALF), l = t - w * 2 * HALF, i = l % HALF, hi = l / HALF;
        const int aa = w * HALF + i;
        jm = hi ? (aa == 0 ? TPS / 2 : TPS - aa) : aa;
    }

    // ---- forward pass 0: packed channels straight from global memory ----
    {
        using P0 = Pass<N, 0, false>;
        C x[MIN][8];
        const float* src = ft.in + (active ? ft.s_in[g] : 0);
        const bool al = (reinterpret_cast<uintptr_t>(src) & 7) == 0;
        if constexpr (COLS) {
            static_assert(MIN == 1 && NOUT == 1 && S >= 2, "image columns: one channel, one output");
            // rows p of the tile's columns into buffer 1 of each column (rotated): thread tid
            // stages column tid mod G, rows tid / G + (256 / G) k, k < P G / 256 = 16
            constexpr int G = 2048 / N, RPI = 256 / G;
            const int gs = tid % G, p0 = tid / G;
            float* dstc = reinterpret_cast<float*>(reinterpret_cast<C*>(smem_raw) + gs * QM * N + N);
            const int q0 = p0 + col_rot<N>(gs);
            if (gs < ft.cnt) {
                const float* src = ft.in + ft.s_in[0] + gs + (int64_t)p0 * ft.ld;
                const int64_t step = (int64_t)RPI * ft.ld;
#pragma unroll
                for (int k = 0; k < P / RPI; ++k) {
                    dstc[(q0 + RPI * k) & (P - 1)] = __ldcs(src);
                    src += step;
                }
            } else {
#pragma unroll
                for (int k = 0; k < P / RPI; ++k) dstc[(q0 + RPI * k) & (P - 1)] = 0.f;
            }
            __syncthreads();
            const float* st = reinterpret_cast<const float*>(sm + N);
            const int rot = col_rot<N>(g);
#pragma unroll
            for (int i = 0; i < P0::NB; ++i)
#pragma unroll
                for (int r = 0; r < P0::R; ++r) {
                    const float2 z = *reinterpret_cast<const float2*>(
                        st + ((2 * (jn + TPS * i + r * P0::ST) + rot) & (P - 1)));
                    x[0][i * P0::R + r] = mk<float>(z.x, z.y);
                }
        } else if (active && al) {
#pragma unroll
            for (int m = 0; m < MIN; ++m)
#pragma unroll
                for (int i = 0; i < P0::NB; ++i)
#pragma unroll
                    for (int r = 0; r < P0::R; ++r) {
                        const float2 z = __ldcs(reinterpret_cast<const float2*>(src + m * P) + jn + TPS * i + r * P0::ST);
                        x[m][i * P0::R + r] = mk<float>(z.x, z.y);
                    }
        } else if (active) {
#pragma unroll
            for (int m = 0; m < MIN; ++m)
#pragma unroll
                for (int i = 0; i < P0::NB; ++i)
#pragma unroll
                    for (int r = 0; r < P0::R; ++r) {
                        const float* e = src + m * P + 2 * (jn + TPS * i + r * P0::ST);
                        x[m][i * P0::R + r] = mk<float>(__ldcs(e), __ldcs(e + 1));
                    }
        } else {
#pragma unroll
            for (int m = 0; m < MIN; ++m)
#pragma unroll
                for (int e = 0; e < 8; ++e) x[m][e] = mk<float>(0.f, 0.f);
        }
        P0::template compute<MIN>(x, jn, tab);
        P0::template store<MIN>(sm, jn, x);
        sig_sync<N>(g);
    }
    middle_passes<N, MIN, 1, false>(sm, jn, tab, g);

    // ---- last forward pass (permuted index), spectra, combine, first inverse pass ----
    {
        using PL = Pass<N, L - 1, false>;
        static_assert(PL::R == 8, "the last forward pass is radix 8");
        C z[MIN][8];
        PL::template load<MIN>(sm, jm, z);
        sig_sync<N>(g);   // the first inverse pass below overwrites these buffers
        PL::template compute<MIN>(z, jm, tab);
        // z[m][r] = Z_m[k], k = jm + TPS r; its mirror N - k is element 7 - r of the partner
        // lane, except on the two self-paired lanes: jm = 0 (k = TPS r <-> TPS (8 - r)) and
        // jm = TPS / 2 (element 7 - r of the same lane)
        const bool self0 = jm == 0, selfh = jm == TPS / 2;
        C wk[8];   // e^{-2 pi i k / P}
#pragma unroll
        for (int r = 0; r < 8; ++r) wk[r] = ldc(tab + jm + r * TPS);
        float xN[MIN];   // X_m[N] (real), used by the jm = 0 lane
#pragma unroll
        for (int m = 0; m < MIN; ++m) {
            xN[m] = z[m][0].x - z[m][0].y;
            C zm[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const C pr = shfl_xor_c(z[m][7 - r], HALF);
                zm[r] = self0 ? z[m][(8 - r) & 7] : (selfh ? z[m][7 - r] : pr);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                // X[k] = (Z[k] + conj Z[N-k]) / 2 + e^{-2 pi i k / P} (Z[k] - conj Z[N-k]) / (2i)
                const C e = scale(z[m][r] + conjc(zm[r]), 0.5f);
                const C d = z[m][r] - conjc(zm[r]);
                z[m][r] = e + cmul(wk[r], mk<float>(0.5f * d.y, -0.5f * d.x));
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            C y[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int k = jm + r * TPS;
                C acc = cmul(z[0][r], ldc(W + (size_t)q * (N + 1) + k));
#pragma unroll
                for (int m = 1; m < MIN; ++m) acc = acc + cmul(z[m][r], ldc(W + (size_t)(m * Q + q) * (N + 1) + k));
                y[r] = acc;
            }
            C yN = mk<float>(0.f, 0.f);   // Y_q[N], on the jm = 0 lane
            if (self0) {
#pragma unroll
                for (int m = 0; m < MIN; ++m) yN = yN + scale(ldc(W + (size_t)(m * Q + q) * (N + 1) + N), xN[m]);
            }
            C zp[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const C pr = shfl_xor_c(y[7 - r], HALF);
                const C ym = self0 ? (r == 0 ? yN : y[(8 - r) & 7]) : (selfh ? y[7 - r] : pr);
                // packing for the real inverse FFT: A + i C, A = Y[k] + conj Y[N-k],
                // C = e^{2 pi i k / P} (Y[k] - conj Y[N-k])
                const C A = y[r] + conjc(ym);
                const C Cc = cmulc(y[r] - conjc(ym), wk[r]);
                zp[r] = mk<float>(A.x - Cc.y, A.y + Cc.x);
            }
            dft<8, true>(zp);   // inverse pass 0 (stride 1): element r of butterfly jm at 8 jm + r
#pragma unroll
            for (int r = 0; r < 8; ++r) sm[q * N + swz<1, 8>(8 * jm + r)] = zp[r];
        }
        sig_sync<N>(g);
    }
    middle_passes<N, Q, 1, true>(sm, jn, tab, g);

    // ---- last inverse pass, output samples straight to global memory ----
    {
        using PL = Pass<N, L - 1, true>;
        C y[Q][8];
        PL::template load<Q>(sm, jn, y);
        PL::template compute<Q>(y, jn, tab);
        if constexpr (COLS) {
            // samples [2 S l, 2 S l + 2 S) of the column (re of phases 0..S-1, then im) into the
            // column's buffers as T = 2 S N floats, rotated, then rows of the G columns out
            constexpr int G = 2048 / N;
            __syncthreads();   // every thread has read its last-pass inputs
            float* oc = reinterpret_cast<float*>(sm);
            const int rot = col_rot<N>(g);
#pragma unroll
            for (int i = 0; i < PL::NB; ++i)
#pragma unroll
                for (int r = 0; r < PL::R; ++r) {
                    const int l = jn + TPS * i + r * PL::ST, e = i * PL::R + r;
                    float v[2 * S];
#pragma unroll
                    for (int u = 0; u < S; ++u) {
                        v[u] = y[u][e].x;
                        v[S + u] = y[u][e].y;
                    }
                    if constexpr (S % 2 == 0 && N >= 256) {
                        // the rotation (4 g or 8 g words) keeps the 2S-word chunks 16-byte aligned;
                        // with s = 4 the two chunks of lanes with bit 2 of l set trade places, so
                        // a quarter warp's eight 16-byte stores hit eight different bank groups
                        // (row x sits at word x ^ ((x >> 3) & 4))
#pragma unroll
                        for (int k = 0; k < S / 2; ++k) {
                            int pos = 2 * S * l + 4 * (S == 4 ? k ^ ((l >> 2) & 1) : k) + rot;
                            if (pos >= T) pos -= T;
                            *reinterpret_cast<float4*>(oc + pos) =
                                make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < S; ++k) {
                            int pos = 2 * S * l + 2 * k + rot;
                            if (pos >= T) pos -= T;
                            *reinterpret_cast<float2*>(oc + pos) = make_float2(v[2 * k], v[2 * k + 1]);
                        }
                    }
                }
            __syncthreads();
            // rows x of the tile's columns out: thread tid writes column tid mod G, rows
            // tid / G + (256 / G) k, k < T G / 256 = 16 S
            const int gs = tid % G, x0 = tid / G;
            if (gs < ft.cnt) {
                const float* srcc = reinterpret_cast<const float*>(reinterpret_cast<C*>(smem_raw) + gs * QM * N);
                float* dst = ft.out + ft.s_out[0] + gs + (int64_t)x0 * ft.ld;
                const int64_t step = (int64_t)(256 / G) * ft.ld;
                const int rg = col_rot<N>(gs);
                int x = x0;
#pragma unroll 8
                for (int k = 0; k < T / (256 / G); ++k) {
                    int pos = (S == 4 && N >= 256 ? x ^ ((x >> 3) & 4) : x) + rg;   // < T + 32
                    if (pos >= T) pos -= T;
                    __stcs(dst, srcc[pos]);
                    dst += step;
                    x += 256 / G;
                }
            }
            return;
        }
        // all lanes take part in the shuffles below; only active signals store
        float* dst0 = ft.out + (active ? ft.s_out[g] : 0);
        // element l of phase buffer (o, u) holds samples s (2l) + u (real part) and
        // s (2l + 1) + u (imaginary part) of output o
        const bool al = (reinterpret_cast<uintptr_t>(dst0) & ((S % 2) == 0 ? 15 : 7)) == 0;
#pragma unroll
        for (int i = 0; i < PL::NB; ++i)
#pragma unroll
            for (int r = 0; r < PL::R; ++r) {
                const int l = jn + TPS * i + r * PL::ST;
                const int e = i * PL::R + r;
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const C* ph = &y[o * S][0];   // phase u of output o: ph[u * 8 + e]
                    if constexpr (S == 4) {
                        // the WG = min(32, N/8) lanes of a signal in this warp hold WG consecutive
                        // l, i.e. 32 WG contiguous bytes; store h writes the h-th half of them:
                        // lane x takes half (x & 1) of element WG h / 2 + x / 2, received by shuffles
                        constexpr int WG = TPS < 32 ? TPS : 32;
                        const int lane = threadIdx.x & 31, x = lane & (WG - 1);
                        const float4 re = make_float4(ph[e].x, ph[8 + e].x, ph[16 + e].x, ph[24 + e].x);
                        const float4 im = make_float4(ph[e].y, ph[8 + e].y, ph[16 + e].y, ph[24 + e].y);
                        float4* wbase = reinterpret_cast<float4*>(dst0 + (size_t)o * T + 2 * S * (l - x));
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int src = (lane - x) + (WG / 2) * h + (x >> 1);
                            const float4 lo = make_float4(__shfl_sync(0xffffffffu, re.x, src), __shfl_sync(0xffffffffu, re.y, src),
                                                          __shfl_sync(0xffffffffu, re.z, src), __shfl_sync(0xffffffffu, re.w, src));
                            const float4 hi = make_float4(__shfl_sync(0xffffffffu, im.x, src), __shfl_sync(0xffffffffu, im.y, src),
                                                          __shfl_sync(0xffffffffu, im.z, src), __shfl_sync(0xffffffffu, im.w, src));
                            if (al && active) __stcs(wbase + WG * h + x, (x & 1) ? hi : lo);
                        }
                        if (al) continue;
                    } else if constexpr (S == 2) {
                        if (al) {
                            if (active)
                                __stcs(reinterpret_cast<float4*>(dst0 + (size_t)o * T + 2 * S * l),
                                       make_float4(ph[e].x, ph[8 + e].x, ph[e].y, ph[8 + e].y));
                            continue;
                        }
                    }
                    if (!active) continue;
                    float* dst = dst0 + (size_t)o * T + 2 * S * l;
#pragma unroll
                    for (int u = 0; u < S; ++u) {
                        dst[u] = ph[u * 8 + e].x;
                        dst[S + u] = ph[u * 8 + e].y;
                    }
                }
            }
    }
}

// One CTA per tile of one size class.
template <int N, int MIN, int S, int NOUT>
__global__ void __launch_bounds__(256, 2) mci_fast_kernel(const KArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_in[kMaxTile];
    __shared__ int64_t s_out[kMaxTile];
    __shared__ int s_cnt;
    // image rows: a grid may exceed the class's tile count (bounded host launches)
    if (a.mode == kModeRows && (int)blockIdx.x >= a.sched2->row_count[a.cls]) return;
    const int list0 = a.mode == kModeRows ? a.sched2->row_start[a.cls] : 0;
    const int cnt = tile_signal_offsets(a, 2048 / N, blockIdx.x, list0, s_in, s_out, &s_cnt);
    const C* W = static_cast<const C*>(a.W);
    fast_tile<N, MIN, S, NOUT>(FastTile{W, W + a.c.tw_rel, static_cast<const float*>(a.in),
                                        static_cast<float*>(a.out), s_in, s_out, cnt},
                               smem_raw);
}

// One CTA per tile of G = 2048/N consecutive columns of one image's intermediate (the column
// pass of the separable 2-D path): item (image, tile) of the class's column list.
template <int N, int MIN, int S, int NOUT>
__global__ void __launch_bounds__(256, 2) mci_fast_cols_kernel(const KArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_in[kMaxTile];
    __shared__ int64_t s_out[kMaxTile];
    constexpr int G = 2048 / N;
    if ((int)blockIdx.x >= a.sched2->col_count[a.cls]) return;   // bounded host launches
    const int2 it = a.items[a.sched2->col_start[a.cls] + blockIdx.x];
    const int i = it.x;
    const int64_t ld = (int64_t)a.scale[i] * a.w[i];   // intermediate and HR row pitch
    const int64_t c0 = (int64_t)it.y * G;
    const int cnt = (int)min((int64_t)G, ld - c0);
    if (threadIdx.x == 0) {
        s_in[0] = a.inter_off[i] + c0;
        s_out[0] = a.img_out_off[i] + c0;
    }
    __syncthreads();
    const C* W = static_cast<const C*>(a.W);
    fast_tile<N, MIN, S, NOUT, true>(FastTile{W, W + a.c.tw_rel, static_cast<const float*>(a.in),
                                              static_cast<float*>(a.out), s_in, s_out, cnt, ld},
                                     smem_raw);
}

}  // namespace

// Fused variants (index, N, input channels, scale, outputs).  The first kFastPersistentVariants
// (the batched 1-D workload's classes) are also compiled into the persistent kernel.
#define MCI_FAST_VARIANTS(X) \
    X(0, 128, 3, 4, 1) X(1, 256, 3, 4, 1) X(2, 512, 3, 4, 1) X(3, 1024, 3, 4, 1) X(4, 2048, 3, 4, 1)
// image rows and columns: one channel (the derivative channels folded into the weights)
#define MCI_FAST_IMG_VARIANTS(X)                                                                \
    X(5, 128, 1, 2, 1) X(6, 256, 1, 2, 1) X(7, 512, 1, 2, 1) X(8, 128, 1, 3, 1) X(9, 256, 1, 3, 1) \
    X(10, 512, 1, 3, 1) X(11, 128, 1, 4, 1) X(12, 256, 1, 4, 1) X(13, 512, 1, 4, 1)

namespace {

// Tile `item` of the persistent launch: class order[oi] (its tiles start at s_t0[oi]),
// signals sorted[start + (item - s_t0[oi]) G ..]; their offsets and count go to shared memory
// (every thread stores the same oi and count).
__device__ __forceinline__ void persistent_item_signals(const PersistArgs& pa, const int* s_t0, int item,
                                                        int* oi_out, int64_t* s_in, int64_t* s_out, int* cnt)
{
    int oi = 0;
    while (oi + 1 < pa.n_classes && item >= s_t0[oi + 1]) ++oi;
    const int c = pa.order[oi];
    const ClassDev& cd = pa.cl[c].c;
    const int tile = item - s_t0[oi];
    const int n = min(cd.G, pa.sched->count[c] - tile * cd.G);
    *oi_out = oi;
    if (threadIdx.x < n) {
        const int64_t b = pa.sorted[pa.sched->start[c] + (int64_t)tile * cd.G + threadIdx.x];
        s_in[threadIdx.x] = pa.in_off ? pa.in_off[b] : b * cd.in_len;
        s_out[threadIdx.x] = pa.out_off ? pa.out_off[b] : b * cd.out_len;
    }
    *cnt = n;
}

// Persistent launch over all fused classes of an uneven batch.  The tiles are numbered class
// after class, largest P first (the small tiles fill the tail); the CTAs take them from the
// counter sched->next_tile, each claiming its next tile while it works on the current one.
__global__ void __launch_bounds__(256, 2) mci_fast_persistent(const PersistArgs pa)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_in[kMaxTile];
    __shared__ int64_t s_out[kMaxTile];
    __shared__ int s_t0[MCI_MAX_SIZES + 1];
    __shared__ int s_cnt, s_oi, s_item;
    if (threadIdx.x == 0) {
        int t = 0;
        for (int oi = 0; oi < pa.n_classes; ++oi) {
            s_t0[oi] = t;
            const int c = pa.order[oi];
            t += (pa.sched->count[c] + pa.cl[c].c.G - 1) / pa.cl[c].c.G;
        }
        s_t0[pa.n_classes] = t;
        s_item = (int)atomicAdd(&pa.sched->next_tile, 1u);
    }
    __syncthreads();
    const int total = s_t0[pa.n_classes];
    while (s_item < total) {
        persistent_item_signals(pa, s_t0, s_item, &s_oi, s_in, s_out, &s_cnt);
        __syncthreads();
        unsigned next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&pa.sched->next_tile, 1u);   // in flight meanwhile
        const ClassLaunch& L = pa.cl[pa.order[s_oi]];
        const C* W = static_cast<const C*>(L.W);
        const FastTile ft{W, W + L.c.tw_rel, pa.in, pa.out, s_in, s_out, s_cnt};
        switch (L.c.fast - 1) {
#define MCI_FAST_PCASE(v, n, m, sc, no) \
    case v: fast_tile<n, m, sc, no>(ft, smem_raw); break;
            MCI_FAST_VARIANTS(MCI_FAST_PCASE)
#undef MCI_FAST_PCASE
        }
        if (threadIdx.x == 0) s_item = (int)next;
        __syncthreads();   // buffers and the tile's offsets are free again; s_item is the next tile
    }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------
// Image columns with a factor 3: N = 3 N' (P = 6 N'), N' a power of two, one channel, one
// output, s phases.  The length-N packed transform is split by decimation in time into the
// three sub-sequences z[3 n + n1], whose length-N' transforms run as three vectors on the
// radix-8 passes above (N'/8 threads per column); a radix-3 step in registers combines them:
//   Z[k1 + N' k2] = sum_n1 e^{-2 pi i n1 k1 / N} e^{-2 pi i n1 k2 / 3} F_n1[k1].
// The inverse of each phase is the transpose: a radix-3 step (decimation in frequency, with
// the conjugate twiddles) and three inverse length-N' transforms, whose element n2 of
// sub-transform n1 is the complex sample n1 + 3 n2.  The mirror bins N - k of the real
// spectra are exchanged through shared memory in natural bin order.  The phases are produced
// one after another from the channel spectrum held in registers, so a column needs N complex
// values of shared memory: its staged input, the sub-transform buffers and one phase's
// output in turn.  G = 2048 / N' columns per CTA, staged as in the radix-8 column kernel.
// With N' = 64 (8 threads per column) two columns share each half warp; then the odd column
// of a pair stores its sub-transform buffers with the element index XOR 12 and its spectra
// with XOR 8, its staged words rotated by 16 more, and a warp stages 16 columns x 2 rows,
// which keeps every access of the pair free of bank conflicts.
// ---------------------------------------------------------------------------------------

// Staged-word rotation of column g, and the staging thread map (column, first row; rows step
// by 256 / G).
template <int NQ>
__device__ __forceinline__ int rot3(int g)
{
    if constexpr (NQ / 8 >= 16) return col_rot<NQ>(g);
    else return (16 * (g & 1) + 2 * (g >> 1)) & 31;
}
template <int NQ>
__device__ __forceinline__ int2 stage3(int t)
{
    constexpr int G = 2048 / NQ;
    if constexpr (G <= 16) return make_int2(t % G, t / G);
    else return make_int2((t & 15) + 16 * ((t >> 5) & 1), 2 * (t >> 6) + ((t >> 4) & 1));
}

template <int NQ, int S>
__global__ void __launch_bounds__(256, 2) mci_fast3_cols_kernel(const KArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int N = 3 * NQ, P = 2 * N, TPS = NQ / 8, G = 2048 / NQ, L = fast_passes(NQ);
    constexpr int RPI = 256 / G;   // rows per staging step
    static_assert(NQ >= 64 && NQ <= 256 && (NQ & (NQ - 1)) == 0 && (P * G) % 256 == 0, "factor-3 column class");
    if ((int)blockIdx.x >= a.sched2->col_count[a.cls]) return;   // bounded host launches
    const int2 item = a.items[a.sched2->col_start[a.cls] + blockIdx.x];
    const int img = item.x;
    const int64_t ld = (int64_t)a.scale[img] * a.w[img];   // intermediate and HR row pitch
    const int64_t c0 = (int64_t)item.y * G;
    const int cnt = (int)min((int64_t)G, ld - c0);
    const float* in = static_cast<const float*>(a.in) + a.inter_off[img] + c0;
    float* out = static_cast<float*>(a.out) + a.img_out_off[img] + c0;
    const C* W = static_cast<const C*>(a.W);
    const C* tab = W + a.c.tw_rel;                                  // e^{-2 pi i k / P}, k <= N
    const C* ptab = tab + (N + 1) - (NQ + 1);                      // pass twiddles (length N')
    const C* tw3 = tab + (N + 1) + fast_tw_count(NQ) - (NQ + 1);   // e^{-2 pi i k / N}, k < N'
    const int tid = threadIdx.x, g = tid / TPS, j = tid - g * TPS;
    C* sm = reinterpret_cast<C*>(smem_raw) + g * N;
    const int rot = rot3<NQ>(g);
    const bool odd = TPS < 16 && (g & 1);
    const int fx = odd ? 12 : 0, sx = odd ? 8 : 0;   // per-column index XORs (see above)

    // ---- rows p < P of the G columns into their buffers, rotated by col_rot words ----
    {
        const int2 m = stage3<NQ>(tid);
        const int gs = m.x, p0 = m.y;
        float* dstc = reinterpret_cast<float*>(reinterpret_cast<C*>(smem_raw) + gs * N);
        int q = p0 + rot3<NQ>(gs);
        if (gs < cnt) {
            const float* src = in + gs + (int64_t)p0 * ld;
            const int64_t step = (int64_t)RPI * ld;
#pragma unroll 8
            for (int k = 0; k < P / RPI; ++k) {
                dstc[q] = __ldcs(src);
                src += step;
                q += RPI;
                if (q >= P) q -= P;
            }
        } else {
#pragma unroll 8
            for (int k = 0; k < P / RPI; ++k) {
                dstc[q] = 0.f;
                q += RPI;
                if (q >= P) q -= P;
            }
        }
    }
    __syncthreads();

    // ---- forward pass 0 of the sub-transforms: sub-sequence n1 is z[3 n + n1] ----
    {
        using P0 = Pass<NQ, 0, false>;
        C x[3][8];
        const float* st = reinterpret_cast<const float*>(sm);
#pragma unroll
        for (int n1 = 0; n1 < 3; ++n1)
#pragma unroll
            for (int i = 0; i < P0::NB; ++i)
#pragma unroll
                for (int r = 0; r < P0::R; ++r) {
                    int pos = 6 * (j + TPS * i + r * P0::ST) + 2 * n1 + rot;
                    if (pos >= P) pos -= P;
                    const float2 v = *reinterpret_cast<const float2*>(st + pos);
                    x[n1][i * P0::R + r] = mk<float>(v.x, v.y);
                }
        sig_sync<NQ>(g);   // the staged column is read before pass 0 overwrites it
        P0::template compute<3>(x, j, ptab);
        P0::template store<3>(sm, j, x, fx);
        sig_sync<NQ>(g);
    }
    middle_passes<NQ, 3, 1, false>(sm, j, ptab, g, fx);

    // ---- last forward pass and the radix-3 step: z[k2][r] = Z[k1 + N' k2], k1 = j + TPS r ----
    C z[3][8];
    {
        using PL = Pass<NQ, L - 1, false>;
        static_assert(PL::R == 8, "the last forward pass is radix 8");
        PL::template load<3>(sm, j, z, fx);
        PL::template compute<3>(z, j, ptab);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const C w1 = ldc(tw3 + j + TPS * r), w2 = cmul(w1, w1);
            C v[3] = {z[0][r], cmul(z[1][r], w1), cmul(z[2][r], w2)};
            dft<3, false>(v);
            z[0][r] = v[0];
            z[1][r] = v[1];
            z[2][r] = v[2];
        }
    }
    // ---- real-input spectrum X[k] = (Z[k] + conj Z[N-k]) / 2 + e^{-2 pi i k / P} (Z[k] - conj Z[N-k]) / (2i)
    const float xN = z[0][0].x - z[0][0].y;   // X[N] (real), on the j = 0 lane
    sig_sync<NQ>(g);   // the last pass has read the sub-transform buffers
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
        for (int r = 0; r < 8; ++r) sm[(j + TPS * r + NQ * k2) ^ sx] = z[k2][r];
    sig_sync<NQ>(g);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int k = j + TPS * r + NQ * k2;
            const C zm = sm[(k == 0 ? 0 : N - k) ^ sx];
            const C e = scale(z[k2][r] + conjc(zm), 0.5f);
            const C d = z[k2][r] - conjc(zm);
            z[k2][r] = e + cmul(ldc(tab + k), mk<float>(0.5f * d.y, -0.5f * d.x));
        }

    // ---- output phases u < s, one at a time ----
#pragma unroll 1
    for (int u = 0; u < S; ++u) {
        // phase spectrum Y_u[k] = X[k] W_u[k] (Eq. (matrixeqn1) through the folded weights)
        const C* Wu = W + (size_t)u * (N + 1);
        C y[3][8];
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
            for (int r = 0; r < 8; ++r) y[k2][r] = cmul(z[k2][r], ldc(Wu + j + TPS * r + NQ * k2));
        const C yN = scale(ldc(Wu + N), xN);   // Y_u[N], used on the j = 0 lane
        sig_sync<NQ>(g);   // earlier reads of the column buffer are done
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
            for (int r = 0; r < 8; ++r) sm[(j + TPS * r + NQ * k2) ^ sx] = y[k2][r];
        sig_sync<NQ>(g);
        // packing for the real inverse FFT: A + i C, A = Y[k] + conj Y[N-k],
        // C = e^{2 pi i k / P} (Y[k] - conj Y[N-k])
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int k = j + TPS * r + NQ * k2;
                const C ym = k == 0 ? yN : sm[(N - k) ^ sx];
                const C A = y[k2][r] + conjc(ym);
                const C Cc = cmulc(y[k2][r] - conjc(ym), ldc(tab + k));
                y[k2][r] = mk<float>(A.x - Cc.y, A.y + Cc.x);
            }
        // radix-3 step of the inverse: G_n1[k1] = e^{2 pi i n1 k1 / N} sum_k2 Zp[k1 + N' k2] e^{2 pi i n1 k2 / 3},
        // then inverse pass 0 (stride 1) of sub-transform n1: butterfly j writes element r at 8 j + r
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const C w1 = ldc(tw3 + j + TPS * r), w2 = cmul(w1, w1);
            C v[3] = {y[0][r], y[1][r], y[2][r]};
            dft<3, true>(v);
            y[0][r] = v[0];
            y[1][r] = cmulc(v[1], w1);
            y[2][r] = cmulc(v[2], w2);
        }
#pragma unroll
        for (int n1 = 0; n1 < 3; ++n1) dft<8, true>(y[n1]);
        sig_sync<NQ>(g);   // every lane has read its mirror bins
#pragma unroll
        for (int n1 = 0; n1 < 3; ++n1)
#pragma unroll
            for (int r = 0; r < 8; ++r) sm[n1 * NQ + (swz<1, 8>(8 * j + r) ^ fx)] = y[n1][r];
        sig_sync<NQ>(g);
        middle_passes<NQ, 3, 1, true>(sm, j, ptab, g, fx);
        // last inverse pass: element n2 = j + TPS i + r ST of sub-transform n1 is the complex
        // sample n1 + 3 n2, i.e. the real samples m = 2 (n1 + 3 n2) and m + 1 of phase u,
        // staged at word m + rot (mod P) of the column buffer
        {
            using PL = Pass<NQ, L - 1, true>;
            PL::template load<3>(sm, j, y, fx);
            PL::template compute<3>(y, j, ptab);
            sig_sync<NQ>(g);
            float* oc = reinterpret_cast<float*>(sm);
#pragma unroll
            for (int n1 = 0; n1 < 3; ++n1)
#pragma unroll
                for (int i = 0; i < PL::NB; ++i)
#pragma unroll
                    for (int r = 0; r < PL::R; ++r) {
                        int pos = 2 * (n1 + 3 * (j + TPS * i + r * PL::ST)) + rot;
                        if (pos >= P) pos -= P;
                        const C v = y[n1][i * PL::R + r];
                        *reinterpret_cast<float2*>(oc + pos) = make_float2(v.x, v.y);
                    }
        }
        __syncthreads();
        // HR rows s m + u, m < P, of the G columns: thread tid writes column tid mod G,
        // m = tid / G + RPI k
        {
            const int2 m = stage3<NQ>(tid);
            const int gs = m.x, m0 = m.y;
            if (gs < cnt) {
                const float* srcc = reinterpret_cast<const float*>(reinterpret_cast<C*>(smem_raw) + gs * N);
                float* dst = out + gs + ((int64_t)S * m0 + u) * ld;
                const int64_t step = (int64_t)S * RPI * ld;
                int q = m0 + rot3<NQ>(gs);
#pragma unroll 8
                for (int k = 0; k < P / RPI; ++k) {
                    __stcs(dst, srcc[q]);
                    dst += step;
                    q += RPI;
                    if (q >= P) q -= P;
                }
            }
        }
        __syncthreads();   // the buffers are free for the next phase
    }
}

}  // namespace

// Factor-3 column variants (N', s).
#define MCI_FAST3_VARIANTS(X) X(64, 2) X(64, 3) X(64, 4) X(128, 2) X(128, 3) X(128, 4)

const void* fast3_cols_kernel_lookup(int N, int M_in, int s, int n_out)
{
    if (M_in != 1 || n_out != 1 || N % 3 != 0) return nullptr;
#define MCI_FAST3_CASE(nq, sc) \
    if (N == 3 * nq && s == sc) return (const void*)mci_fast3_cols_kernel<nq, sc>;
    MCI_FAST3_VARIANTS(MCI_FAST3_CASE)
#undef MCI_FAST3_CASE
    return nullptr;
}

__device__ bool device_launch_fast3_cols(const ClassDev& c, int grid, int smem, const KArgs& a)
{
#define MCI_FAST3_DCASE(nq, sc)                                                             \
    if (c.N == 3 * nq && c.s == sc) {                                                       \
        mci_fast3_cols_kernel<nq, sc><<<grid, 256, smem, cudaStreamFireAndForget>>>(a);     \
        return true;                                                                        \
    }
    MCI_FAST3_VARIANTS(MCI_FAST3_DCASE)
#undef MCI_FAST3_DCASE
    return false;
}

const void* fast_kernel_lookup(int N, int M_in, int s, int n_out, int* variant)
{
#define MCI_FAST_CASE(v, n, m, sc, no)                              \
    if (N == n && M_in == m && s == sc && n_out == no) {             \
        if (variant) *variant = v;                                   \
        return (const void*)mci_fast_kernel<n, m, sc, no>;           \
    }
    MCI_FAST_VARIANTS(MCI_FAST_CASE)
    MCI_FAST_IMG_VARIANTS(MCI_FAST_CASE)
#undef MCI_FAST_CASE
    return nullptr;
}

const void* fast_cols_kernel_lookup(int N, int M_in, int s, int n_out)
{
#define MCI_FAST_CCASE(v, n, m, sc, no) \
    if (N == n && M_in == m && s == sc && n_out == no) return (const void*)mci_fast_cols_kernel<n, m, sc, no>;
    MCI_FAST_IMG_VARIANTS(MCI_FAST_CCASE)
#undef MCI_FAST_CCASE
    return nullptr;
}

const void* fast_persistent_kernel() { return (const void*)mci_fast_persistent; }

// Device-side launch of a fused-path class (dynamic parallelism, from the scheduler).
__device__ bool device_launch_fast(const ClassDev& c, int grid, int smem, const KArgs& a)
{
#define MCI_FAST_DCASE(v, n, m, sc, no)                                                       \
    if (c.N == n && c.M_in == m && c.s == sc && c.n_out == no) {                               \
        mci_fast_kernel<n, m, sc, no><<<grid, 256, smem, cudaStreamFireAndForget>>>(a);        \
        return true;                                                                          \
    }
    MCI_FAST_VARIANTS(MCI_FAST_DCASE)
    MCI_FAST_IMG_VARIANTS(MCI_FAST_DCASE)
#undef MCI_FAST_DCASE
    return false;
}

__device__ bool device_launch_fast_cols(const ClassDev& c, int grid, int smem, const KArgs& a)
{
#define MCI_FAST_DCCASE(v, n, m, sc, no)                                                      \
    if (c.N == n && c.M_in == m && c.s == sc && c.n_out == no) {                               \
        mci_fast_cols_kernel<n, m, sc, no><<<grid, 256, smem, cudaStreamFireAndForget>>>(a);   \
        return true;                                                                          \
    }
    MCI_FAST_IMG_VARIANTS(MCI_FAST_DCCASE)
#undef MCI_FAST_DCCASE
    return false;
}

}  // namespace mci
