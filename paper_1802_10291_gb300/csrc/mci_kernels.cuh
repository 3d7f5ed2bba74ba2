// Interpolation kernels, one instantiation per (precision, FFT length, access
// pattern).  A launch serves one size class with one CTA per tile (G signals,
// image rows or image columns each); its grid is the class's tile count.
#pragma once
#include "mci_tile.cuh"

namespace mci {

// Signals of a contiguous-signal tile (1-D modes and image rows): their count (returned,
// at most G) and their input and output offsets in s_in[g], s_out[g] (shared memory).
// All threads call it; it ends with a barrier.
__device__ __forceinline__ int tile_signal_offsets(const KArgs& a, int G, int item, int list0,
                                                   int64_t* s_in, int64_t* s_out, int* s_cnt)
{
    const ClassDev& c = a.c;
    if (threadIdx.x == 0) {
        int cnt;
        if (a.mode == kModeUniform) {
            cnt = (int)min((int64_t)G, a.batch - (int64_t)item * G);
        } else if (a.mode == kModeSorted) {
            cnt = min(G, a.sched1->count[a.cls] - item * G);
        } else {
            const int2 it = a.items[list0 + item];
            cnt = min(G, a.h[it.x] - it.y * G);
        }
        *s_cnt = cnt;
    }
    __syncthreads();
    const int cnt = *s_cnt;
    if (threadIdx.x < cnt) {
        const int g = threadIdx.x;
        if (a.mode == kModeRows) {
            const int2 it = a.items[list0 + item];
            const int i = it.x, r = it.y * G + g;
            s_in[g] = a.img_in_off[i] + (int64_t)r * a.w[i];
            s_out[g] = a.inter_off[i] + (int64_t)r * c.T;
        } else {
            const int64_t b = a.mode == kModeSorted ? a.sorted[a.sched1->start[a.cls] + (int64_t)item * G + g]
                                                    : (int64_t)item * G + g;
            s_in[g] = a.in_off ? a.in_off[b] : b * c.in_len;
            s_out[g] = a.out_off ? a.out_off[b] : b * c.out_len;
        }
    }
    __syncthreads();
    return cnt;
}

// One tile (one work item) of a size-class launch.
template <typename R, int N, bool COLS>
__device__ __forceinline__ void mci_tile_item(const KArgs& a, int item, int list0, cpx<R>* sm)
{
    __shared__ int64_t s_in[kMaxTile];
    __shared__ int64_t s_out[kMaxTile];
    __shared__ int s_cnt;
    const ClassDev& c = a.c;
    const cpx<R>* W = static_cast<const cpx<R>*>(a.W);
    const int G = c.G;
    if constexpr (COLS) {
        const int2 it = a.items[list0 + item];
        const int i = it.x;
        const int64_t ld = (int64_t)a.scale[i] * a.w[i];  // intermediate and HR row pitch
        const int c0 = it.y * G;
        const int cnt = (int)min((int64_t)G, ld - c0);
        load_cols<R>(sm, c, static_cast<const R*>(a.in), a.inter_off[i] + c0, ld, cnt);
        __syncthreads();
        compute_tile<R, N>(sm, c, cnt, W);
        store_cols<R>(sm, c, static_cast<R*>(a.out), a.img_out_off[i] + c0, ld, cnt);
        __syncthreads();
    } else {
        const int cnt = tile_signal_offsets(a, G, item, list0, s_in, s_out, &s_cnt);
        // signals whose complex pairs are 8-byte aligned are read by the first FFT pass
        // directly; others are staged in shared memory first
        bool direct = c.cplx || (c.P % 2) == 0;
        for (int g = 0; g < cnt; ++g)
            direct = direct && ((reinterpret_cast<uintptr_t>(static_cast<const R*>(a.in) + s_in[g]) &
                                 (2 * sizeof(R) - 1)) == 0);
        // phases of this CTA: all, or the blockIdx.y-th of qchunks shares (real signals)
        int q0 = 0, q1 = c.Q;
        if (a.qchunks > 1 && !c.cplx) {
            const int per = (c.Q + a.qchunks - 1) / a.qchunks;
            q0 = min(c.Q, (int)blockIdx.y * per);
            q1 = min(c.Q, q0 + per);
        }
        if (direct) {
            compute_tile<R, N>(sm, c, cnt, W, static_cast<const R*>(a.in), s_in, q0, q1);
        } else {
            load_contig<R>(sm, c, static_cast<const R*>(a.in), s_in, cnt);
            __syncthreads();
            compute_tile<R, N>(sm, c, cnt, W, nullptr, nullptr, q0, q1);
        }
        if (c.cplx) store_contig_complex<R, N>(sm, c, static_cast<R*>(a.out), s_out, cnt);
        else store_contig<R, N>(sm, c, static_cast<R*>(a.out), s_out, cnt, q0, q1);
        __syncthreads();
    }
}

// One CTA per tile.  (A persistent tile loop makes the compiler keep the tile's
// index arithmetic live across iterations and spill; single-tile CTAs need no
// spills.)  Launches size their grid to the class's tile count, from the host
// for uniform batches, from the device-side scheduler otherwise.
template <typename R, int N, bool COLS>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 2) mci_kernel(const KArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    int list0 = 0;
    // image passes: a grid may exceed the class's tile count (host launches sized by a bound
    // for device-grouped batches); the extra CTAs leave at once
    if (a.mode == kModeRows) {
        if ((int)blockIdx.x >= a.sched2->row_count[a.cls]) return;
        list0 = a.sched2->row_start[a.cls];
    } else if (a.mode == kModeCols) {
        if ((int)blockIdx.x >= a.sched2->col_count[a.cls]) return;
        list0 = a.sched2->col_start[a.cls];
    }
    mci_tile_item<R, N, COLS>(a, blockIdx.x, list0, sm);
}

// Kernel lookup (host) for the lengths of one translation unit.
#define MCI_KERNEL_CASE(n)                                                                      \
    case n:                                                                                     \
        if (prec == MCI_FP64) return cols ? nullptr : (const void*)mci_kernel<double, n, false>; \
        return cols ? (const void*)mci_kernel<float, n, true> : (const void*)mci_kernel<float, n, false>;

// Device-side launch (dynamic parallelism) for the lengths of one translation unit.
#define MCI_DEVICE_LAUNCH_CASE(n)                                                               \
    case n:                                                                                     \
        if (prec == MCI_FP64) {                                                                 \
            if (cols) return false;                                                             \
            mci_kernel<double, n, false><<<grid, kThreads, smem, cudaStreamFireAndForget>>>(a); \
        } else if (cols) {                                                                      \
            mci_kernel<float, n, true><<<grid, kThreads, smem, cudaStreamFireAndForget>>>(a);   \
        } else {                                                                                \
            mci_kernel<float, n, false><<<grid, kThreads, smem, cudaStreamFireAndForget>>>(a);  \
        }                                                                                       \
        return true;

}  // namespace mci
