// Device-side scheduling: batches whose composition lives only in device memory
// (a size class per 1-D signal, a size per image) are grouped by size class on
// the device, and every class's kernel is launched from the device with a grid
// of exactly its tile count (dynamic parallelism), so a call needs no host
// round trip.  Each scheduler is one CTA.
#include <cuda_runtime.h>

#include "mci_internal.h"

namespace mci {

constexpr int kSchedThreads = 1024;

__device__ bool device_launch_a(int prec, bool cols, int N, int grid, int smem, const KArgs& a);
__device__ bool device_launch_b(int prec, bool cols, int N, int grid, int smem, const KArgs& a);
__device__ bool device_launch_c(int prec, bool cols, int N, int grid, int smem, const KArgs& a);
__device__ bool device_launch_d(int prec, bool cols, int N, int grid, int smem, const KArgs& a);
__device__ bool device_launch_e(int prec, bool cols, int N, int grid, int smem, const KArgs& a);

__device__ bool device_launch_fast(const ClassDev& c, int grid, int smem, const KArgs& a);
__device__ bool device_launch_fast_cols(const ClassDev& c, int grid, int smem, const KArgs& a);
__device__ bool device_launch_fast3_cols(const ClassDev& c, int grid, int smem, const KArgs& a);

__device__ void launch_class(const ClassLaunch& L, bool cols, int grid, const KArgs& a, int* status)
{
    const int sm = cols ? L.smem_cols : L.smem;
    bool ok = L.c.fast ? (cols ? device_launch_fast_cols(L.c, grid, sm, a) : device_launch_fast(L.c, grid, sm, a)) :
              cols && L.c.fast3 ? device_launch_fast3_cols(L.c, grid, sm, a) :
              device_launch_a(L.prec, cols, L.c.N, grid, sm, a) ||
              device_launch_b(L.prec, cols, L.c.N, grid, sm, a) ||
              device_launch_c(L.prec, cols, L.c.N, grid, sm, a) ||
              device_launch_d(L.prec, cols, L.c.N, grid, sm, a) ||
              device_launch_e(L.prec, cols, L.c.N, grid, sm, a);
    if (!ok || cudaGetLastError() != cudaSuccess) atomicOr(status, kStatusLaunch);
}

// Block-wide exclusive scan of one int64 per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* out_excl)
{
    __shared__ int64_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const int64_t before = wid ? warp_tot[wid - 1] : 0;
    *out_excl = before + x - v;
    const int64_t total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------------------
// 1-D: counting sort of the signals by size class, packed offsets when the
// caller passed none, then one launch per non-empty class (largest P first).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSchedThreads)
sched_1d_kernel(const int* __restrict__ size_class, int64_t batch, int n_classes,
                const ClassLaunch* __restrict__ cl, const int* __restrict__ order,
                int64_t* __restrict__ sorted, Sched1D* __restrict__ st, int64_t* in_pref,
                int64_t* out_pref, KArgs tmpl, int persist)
{
    __shared__ int cnt[MCI_MAX_SIZES], cursor[MCI_MAX_SIZES], start[MCI_MAX_SIZES];
    if (threadIdx.x < MCI_MAX_SIZES) {
        cnt[threadIdx.x] = 0;
        cursor[threadIdx.x] = 0;
    }
    __syncthreads();
    int bad = 0;
    for (int64_t b = threadIdx.x; b < batch; b += blockDim.x) {
        const int c = size_class[b];
        if (c < 0 || c >= n_classes) bad = 1;
        else atomicAdd(&cnt[c], 1);
    }
    if (bad) atomicOr(tmpl.status, kStatusBadClass);
    __syncthreads();
    if (threadIdx.x == 0) {
        int pos = 0;
        for (int oi = 0; oi < n_classes; ++oi) {
            const int c = order[oi];
            start[c] = pos;
            st->start[c] = pos;
            st->count[c] = cnt[c];
            pos += cnt[c];
        }
    }
    __syncthreads();
    for (int64_t b = threadIdx.x; b < batch; b += blockDim.x) {
        const int c = size_class[b];
        if (c >= 0 && c < n_classes) sorted[start[c] + atomicAdd(&cursor[c], 1)] = b;
    }
    if (in_pref || out_pref) {
        int64_t carry_in = 0, carry_out = 0;
        for (int64_t base = 0; base < batch; base += blockDim.x) {
            const int64_t b = base + threadIdx.x;
            const int c = b < batch ? size_class[b] : -1;
            const bool ok = c >= 0 && c < n_classes;
            int64_t ex;
            const int64_t tin = block_exclusive_scan(ok ? cl[c].c.in_len : 0, &ex);
            if (b < batch && in_pref) in_pref[b] = carry_in + ex;
            carry_in += tin;
            const int64_t tout =
                block_exclusive_scan(ok ? cl[c].c.out_len : 0, &ex);
            if (b < batch && out_pref) out_pref[b] = carry_out + ex;
            carry_out += tout;
        }
    }
    __threadfence();
    __syncthreads();
    if (persist) {   // the host launches the persistent kernel next, stream-ordered
        if (threadIdx.x == 0) st->next_tile = 0;
        return;
    }
    if (threadIdx.x == 0) {
        for (int oi = 0; oi < n_classes; ++oi) {
            const int c = order[oi];
            if (cnt[c] == 0) continue;
            KArgs a = tmpl;
            a.c = cl[c].c;
            a.cls = c;
            a.W = cl[c].W;
            a.mode = kModeSorted;
            if (!a.in_off) a.in_off = in_pref;
            if (!a.out_off) a.out_off = out_pref;
            launch_class(cl[c], false, (cnt[c] + cl[c].c.G - 1) / cl[c].c.G, a, tmpl.status);
        }
    }
}

int launch_sched_1d(const int* size_class, int64_t batch, int n_classes, const ClassLaunch* cl,
                    const int* order, int64_t* sorted, Sched1D* st, int64_t* in_pref,
                    int64_t* out_pref, const KArgs& tmpl, void* stream, int persist)
{
    sched_1d_kernel<<<1, kSchedThreads, 0, (cudaStream_t)stream>>>(
        size_class, batch, n_classes, cl, order, sorted, st, in_pref, out_pref, tmpl, persist);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 2-D: per image the row and column size classes, the intermediate offsets,
// packed LR/HR offsets when the caller passed none, and per class the lists of
// (image, tile) items; then the row-pass launches.  The column pass is
// launched by dispatch_cols_kernel, stream-ordered after this kernel and its
// children.
// ---------------------------------------------------------------------------
__device__ int lookup_class(const ClassLaunch* cl, int n, int P, int64_t T)
{
    for (int c = 0; c < n; ++c)
        if (cl[c].c.P == P && cl[c].c.T == T) return c;
    return -1;
}

__global__ void __launch_bounds__(kSchedThreads)
sched_2d_kernel(int64_t n_img, int n_classes, const ClassLaunch* __restrict__ cl,
                int64_t max_inter, int64_t max_items, int64_t* inter_off, int64_t* lr_pref,
                int64_t* hr_pref, int* row_cls, int* col_cls, int2* items, Sched2D* st,
                KArgs tmpl, int child)
{
    __shared__ int rcnt[MCI_MAX_SIZES], ccnt[MCI_MAX_SIZES];
    __shared__ int rcur[MCI_MAX_SIZES], ccur[MCI_MAX_SIZES];
    __shared__ int ok_all;
    if (threadIdx.x < MCI_MAX_SIZES) {
        rcnt[threadIdx.x] = ccnt[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) ok_all = 1;
    __syncthreads();
    const int* h = tmpl.h;
    const int* w = tmpl.w;
    const int* scale = tmpl.scale;
    int64_t carry_inter = 0, carry_lr = 0, carry_hr = 0;
    int bad = 0;
    for (int64_t base = 0; base < n_img; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int64_t inter = 0, lr = 0, hr = 0;
        if (i < n_img) {
            const int hi = h[i], wi = w[i], si = scale[i];
            int rc = -1, cc = -1;
            if (hi > 0 && wi > 0 && si > 0) {
                rc = lookup_class(cl, n_classes, wi, (int64_t)si * wi);
                cc = lookup_class(cl, n_classes, hi, (int64_t)si * hi);
                lr = (int64_t)hi * wi;
                hr = (int64_t)si * si * hi * wi;
            }
            if (rc < 0 || cc < 0) {
                bad = 1;
                rc = cc = -1;
            } else {
                inter = (int64_t)hi * si * wi;
                atomicAdd(&rcnt[rc], (hi + cl[rc].c.G - 1) / cl[rc].c.G);
                atomicAdd(&ccnt[cc], (int)(((int64_t)si * wi + cl[cc].c.Gc - 1) / cl[cc].c.Gc));
            }
            row_cls[i] = rc;
            col_cls[i] = cc;
        }
        int64_t ex;
        int64_t t = block_exclusive_scan(inter, &ex);
        if (i < n_img) inter_off[i] = carry_inter + ex;
        carry_inter += t;
        t = block_exclusive_scan(lr, &ex);
        if (i < n_img && lr_pref) lr_pref[i] = carry_lr + ex;
        carry_lr += t;
        t = block_exclusive_scan(hr, &ex);
        if (i < n_img && hr_pref) hr_pref[i] = carry_hr + ex;
        carry_hr += t;
    }
    if (bad) atomicOr(tmpl.status, kStatusBadImage);
    __syncthreads();
    if (threadIdx.x == 0) {
        int pos = 0;
        for (int c = 0; c < n_classes; ++c) {
            st->row_start[c] = pos;
            rcur[c] = pos;
            pos += rcnt[c];
        }
        for (int c = 0; c < n_classes; ++c) {
            st->col_start[c] = pos;
            ccur[c] = pos;
            pos += ccnt[c];
        }
        if (carry_inter > max_inter || pos > max_items) {
            atomicOr(tmpl.status, kStatusIntermediate);
            ok_all = 0;
        }
        for (int c = 0; c < n_classes; ++c) {
            st->row_count[c] = ok_all ? rcnt[c] : 0;
            st->col_count[c] = ok_all ? ccnt[c] : 0;
        }
    }
    __syncthreads();
    if (ok_all) {
        for (int64_t i = threadIdx.x; i < n_img; i += blockDim.x) {
            const int rc = row_cls[i], cc = col_cls[i];
            if (rc < 0) continue;
            const int nr = (h[i] + cl[rc].c.G - 1) / cl[rc].c.G;
            const int nc = (int)(((int64_t)scale[i] * w[i] + cl[cc].c.Gc - 1) / cl[cc].c.Gc);
            int p = atomicAdd(&rcur[rc], nr);
            for (int t = 0; t < nr; ++t) items[p + t] = make_int2((int)i, t);
            p = atomicAdd(&ccur[cc], nc);
            for (int t = 0; t < nc; ++t) items[p + t] = make_int2((int)i, t);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && ok_all && child) {
        for (int c = 0; c < n_classes; ++c) {
            if (rcnt[c] == 0) continue;
            KArgs a = tmpl;
            a.c = cl[c].c;
            a.cls = c;
            a.W = cl[c].W;
            a.mode = kModeRows;
            launch_class(cl[c], false, rcnt[c], a, tmpl.status);
        }
    }
}

__global__ void dispatch_cols_kernel(int n_classes, const ClassLaunch* __restrict__ cl,
                                     const Sched2D* __restrict__ st, KArgs tmpl)
{
    if (threadIdx.x != 0) return;
    for (int c = 0; c < n_classes; ++c) {
        const int n = st->col_count[c];
        if (n == 0) continue;
        KArgs a = tmpl;
        a.c = cl[c].c;
        a.cls = c;
        a.W = cl[c].W;
        a.mode = kModeCols;
        launch_class(cl[c], true, n, a, tmpl.status);
    }
}

int launch_sched_2d(int64_t n_img, int n_classes, const ClassLaunch* cl, int64_t max_inter,
                    int64_t max_items, int64_t* inter_off, int64_t* lr_pref, int64_t* hr_pref,
                    int* row_cls, int* col_cls, int2* items, Sched2D* st, const KArgs& rows_tmpl,
                    const KArgs& cols_tmpl, void* stream, int child)
{
    cudaStream_t s = (cudaStream_t)stream;
    sched_2d_kernel<<<1, kSchedThreads, 0, s>>>(n_img, n_classes, cl, max_inter, max_items,
                                                 inter_off, lr_pref, hr_pref, row_cls, col_cls,
                                                 items, st, rows_tmpl, child);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !child) return (int)e;
    dispatch_cols_kernel<<<1, 32, 0, s>>>(n_classes, cl, st, cols_tmpl);
    return (int)cudaGetLastError();
}

}  // namespace mci
