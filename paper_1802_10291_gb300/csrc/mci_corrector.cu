// Learned residual corrector on top of MCI upsampling, and an on-device
// generator of the synthetic training images.
//
// Network: pred = mci + f(mci), f = conv5 o relu o conv4 o relu o conv3 o relu o
// conv2 o relu o conv1, every conv 3x3 with bias and periodic padding (images
// are periodic in the interpolation model), channels 1 -> 32 -> 32 -> 32 -> 32 -> 1.
// Weights are BF16 in the forward and backward passes (FP32 master copies in
// the optimizer), activations and accumulation FP32.  Loss: mean squared error
// of pred against the HR image.  Training: Adam.
//
// Kernels (CUDA cores on 16 x 16 pixel tiles, except the 32 -> 32 convolutions, which
// run on the tensor cores; see conv32_tc_kernel):
//   conv_fwd      out[co] = b[co] + sum_ci sum_taps w[co][ci][t] x[ci](p + d_t), optional
//                 ReLU, optional residual add;
//   conv_bwd_data gin[ci] = (sum_co sum_taps w[co][ci][t] g[co](p - d_t)) * (h[ci](p) > 0),
//                 h the ReLU output of the layer below (the same kernel with the weights
//                 transposed, the taps reversed and an output mask);
//   conv_bwd_w    gw[co][ci][t] = sum_p g[co](p) x[ci](p + d_t), gb[co] = sum_p g[co](p):
//                 32 -> 32 layers on the tensor cores (wgrad32_tc_kernel), the 1 -> 32 and
//                 32 -> 1 layers register-blocked on CUDA cores, persistent CTAs reduced
//                 with atomics;
//   mse, adam, image generator.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mci_corrector.h"
#include "tc_ptx.cuh"

namespace {

constexpr int kTile = 16;          // output tile edge
constexpr int kHalo = kTile + 2;   // input tile edge
constexpr int kCThreads = kTile * kTile;
constexpr int kWide = 32;          // hidden channels
constexpr int kLayers = 5;
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 1 : kWide; }
__host__ __device__ constexpr int cout_of(int l) { return l == kLayers - 1 ? 1 : kWide; }

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------------------
// forward conv (also the data-gradient conv): COUT output channels per pixel
// ---------------------------------------------------------------------------
// x: [B][cin][H][W]; w: bf16 [COUT][cin][9] (forward) -- when transposed_w, the weights
// are read as w[ci][co][8 - t] from a [cin_fwd = COUT... ] tensor laid out [cin][COUT][9]
// (i.e. the forward tensor of the layer whose data gradient this is).
// out_mask: optional [B][COUT][H][W]; outputs where out_mask <= 0 are zeroed (the ReLU
// derivative of the layer below, applied to a data gradient).
template <int COUT>
__global__ void __launch_bounds__(kCThreads) conv3x3_kernel(
    const float* __restrict__ x, int cin, const __nv_bfloat16* __restrict__ w, bool transposed_w,
    const float* __restrict__ bias, const float* __restrict__ out_mask, const float* __restrict__ res,
    float* __restrict__ out, int H, int W, bool relu)
{
    extern __shared__ float csm[];
    float* xs = csm;                          // [cin][18][18]
    float* ws = csm + cin * kHalo * kHalo;    // [cin][9][COUT]
    const int b = blockIdx.z;
    const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
    const int tid = threadIdx.x;
    const int64_t plane = (int64_t)H * W;
    for (int i = tid; i < cin * kHalo * kHalo; i += kCThreads) {
        const int ci = i / (kHalo * kHalo), r = i % (kHalo * kHalo);
        const int yy = wrap(y0 + r / kHalo - 1, H), xx = wrap(x0 + r % kHalo - 1, W);
        xs[i] = x[((int64_t)b * cin + ci) * plane + (int64_t)yy * W + xx];
    }
    for (int i = tid; i < cin * 9 * COUT; i += kCThreads) {
        const int ci = i / (9 * COUT), t = (i / COUT) % 9, co = i % COUT;
        const float wv = transposed_w ? __bfloat162float(w[((int64_t)ci * COUT + co) * 9 + (8 - t)])
                                      : __bfloat162float(w[((int64_t)co * cin + ci) * 9 + t]);
        ws[i] = wv;
    }
    __syncthreads();
    const int ty = tid / kTile, tx = tid % kTile;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.f;
    for (int ci = 0; ci < cin; ++ci) {
        const float* xc = xs + ci * kHalo * kHalo;
        const float* wc = ws + ci * 9 * COUT;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float v = xc[(ty + t / 3) * kHalo + tx + t % 3];
            if constexpr (COUT % 4 == 0) {
#pragma unroll
                for (int co = 0; co < COUT; co += 4) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wc + t * COUT + co);
                    acc[co] += v * w4.x;
                    acc[co + 1] += v * w4.y;
                    acc[co + 2] += v * w4.z;
                    acc[co + 3] += v * w4.w;
                }
            } else {
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] += v * wc[t * COUT + co];
            }
        }
    }
    const int y = y0 + ty, xq = x0 + tx;
    if (y < H && xq < W) {
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            const int64_t o = ((int64_t)b * COUT + co) * plane + (int64_t)y * W + xq;
            float v = acc[co];
            if (relu) v = fmaxf(v, 0.f);
            if (res) v += res[o];
            if (out_mask && !(out_mask[o] > 0.f)) v = 0.f;
            out[o] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// 32 -> 32 channel 3x3 conv on the tensor cores (tcgen05), used for the hidden
// layers' forward convs and their data-gradient convs.
//
// Implicit GEMM per tile of 4 image rows x 32 pixels (M = 128 pixels, N = 32
// output channels): out[p][co] = sum over taps t and input channels ci of
// A_t[p][ci] B_t[co][ci], A_t[p] = x(p + d_t).  The FP32 input is split as
// x = hi + lo, two BF16 values, and one pixel row of A holds [hi(ci 0..31) |
// lo(ci 0..31)] (64 BF16 = one 128-byte swizzle row); B_t rows hold the BF16
// weights twice, [w(ci 0..31) | w(ci 0..31)], so one K = 64 contraction gives
// hi*w + lo*w with FP32 accumulation (the weights are exact in BF16, the
// split leaves an input error near 2^-17 relative).  Shared memory holds three
// copies of the tile's 6 x 32 halo rows shifted by dx = -1, 0, +1; the A
// operand of tap (dy, dx) is rows (dy + 1) * 32 .. + 127 of copy dx, which
// starts on a 1024-byte swizzle-atom boundary, so every tap is a plain
// descriptor offset.  Nine taps x four K = 16 MMAs per tile, issued by one
// thread into four partial accumulators (one per K step, so consecutive MMAs are
// independent), summed when the accumulator (128 lanes x 4 x 32 FP32 columns of
// tensor memory, two buffers) is read back with tcgen05.ld.  Persistent CTAs of 9
// warps (8 stage and store, one issues the MMAs), two per SM (256 of the 512
// tensor-memory columns each).
// ---------------------------------------------------------------------------
constexpr int kTcWorkers = 256;                              // staging and epilogue warps 0..7
constexpr int kTcThreads = kTcWorkers + 32;                  // + warp 8: issues the MMAs
constexpr int kTcRows = 4, kTcCols = 32;                       // 4 x 32 = 128 MMA rows
constexpr int kTcHaloRows = kTcRows + 2;
constexpr int kTcHaloCols = kTcCols + 2;                       // 6 x 34 = 204 halo pixels
constexpr int kTcCopyBytes = kTcHaloRows * kTcCols * 128;      // one dx-shifted copy
constexpr int kTcTapBytes = kWide * 128;                       // one tap's weights
constexpr int kTcSmem = 3 * kTcCopyBytes + 9 * kTcTapBytes + 1024;
constexpr int kTcParts = 4;                                    // independent accumulation chains
constexpr int kTcTmemCols = 2 * kTcParts * 32;                 // two tiles in flight

__device__ __forceinline__ int wrapg(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ uint32_t bf16_pair_bits(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Software pipeline over a CTA's tiles k = 0, 1, ...: stage tile k from registers into
// the A copies, issue its MMAs into accumulator buffer k mod 2, issue the global loads
// of tile k + 1 into registers, run the epilogue of tile k - 1 from the other buffer,
// then wait for tile k's MMAs.  Loads, MMAs and stores of neighbouring tiles overlap.
// Each of the first 204 threads owns one halo pixel of every tile.
__global__ void __launch_bounds__(kTcThreads, 2) conv32_tc_kernel(
    const float* __restrict__ x, const __nv_bfloat16* __restrict__ w, bool transposed_w,
    const float* __restrict__ bias, const float* __restrict__ out_mask, float* __restrict__ out, int B,
    int H, int W, bool relu, int* status)
{
    using namespace mci;
    extern __shared__ __align__(1024) unsigned char tsm_raw[];
    char* sbase = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~uintptr_t(1023));
    char* Acp = sbase;                        // copies dx = -1, 0, +1
    char* Bw = sbase + 3 * kTcCopyBytes;      // taps 0..8
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;

    // B_t[co][.] = [w(co, ci = 0..31, t) | the same], BF16 bits copied as they are
    for (int i = tid; i < 9 * kWide * 4; i += kTcThreads) {
        const int t = i / (kWide * 4), co = (i >> 2) % kWide, j = i & 3;
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c0 = j * 8 + 2 * e;
            __nv_bfloat16 v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ci = c0 + h;
                v[h] = transposed_w ? w[((int64_t)ci * kWide + co) * 9 + (8 - t)]
                                    : w[((int64_t)co * kWide + ci) * 9 + t];
            }
            pk[e] = bf16_pair_bits(v[0], v[1]);
        }
        const uint4 q = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        char* tap = Bw + t * kTcTapBytes;
        *reinterpret_cast<uint4*>(tap + sw128_offset(co, j * 8)) = q;
        *reinterpret_cast<uint4*>(tap + sw128_offset(co, kWide + j * 8)) = q;
    }
    if (warp == 0) {   // two buffers of four 32-column partial accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(kTcTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_bf16_f32(128, kWide);

    const int64_t plane = (int64_t)H * W;
    const int tiles_x = (W + kTcCols - 1) / kTcCols, tiles_y = (H + kTcRows - 1) / kTcRows;
    const int n_tiles = B * tiles_y * tiles_x;
    // threads 0..191: halo rows 0..5 x columns 1..32 (warp w loads row w: every channel
    // row segment is one aligned 128-byte line); threads 192..203: the edge columns 0, 33
    const bool has_item = tid < kTcHaloRows * kTcHaloCols;
    const int r_it = tid < kTcHaloRows * kTcCols ? tid / kTcCols : (tid - kTcHaloRows * kTcCols) >> 1;
    const int h_it = tid < kTcHaloRows * kTcCols ? tid % kTcCols + 1 : ((tid & 1) ? kTcHaloCols - 1 : 0);
    auto tile_origin = [&](int tile, int& b, int& y0, int& x0) {
        b = tile / (tiles_y * tiles_x);
        const int r2 = tile - b * tiles_y * tiles_x;
        y0 = (r2 / tiles_x) * kTcRows;
        x0 = (r2 % tiles_x) * kTcCols;
    };
    // halo pixel (r, h) = image pixel (y0 - 1 + r, x0 - 1 + h), periodic
    float v[kWide];
    auto load_tile = [&](int tile) {
        if (!has_item || tile >= n_tiles) return;
        int b, y0, x0;
        tile_origin(tile, b, y0, x0);
        const float* src = x + (int64_t)b * kWide * plane + (int64_t)wrapg(y0 - 1 + r_it, H) * W +
                           wrapg(x0 - 1 + h_it, W);
#pragma unroll
        for (int c = 0; c < kWide; ++c) v[c] = __ldg(src + c * plane);
    };
    // split into hi + lo BF16 and store as row r * 32 + (h - 1 - dx) of copy dx
    auto stage = [&]() {
        if (!has_item) return;
        uint4 hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t ph[4], pl[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c0 = j * 8 + 2 * e;
                const __nv_bfloat16 h0 = __float2bfloat16_rn(v[c0]), h1 = __float2bfloat16_rn(v[c0 + 1]);
                ph[e] = bf16_pair_bits(h0, h1);
                pl[e] = bf16_pair_bits(__float2bfloat16_rn(v[c0] - __bfloat162float(h0)),
                                       __float2bfloat16_rn(v[c0 + 1] - __bfloat162float(h1)));
            }
            hi[j] = make_uint4(ph[0], ph[1], ph[2], ph[3]);
            lo[j] = make_uint4(pl[0], pl[1], pl[2], pl[3]);
        }
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int px = h_it - 1 - dx;
            if (px >= 0 && px < kTcCols) {
                char* cp = Acp + (dx + 1) * kTcCopyBytes;
                const int row = r_it * kTcCols + px;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    *reinterpret_cast<uint4*>(cp + sw128_offset(row, j * 8)) = hi[j];
                    *reinterpret_cast<uint4*>(cp + sw128_offset(row, kWide + j * 8)) = lo[j];
                }
            }
        }
    };
    // warp w: pixels 32 (w mod 4) .. + 31 (its TMEM lanes), channels 16 (w div 4) .. + 15
    auto epilogue = [&](int tile, int buf) {
        int b, y0, x0;
        tile_origin(tile, b, y0, x0);
        const int quarter = warp & 3, half = warp >> 2;
        float acc[16];
#pragma unroll
        for (int part = 0; part < kTcParts; ++part) {
            uint32_t pv[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) +
                          (uint32_t)(buf * kTcParts * 32 + part * 32 + half * 16),
                      pv);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = part == 0 ? __uint_as_float(pv[j]) : acc[j] + __uint_as_float(pv[j]);
        }
        const int m = quarter * 32 + (tid & 31);
        const int y = y0 + m / kTcCols, xq = x0 + m % kTcCols;
        if (y < H && xq < W) {
            const int64_t o0 = (int64_t)b * kWide * plane + (int64_t)y * W + xq;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int co = half * 16 + j;
                const int64_t o = o0 + co * plane;
                float val = acc[j] + (bias ? bias[co] : 0.f);
                if (relu) val = fmaxf(val, 0.f);
                if (out_mask && !(out_mask[o] > 0.f)) val = 0.f;
                out[o] = val;
            }
        }
    };

    uint32_t phase = 0;
    int k = 0, prev = -1;
    load_tile(blockIdx.x);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
        stage();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == kTcWorkers) {   // lane 0 of the MMA warp, which has no other work
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // K step kk (16 of the 64 BF16 of a row) of every tap accumulates into partial
            // accumulator kk: four independent chains, issued interleaved
            const uint32_t dst = tmem + (uint32_t)((k & 1) * kTcParts * 32);
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3 - 1, dx = t % 3 - 1;
                const uint32_t a0 = smem_u32(Acp + (dx + 1) * kTcCopyBytes + (dy + 1) * kTcCols * 128);
                const uint32_t b0 = smem_u32(Bw + t * kTcTapBytes);
#pragma unroll
                for (int kk = 0; kk < kTcParts; ++kk)   // K = 16 per MMA: 32 bytes into the row
                    mma_bf16(dst + kk * 32, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(b0 + kk * 32), idesc,
                             t > 0);
            }
            mma_commit(smem_u32(&bar));
        }
        load_tile(tile + gridDim.x);
        if (prev >= 0 && warp < kTcWorkers / 32) epilogue(prev, (k - 1) & 1);
        if (!mbar_wait(smem_u32(&bar), phase)) {
            atomicOr(status, 1);
            s_abort = 1;
        }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (s_abort) break;
        prev = tile;
    }
    if (prev >= 0 && !s_abort && warp < kTcWorkers / 32) epilogue(prev, (k - 1) & 1);
    // after a timeout the committed MMAs may still write the accumulators: wait for their
    // commit once more (bounded) and free the tensor memory only once they are done; if they
    // never finish it stays allocated (the status word already reports the timeout)
    __shared__ int s_drained;
    if (s_abort) {
        if (tid == 0) s_drained = mbar_wait(smem_u32(&bar), phase ^ 1) ? 1 : 0;
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && (!s_abort || s_drained)) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient of a 32 -> 32 layer on the tensor cores (tcgen05):
//     gw[co][ci][t] = sum_p g[co](p) x[ci](p + d_t),  d_t = (dy, dx),
// a contraction over the pixels.  Per tile of 4 x 32 pixels and per dy it is one GEMM
// D_dy[m][co] += sum_k A[m][k] B[co][k], with K the tile's 128 pixels:
//   A rows m = ((dx + 1) 32 + ci) 2 + h hold part h (hi, lo BF16 split of FP32) of x[ci]
//     over the tile's 6 halo rows, shifted by dx (three copies), K index 32 r + c for halo
//     row r, tile column c; the rows of tap dy are K offset 32 (dy + 1) of that, so every
//     tap is a descriptor offset;
//   B rows co hold part h' of g[co] over the tile (0 outside the image), K index 32 y + c.
// MMAs with B = g_hi and B = g_lo into the same accumulator give, summed over the two A
// rows of (dx, ci), x_hi g_hi + x_hi g_lo + x_lo g_hi + x_lo g_lo: FP32-accurate products
// with FP32 accumulation.  The 192 A rows form two M = 128 blocks (the second one's last
// 64 rows are never read back); per tile 3 dy x 2 blocks x 8 K steps x 2 = 96 MMAs with
// N = 32 into six 32-column accumulators that stay in tensor memory for all the tiles of a
// persistent CTA; the CTA adds them to gw with atomics at the end.  The bias gradient
// gb[co] = sum_p g[co](p) is summed by the threads that stage g.
// ---------------------------------------------------------------------------
constexpr int kWgThreads = 256;
constexpr int kWgRows = 4, kWgCols = 32;                 // tile: 128 pixels
constexpr int kWgArows = 192;                            // (dx, ci, h)
constexpr int kWgAplane = kWgArows * 128;                // one K atom (64 BF16) of every A row
constexpr int kWgBplane = kWide * 128;                   // one K atom of every B row
constexpr int kWgSmem = 3 * kWgAplane + 4 * kWgBplane + 1024;
constexpr int kWgTmemCols = 256;                         // 6 accumulators of 32 columns

__global__ void __launch_bounds__(kWgThreads, 2) wgrad32_tc_kernel(const float* __restrict__ x,
                                                                   const float* __restrict__ g,
                                                                   float* __restrict__ gw,
                                                                   float* __restrict__ gb, int B,
                                                                   int H, int W, int* status)
{
    using namespace mci;
    extern __shared__ __align__(1024) unsigned char wsm_raw[];
    char* A = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(wsm_raw) + 1023) & ~uintptr_t(1023));
    char* Bm = A + 3 * kWgAplane;   // [h'][K atom][co][128 B]; the second A block's unread rows
                                    // of the last plane overlap its start
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort, s_drained;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(kWgTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_bf16_f32(128, kWide);

    const int64_t plane = (int64_t)H * W;
    const int tiles_x = (W + kWgCols - 1) / kWgCols, tiles_y = (H + kWgRows - 1) / kWgRows;
    const int n_tiles = B * tiles_y * tiles_x;
    // B staging: thread (co = tid / 8, chunk = tid % 8) owns 16 pixels: tile row chunk / 2,
    // columns 16 (chunk % 2) .. + 15; it also sums them for the bias gradient
    const int bco = tid >> 3, bch = tid & 7, brow = bch >> 1, bc0 = (bch & 1) * 16;
    // A staging: items tid + 256 i, i < 3, of (ci, halo row r, 8-column chunk q): the 10 values
    // at columns x0 + 8q - 1 .. x0 + 8q + 8 feed the chunks of all three dx copies
    const bool vec = (W & 3) == 0;
    float xv[3][10], gv[16];
    auto tile_origin = [&](int tile, int& b, int& y0, int& x0) {
        b = tile / (tiles_y * tiles_x);
        const int r2 = tile - b * tiles_y * tiles_x;
        y0 = (r2 / tiles_x) * kWgRows;
        x0 = (r2 % tiles_x) * kWgCols;
    };
    auto load = [&](int tile) {
        if (tile >= n_tiles) return;
        int b, y0, x0;
        tile_origin(tile, b, y0, x0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int it = tid + kWgThreads * i, q = it & 3, r = (it >> 2) % 6, ci = it / 24;
            const float* src = x + ((int64_t)b * kWide + ci) * plane + (int64_t)wrapg(y0 - 1 + r, H) * W;
            const int c0 = x0 + 8 * q;
            if (vec && c0 >= 1 && c0 + 8 < W) {
                const float4 u0 = __ldg(reinterpret_cast<const float4*>(src + c0));
                const float4 u1 = __ldg(reinterpret_cast<const float4*>(src + c0 + 4));
                xv[i][0] = __ldg(src + c0 - 1);
                xv[i][1] = u0.x; xv[i][2] = u0.y; xv[i][3] = u0.z; xv[i][4] = u0.w;
                xv[i][5] = u1.x; xv[i][6] = u1.y; xv[i][7] = u1.z; xv[i][8] = u1.w;
                xv[i][9] = __ldg(src + c0 + 8);
            } else {
#pragma unroll
                for (int e = 0; e < 10; ++e) xv[i][e] = __ldg(src + wrapg(c0 - 1 + e, W));
            }
        }
        const int yy = y0 + brow, xb = x0 + bc0;
        const float* gsrc = g + ((int64_t)b * kWide + bco) * plane + (int64_t)yy * W + xb;
        if (vec && yy < H && xb + 15 < W) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float4 u = __ldg(reinterpret_cast<const float4*>(gsrc) + e);
                gv[4 * e] = u.x; gv[4 * e + 1] = u.y; gv[4 * e + 2] = u.z; gv[4 * e + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) gv[e] = (yy < H && xb + e < W) ? __ldg(gsrc + e) : 0.f;
        }
    };
    auto split8 = [](const float* v, uint4& hi, uint4& lo) {
        uint32_t ph[4], pl[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * e]), h1 = __float2bfloat16_rn(v[2 * e + 1]);
            ph[e] = bf16_pair_bits(h0, h1);
            pl[e] = bf16_pair_bits(__float2bfloat16_rn(v[2 * e] - __bfloat162float(h0)),
                                   __float2bfloat16_rn(v[2 * e + 1] - __bfloat162float(h1)));
        }
        hi = make_uint4(ph[0], ph[1], ph[2], ph[3]);
        lo = make_uint4(pl[0], pl[1], pl[2], pl[3]);
    };
    float gsum = 0.f;
    auto stage = [&]() {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int it = tid + kWgThreads * i, q = it & 3, r = (it >> 2) % 6, ci = it / 24;
            const int k = 32 * r + 8 * q;
            char* pa = A + (k >> 6) * kWgAplane;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {   // copy dx, K chunk k: columns x0 + 8q + dx ..
                uint4 hi, lo;
                split8(&xv[i][dx + 1], hi, lo);
                const int m = ((dx + 1) * kWide + ci) * 2;
                *reinterpret_cast<uint4*>(pa + sw128_offset(m, k & 63)) = hi;
                *reinterpret_cast<uint4*>(pa + sw128_offset(m + 1, k & 63)) = lo;
            }
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) gsum += gv[e];
        const int k = 32 * brow + bc0;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            uint4 hi, lo;
            split8(&gv[8 * hf], hi, lo);
            const int kk = k + 8 * hf;
            *reinterpret_cast<uint4*>(Bm + (0 * 2 + (kk >> 6)) * kWgBplane + sw128_offset(bco, kk & 63)) = hi;
            *reinterpret_cast<uint4*>(Bm + (1 * 2 + (kk >> 6)) * kWgBplane + sw128_offset(bco, kk & 63)) = lo;
        }
    };
    uint32_t phase = 0;
    bool first = true;
    // software pipeline: stage tile k from registers, issue its MMAs, load tile k + 1 into
    // registers while they run, then wait for them (they read the shared memory)
    load(blockIdx.x);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        stage();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int dyi = 0; dyi < 3; ++dyi)
#pragma unroll
                for (int mb = 0; mb < 2; ++mb) {
                    const uint32_t d = tmem + (uint32_t)((dyi * 2 + mb) * 32);
#pragma unroll
                    for (int hp = 0; hp < 2; ++hp)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int ka = 32 * dyi + 16 * j, kb = 16 * j;
                            const uint32_t a = smem_u32(A + (ka >> 6) * kWgAplane + mb * 128 * 128) + (ka & 63) * 2;
                            const uint32_t bb = smem_u32(Bm + (hp * 2 + (kb >> 6)) * kWgBplane) + (kb & 63) * 2;
                            mma_bf16(d, smem_desc_sw128(a), smem_desc_sw128(bb), idesc, !(first && hp == 0 && j == 0));
                        }
                }
            mma_commit(smem_u32(&bar));
        }
        load(tile + gridDim.x);
        first = false;
        if (!mbar_wait(smem_u32(&bar), phase)) {
            atomicOr(status, 1);
            s_abort = 1;
        }
        phase ^= 1;
        __syncthreads();
        if (s_abort) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_abort && !first) {
        // warp w reads TMEM lanes (A rows) 32 (w % 4) .. + 31, columns (co) 16 (w / 4) .. + 15
        const int quarter = warp & 3, half = warp >> 2;
#pragma unroll 1
        for (int acc = 0; acc < 6; ++acc) {
            const int dyi = acc >> 1, mb = acc & 1;
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 32 + half * 16), v);
            const int m = mb * 128 + quarter * 32 + lane;   // rows m (hi) and m + 1 (lo) of (dx, ci)
            float sv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float f = __uint_as_float(v[j]);
                sv[j] = f + __shfl_down_sync(0xffffffffu, f, 1);
            }
            if ((lane & 1) == 0 && m < kWgArows) {
                const int dx1 = (m >> 1) / kWide, ci = (m >> 1) % kWide, t = dyi * 3 + dx1;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    atomicAdd(&gw[((int64_t)(half * 16 + j) * kWide + ci) * 9 + t], sv[j]);
            }
        }
    }
    // bias: the 8 threads of one co are consecutive lanes
    gsum += __shfl_xor_sync(0xffffffffu, gsum, 1);
    gsum += __shfl_xor_sync(0xffffffffu, gsum, 2);
    gsum += __shfl_xor_sync(0xffffffffu, gsum, 4);
    if (!s_abort && bch == 0) atomicAdd(&gb[bco], gsum);
    // after a timeout the committed MMAs may still write the accumulators: wait for their
    // commit once more (bounded) and free the tensor memory only once they are done; if they
    // never finish it stays allocated (the status word already reports the timeout)
    if (s_abort) {
        if (tid == 0) s_drained = mbar_wait(smem_u32(&bar), phase ^ 1) ? 1 : 0;
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && (!s_abort || s_drained)) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Narrow layers (1 -> 32 and 32 -> 1) on CUDA cores, tiles of 8 rows x 32 columns: lane =
// image column (every row access of a warp is one coalesced segment), warp w takes the wide
// channels w, w + 8, w + 16, w + 24, and a 3 x 3 window slides down the tile's rows (one new
// row of three columns per step, read through L1).  Persistent CTAs; weight gradients are
// reduced over the warp's lanes and added with one atomic per (channel, tap) and warp.
// ---------------------------------------------------------------------------
constexpr int kNRows = 8, kNCols = 32, kNThreads = 256;

// Row yy (already wrapped) of one channel plane at the lane's three columns cm, c0, cp.
__device__ __forceinline__ void load3(const float* __restrict__ p, int yy, int W, int cm, int c0, int cp,
                                      float (&v)[3])
{
    const float* row = p + (int64_t)yy * W;
    v[0] = __ldg(row + cm);
    v[1] = __ldg(row + c0);
    v[2] = __ldg(row + cp);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 32 -> 1 convolution (the last layer): out = bias + sum_ci sum_t w[ci][t] x[ci](p + d_t), then
// optional ReLU, residual add and mask as in conv3x3_kernel.  One tile per CTA; each warp sums
// its four channels, the eight partial sums of a pixel are added through shared memory.
__global__ void __launch_bounds__(kNThreads) conv32to1_kernel(const float* __restrict__ x,
                                                              const __nv_bfloat16* __restrict__ w,
                                                              bool transposed_w, const float* __restrict__ bias,
                                                              const float* __restrict__ out_mask,
                                                              const float* __restrict__ res,
                                                              float* __restrict__ out, int H, int W, bool relu)
{
    __shared__ float red[kNThreads / 32][kNRows][kNCols];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.z, y0 = blockIdx.y * kNRows, col = blockIdx.x * kNCols + lane;
    const int64_t plane = (int64_t)H * W;
    const int cm = wrapg(col - 1, W), c0 = wrapg(col, W), cp = wrapg(col + 1, W);
    float part[kNRows];
#pragma unroll
    for (int r = 0; r < kNRows; ++r) part[r] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int ci = warp + 8 * j;
        float wv[9];
#pragma unroll
        for (int t = 0; t < 9; ++t)
            wv[t] = __bfloat162float(transposed_w ? w[(int64_t)ci * 9 + (8 - t)] : w[(int64_t)ci * 9 + t]);
        const float* xp = x + ((int64_t)b * kWide + ci) * plane;
        float w0[3], w1[3], w2[3];
        load3(xp, wrapg(y0 - 1, H), W, cm, c0, cp, w0);
        load3(xp, wrapg(y0, H), W, cm, c0, cp, w1);
#pragma unroll
        for (int r = 0; r < kNRows; ++r) {
            load3(xp, wrapg(y0 + r + 1, H), W, cm, c0, cp, w2);
#pragma unroll
            for (int d = 0; d < 3; ++d) part[r] += wv[d] * w0[d] + wv[3 + d] * w1[d] + wv[6 + d] * w2[d];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                w0[d] = w1[d];
                w1[d] = w2[d];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kNRows; ++r) red[warp][r][lane] = part[r];
    __syncthreads();
    const int r = warp, y = y0 + r;   // thread (r, lane) finishes pixel (y0 + r, col)
    if (y < H && col < W) {
        float v = bias ? bias[0] : 0.f;
#pragma unroll
        for (int k = 0; k < kNThreads / 32; ++k) v += red[k][r][lane];
        const int64_t o = (int64_t)b * plane + (int64_t)y * W + col;
        if (relu) v = fmaxf(v, 0.f);
        if (res) v += res[o];
        if (out_mask && !(out_mask[o] > 0.f)) v = 0.f;
        out[o] = v;
    }
}

// gw[co][ci][t] = sum_p g[co](p) x[ci](p + d_t), gb[co] = sum_p g[co](p) for the layers with one
// narrow side: CIN = 32, COUT = 1 (the last layer: the wide side is x) or CIN = 1, COUT = 32
// (the first layer: the wide side is g).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kNThreads, 2) wgrad_narrow_kernel(const float* __restrict__ x,
                                                                    const float* __restrict__ g,
                                                                    float* __restrict__ gw,
                                                                    float* __restrict__ gb, int B, int H,
                                                                    int W)
{
    static_assert((CIN == 1 && COUT == kWide) || (CIN == kWide && COUT == 1), "one narrow side");
    constexpr bool WIDE_X = CIN == kWide;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t plane = (int64_t)H * W;
    const int tiles_x = (W + kNCols - 1) / kNCols, tiles_y = (H + kNRows - 1) / kNRows;
    const int n_tiles = B * tiles_x * tiles_y;
    float acc[4][9], accb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        accb[j] = 0.f;
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[j][t] = 0.f;
    }
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int b = tile / (tiles_x * tiles_y);
        const int r2 = tile - b * tiles_x * tiles_y;
        const int y0 = (r2 / tiles_x) * kNRows, col = (r2 % tiles_x) * kNCols + lane;
        const bool in_w = col < W;
        const int cm = wrapg(col - 1, W), c0 = wrapg(col, W), cp = wrapg(col + 1, W);
        if constexpr (WIDE_X) {
            // the one gradient channel at the tile's pixels, then the 32 x channels
            float gv[kNRows];
#pragma unroll
            for (int r = 0; r < kNRows; ++r)
                gv[r] = (in_w && y0 + r < H) ? __ldg(g + (int64_t)b * plane + (int64_t)(y0 + r) * W + col) : 0.f;
#pragma unroll
            for (int r = 0; r < kNRows; ++r) accb[0] += gv[r];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float* xp = x + ((int64_t)b * kWide + warp + 8 * j) * plane;
                float w0[3], w1[3], w2[3];
                load3(xp, wrapg(y0 - 1, H), W, cm, c0, cp, w0);
                load3(xp, wrapg(y0, H), W, cm, c0, cp, w1);
#pragma unroll
                for (int r = 0; r < kNRows; ++r) {
                    load3(xp, wrapg(y0 + r + 1, H), W, cm, c0, cp, w2);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        acc[j][d] += gv[r] * w0[d];
                        acc[j][3 + d] += gv[r] * w1[d];
                        acc[j][6 + d] += gv[r] * w2[d];
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        w0[d] = w1[d];
                        w1[d] = w2[d];
                    }
                }
            }
        } else {
            // the one x channel around the tile, then the 32 gradient channels
            float xw[kNRows + 2][3];
#pragma unroll
            for (int r = 0; r < kNRows + 2; ++r) load3(x + (int64_t)b * plane, wrapg(y0 - 1 + r, H), W, cm, c0, cp, xw[r]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float* gp = g + ((int64_t)b * kWide + warp + 8 * j) * plane;
#pragma unroll
                for (int r = 0; r < kNRows; ++r) {
                    const float gv = (in_w && y0 + r < H) ? __ldg(gp + (int64_t)(y0 + r) * W + col) : 0.f;
                    accb[j] += gv;
#pragma unroll
                    for (int t = 0; t < 9; ++t) acc[j][t] += gv * xw[r + t / 3][t % 3];
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = warp + 8 * j;   // the wide channel
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const float v = warp_sum(acc[j][t]);
            if (lane == 0) atomicAdd(&gw[(int64_t)c * 9 + t], v);   // [co][ci][t] with one side 1
        }
        if (!WIDE_X) {
            const float v = warp_sum(accb[j]);
            if (lane == 0) atomicAdd(&gb[c], v);
        }
    }
    if (WIDE_X && warp == 0) {
        const float v = warp_sum(accb[0]);
        if (lane == 0) atomicAdd(&gb[0], v);
    }
}

// d pred: grad = 2 (pred - hr) / n, loss += sum (pred - hr)^2 / n
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ hr, float* __restrict__ grad,
                           float* __restrict__ loss, int64_t n)
{
    float part = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = pred[i] - hr[i];
        if (grad) grad[i] = 2.f * d / (float)n;
        part += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, part / (float)n);
}

// Adam on FP32 master weights; refresh the BF16 copy used by the convolutions.
__global__ void adam_kernel(float* __restrict__ master, __nv_bfloat16* __restrict__ wbf,
                            const float* __restrict__ grad, float* __restrict__ m1, float* __restrict__ m2,
                            int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float v = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    const float wv = master[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    master[i] = wv;
    if (wbf) wbf[i] = __float2bfloat16_rn(wv);
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// ---------------------------------------------------------------------------
// synthetic images: 0.5 + 20 anisotropic Gaussian blobs + 10 straight edges
// + 8 low-frequency waves of amplitude 0.01, clipped to [0, 1].  Parameters per image
// (host-drawn, seeded): blobs (cy, cx, 1/s_major, 1/s_minor, angle, amp), edges
// (py, px, angle, step), waves (fy, fx, phase, amp) -- all in pixel units.
// ---------------------------------------------------------------------------
__global__ void image_gen_kernel(const float* __restrict__ prm, float* __restrict__ img, int H, int W)
{
    const int b = blockIdx.z;
    const float* q = prm + (int64_t)b * MCI_IMAGE_PARAMS;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, x = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= H || x >= W) return;
    float v = 0.5f;
    for (int k = 0; k < 20; ++k) {
        const float* p = q + 6 * k;
        const float dy = y - p[0], dx = x - p[1];
        float sa, ca;
        sincosf(p[4], &sa, &ca);
        const float u = (dx * ca + dy * sa) * p[2], w = (-dx * sa + dy * ca) * p[3];
        v += p[5] * __expf(-0.5f * (u * u + w * w));
    }
    for (int k = 0; k < 10; ++k) {
        const float* p = q + 120 + 4 * k;
        float sa, ca;
        sincosf(p[2], &sa, &ca);
        if ((x - p[1]) * sa - (y - p[0]) * ca > 0.f) v += p[3];
    }
    for (int k = 0; k < 8; ++k) {
        const float* p = q + 160 + 4 * k;
        float t = p[0] * y / H + p[1] * x / W;     // integer cycles: reduce to [-1/2, 1/2]
        t -= rintf(t);
        v += p[3] * __cosf(6.2831853f * t + p[2]);
    }
    img[((int64_t)b * H + y) * W + x] = fminf(fmaxf(v, 0.f), 1.f);
}

// pure decimation LR[y][x] = HR[s y][s x]
__global__ void decimate_kernel(const float* __restrict__ hr, float* __restrict__ lr, int H, int W, int s)
{
    const int b = blockIdx.z;
    const int h = H / s, w = W / s;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, x = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= h || x >= w) return;
    lr[((int64_t)b * h + y) * w + x] = hr[((int64_t)b * H + (int64_t)s * y) * W + (int64_t)s * x];
}

// Gaussian blur (periodic) followed by decimation: lr[y][x] = sum_{i,j} w_i w_j
// hr[(s y - i) mod H][(s x - j) mod W], |i|, |j| <= K; one thread per LR pixel.
struct BlurTaps {
    float w[256];
    int K;
};

__device__ __forceinline__ int wrap_index(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__global__ void degrade_kernel(const float* __restrict__ hr, float* __restrict__ lr, int H, int W, int s,
                               const BlurTaps t)
{
    const int b = blockIdx.z;
    const int h = H / s, w = W / s;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, x = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= h || x >= w) return;
    const float* img = hr + (int64_t)b * H * W;
    float acc = 0.f;
    for (int i = -t.K; i <= t.K; ++i) {
        const float* row = img + (int64_t)wrap_index(s * y - i, H) * W;
        float r = 0.f;
        for (int j = -t.K; j <= t.K; ++j) r = fmaf(t.w[j + t.K], __ldg(row + wrap_index(s * x - j, W)), r);
        acc = fmaf(t.w[i + t.K], r, acc);
    }
    lr[((int64_t)b * h + y) * w + x] = acc;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct mci_corrector_s {
    int64_t max_pixels = 0;
    int n_params = 0;
    int woff[kLayers], boff[kLayers];
    float* master = nullptr;        // FP32 master weights and biases (flat)
    __nv_bfloat16* wbf = nullptr;   // BF16 copy
    float* grad = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    float* act = nullptr;           // layer outputs: kLayers - 1 hidden [B][32][H][W] + pred
    float* gbuf[2] = {nullptr, nullptr};
    float* loss = nullptr;
    int* status = nullptr;          // device: bit 0 = a tensor-core wait timed out
    int step = 0;
};

namespace {

int corrector_param_layout(int* woff, int* boff)
{
    int n = 0;
    for (int l = 0; l < kLayers; ++l) {
        woff[l] = n;
        n += cout_of(l) * cin_of(l) * 9;
        boff[l] = n;
        n += cout_of(l);
    }
    return n;
}

int tc_grid_limit()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        n = 2 * (sms > 0 ? sms : 1);
        cudaFuncSetAttribute(conv32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        cudaFuncSetAttribute(wgrad32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
    }
    return n;
}

// out_mask: optional tensor shaped like out; outputs where it is <= 0 are zeroed.
cudaError_t conv(const float* x, int cin, int cout, const __nv_bfloat16* w, bool tw, const float* bias,
                 const float* out_mask, const float* res, float* out, int B, int H, int W, bool relu,
                 cudaStream_t s, int* status)
{
    if (cin == kWide && cout == kWide && !res) {
        const int tiles = B * ((H + kTcRows - 1) / kTcRows) * ((W + kTcCols - 1) / kTcCols);
        const int grid = tiles < tc_grid_limit() ? tiles : tc_grid_limit();
        conv32_tc_kernel<<<grid, kTcThreads, kTcSmem, s>>>(x, w, tw, bias, out_mask, out, B, H, W, relu, status);
        return cudaGetLastError();
    }
    const dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, B);
    const size_t smem = sizeof(float) * (cin * kHalo * kHalo + cin * 9 * cout);
    if (cout == kWide) {
        cudaFuncSetAttribute(conv3x3_kernel<kWide>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        conv3x3_kernel<kWide><<<grid, kCThreads, smem, s>>>(x, cin, w, tw, bias, out_mask, res, out, H, W, relu);
    } else if (cin == kWide) {
        const dim3 ngrid((W + kNCols - 1) / kNCols, (H + kNRows - 1) / kNRows, B);
        conv32to1_kernel<<<ngrid, kNThreads, 0, s>>>(x, w, tw, bias, out_mask, res, out, H, W, relu);
    } else {
        conv3x3_kernel<1><<<grid, kCThreads, smem, s>>>(x, cin, w, tw, bias, out_mask, res, out, H, W, relu);
    }
    return cudaGetLastError();
}

cudaError_t wgrad(int l, const float* x, const float* g, float* gw, float* gb, int B, int H, int W,
                  cudaStream_t s, int* status)
{
    const int tiles = B * ((H + kNRows - 1) / kNRows) * ((W + kNCols - 1) / kNCols);
    const int grid = tiles < tc_grid_limit() ? tiles : tc_grid_limit();
    const int cin = cin_of(l), cout = cout_of(l);
    if (cin == 1) {
        wgrad_narrow_kernel<1, kWide><<<grid, kNThreads, 0, s>>>(x, g, gw, gb, B, H, W);
    } else if (cout == 1) {
        wgrad_narrow_kernel<kWide, 1><<<grid, kNThreads, 0, s>>>(x, g, gw, gb, B, H, W);
    } else {
        // 32 -> 32: tensor cores, tiles of 4 x 32 pixels
        const int tc_tiles = B * ((H + kWgRows - 1) / kWgRows) * ((W + kWgCols - 1) / kWgCols);
        const int tc_grid = tc_tiles < tc_grid_limit() ? tc_tiles : tc_grid_limit();
        wgrad32_tc_kernel<<<tc_grid, kWgThreads, kWgSmem, s>>>(x, g, gw, gb, B, H, W, status);
    }
    return cudaGetLastError();
}

float* hidden(mci_corrector_t c, int l, int64_t pix) { return c->act + (int64_t)l * kWide * pix; }

// forward: hidden activations 0..3, prediction into pred
cudaError_t forward(mci_corrector_t c, const float* mci, float* pred, int B, int H, int W, cudaStream_t s)
{
    const int64_t pix = (int64_t)B * H * W;
    const float* x = mci;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        const bool last = l == kLayers - 1;
        float* y = last ? pred : hidden(c, l, pix);
        e = conv(x, cin_of(l), cout_of(l), c->wbf + c->woff[l], false, c->master + c->boff[l], nullptr,
                 last ? mci : nullptr, y, B, H, W, !last, s, c->status);
        x = y;
    }
    return e;
}

// backward from d pred ([B][1][H][W]); parameter gradients into grad.  g is the gradient
// with respect to layer l's pre-activation output: the data-gradient conv of layer l
// zeroes its output where hidden(l - 1) <= 0 (the ReLU derivative of layer l - 1).
cudaError_t backward(mci_corrector_t c, const float* mci, const float* gpred, int B, int H, int W,
                     cudaStream_t s)
{
    const int64_t pix = (int64_t)B * H * W;
    cudaError_t e = cudaMemsetAsync(c->grad, 0, sizeof(float) * c->n_params, s);
    const float* g = gpred;
    int gi = 0;
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
        const float* x = l == 0 ? mci : hidden(c, l - 1, pix);
        e = wgrad(l, x, g, c->grad + c->woff[l], c->grad + c->boff[l], B, H, W, s, c->status);
        if (l > 0 && e == cudaSuccess) {
            // gradient with respect to layer l's input: conv with transposed, reversed weights
            float* gin = c->gbuf[gi];
            e = conv(g, cout_of(l), cin_of(l), c->wbf + c->woff[l], true, nullptr, hidden(c, l - 1, pix), nullptr,
                     gin, B, H, W, false, s, c->status);
            g = gin;
            gi ^= 1;
        }
    }
    return e;
}

}  // namespace

extern "C" {

mci_status mci_corrector_create(mci_corrector_t* out, int64_t max_pixels, const float* init_params,
                                mci_stream_t stream)
{
    if (!out || max_pixels <= 0) return MCI_ERR_INVALID_ARG;
    *out = nullptr;
    mci_corrector_s* c = new (std::nothrow) mci_corrector_s();
    if (!c) return MCI_ERR_OOM;
    c->max_pixels = max_pixels;
    c->n_params = corrector_param_layout(c->woff, c->boff);
    const int n = c->n_params;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&c->master, sizeof(float) * n * 4);
    if (e == cudaSuccess) {
        c->grad = c->master + n;
        c->m1 = c->master + 2 * n;
        c->m2 = c->master + 3 * n;
        e = cudaMalloc(&c->wbf, sizeof(__nv_bfloat16) * n);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->act, sizeof(float) * max_pixels * (kWide * (kLayers - 1)));
    if (e == cudaSuccess) e = cudaMalloc(&c->gbuf[0], sizeof(float) * max_pixels * kWide * 2);
    if (e == cudaSuccess) c->gbuf[1] = c->gbuf[0] + max_pixels * kWide;
    if (e == cudaSuccess) e = cudaMalloc(&c->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->master, 0, sizeof(float) * n * 4, s);
    if (e == cudaSuccess && init_params)
        e = cudaMemcpyAsync(c->master, init_params, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(n + 255) / 256, 256, 0, s>>>(c->master, c->wbf, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        mci_corrector_destroy(c);
        return e == cudaErrorMemoryAllocation ? MCI_ERR_OOM : MCI_ERR_CUDA;
    }
    *out = c;
    return MCI_OK;
}

int mci_corrector_num_params(void)
{
    int wo[kLayers], bo[kLayers];
    return corrector_param_layout(wo, bo);
}

mci_status mci_corrector_destroy(mci_corrector_t c)
{
    if (!c) return MCI_OK;
    cudaDeviceSynchronize();
    cudaFree(c->master);
    cudaFree(c->wbf);
    cudaFree(c->act);
    cudaFree(c->gbuf[0]);
    cudaFree(c->loss);
    cudaFree(c->status);
    delete c;
    return MCI_OK;
}

mci_status mci_corrector_forward(mci_corrector_t c, const float* mci, float* out, int batch, int h, int w,
                                 mci_stream_t stream)
{
    if (!c || !mci || !out || batch <= 0 || h < 3 || w < 3) return MCI_ERR_INVALID_ARG;
    if ((int64_t)batch * h * w > c->max_pixels) return MCI_ERR_UNSUPPORTED_SIZE;
    return forward(c, mci, out, batch, h, w, (cudaStream_t)stream) == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_corrector_loss_grad(mci_corrector_t c, const float* mci, const float* hr, int batch, int h,
                                   int w, float* grad_out, float* loss_out, mci_stream_t stream)
{
    if (!c || !mci || !hr || batch <= 0 || h < 3 || w < 3) return MCI_ERR_INVALID_ARG;
    const int64_t pix = (int64_t)batch * h * w;
    if (pix > c->max_pixels) return MCI_ERR_UNSUPPORTED_SIZE;
    cudaStream_t s = (cudaStream_t)stream;
    float* pred = c->gbuf[1];        // reused: the first data gradient goes to gbuf[0]
    float* gpred = c->gbuf[1] + pix;
    cudaError_t e = forward(c, mci, pred, batch, h, w, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->loss, 0, sizeof(float), s);
    if (e == cudaSuccess) {
        mse_kernel<<<304, 256, 0, s>>>(pred, hr, gpred, c->loss, pix);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward(c, mci, gpred, batch, h, w, s);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, c->grad, sizeof(float) * c->n_params, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && loss_out)
        e = cudaMemcpyAsync(loss_out, c->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_corrector_train_step(mci_corrector_t c, const float* mci, const float* hr, int batch, int h,
                                    int w, float lr, float* loss_out, mci_stream_t stream)
{
    mci_status st = mci_corrector_loss_grad(c, mci, hr, batch, h, w, nullptr, loss_out, stream);
    if (st != MCI_OK) return st;
    const float b1 = 0.9f, b2 = 0.999f;
    c->step += 1;
    const float c1 = 1.f - std::pow(b1, (float)c->step), c2 = 1.f - std::pow(b2, (float)c->step);
    adam_kernel<<<(c->n_params + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        c->master, c->wbf, c->grad, c->m1, c->m2, c->n_params, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_corrector_get_state(mci_corrector_t c, float* host, int* step)
{
    if (!c || !host) return MCI_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, c->master, sizeof(float) * c->n_params, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(host + c->n_params, c->m1, sizeof(float) * 2 * c->n_params, cudaMemcpyDeviceToHost);
    if (step) *step = c->step;
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_corrector_set_state(mci_corrector_t c, const float* host, int step)
{
    if (!c || !host || step < 0) return MCI_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c->master, host, sizeof(float) * c->n_params, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->m1, host + c->n_params, sizeof(float) * 2 * c->n_params, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(c->n_params + 255) / 256, 256>>>(c->master, c->wbf, c->n_params);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    c->step = step;
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_corrector_status(mci_corrector_t c, int* status)
{
    if (!c || !status) return MCI_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, c->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_generate_images(const float* params, float* img, int n, int h, int w, mci_stream_t stream)
{
    if (!params || !img || n <= 0 || h <= 0 || w <= 0) return MCI_ERR_INVALID_ARG;
    const dim3 blk(32, 8), grid((w + 31) / 32, (h + 7) / 8, n);
    image_gen_kernel<<<grid, blk, 0, (cudaStream_t)stream>>>(params, img, h, w);
    return cudaGetLastError() == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_decimate(const float* hr, float* lr, int n, int h, int w, int s, mci_stream_t stream)
{
    if (!hr || !lr || n <= 0 || n > 65535 || s <= 0 || h <= 0 || w <= 0 || h % s || w % s)
        return MCI_ERR_INVALID_ARG;
    const dim3 blk(32, 8), grid((w / s + 31) / 32, (h / s + 7) / 8, n);
    decimate_kernel<<<grid, blk, 0, (cudaStream_t)stream>>>(hr, lr, h, w, s);
    return cudaGetLastError() == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_degrade(const float* hr, float* lr, int n, int h, int w, int s, int taps, double sigma,
                       mci_stream_t stream)
{
    if (!hr || !lr || n <= 0 || n > 65535 || s <= 0 || h <= 0 || w <= 0 || h % s || w % s)
        return MCI_ERR_INVALID_ARG;
    if (taps < 1 || taps > 255 || taps % 2 == 0 || !(sigma > 0.0) || !std::isfinite(sigma))
        return MCI_ERR_INVALID_ARG;
    BlurTaps t{};
    t.K = taps / 2;
    double sum = 0.0, wd[256];
    for (int k = -t.K; k <= t.K; ++k) sum += (wd[k + t.K] = std::exp(-(double)k * k / (2.0 * sigma * sigma)));
    for (int k = 0; k < taps; ++k) t.w[k] = (float)(wd[k] / sum);
    const dim3 blk(32, 8), grid((w / s + 31) / 32, (h / s + 7) / 8, n);
    degrade_kernel<<<grid, blk, 0, (cudaStream_t)stream>>>(hr, lr, h, w, s, t);
    return cudaGetLastError() == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

}  // extern "C"
