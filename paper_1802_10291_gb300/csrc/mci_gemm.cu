// Tensor-core (tcgen05) GEMM for the small-P image path.
//
// For a fixed size class (P, T) in derivative-channel mode, one 1-D interpolation is a real
// linear map out = K in with K a T x P matrix (a phase-interleaved circulant, built by the
// plan from the FP64 weights).  A batch of images then needs two GEMMs per image: the row
// pass Y^T = K_w X^T and the column pass HR = K_h Y.  Both run here as jobs of
//     C[M x N] = sum over split pairs  A_a[M x K] * B_b[N x K]^T
// with every operand split into three BF16 planes (x = x_h + x_m + x_l) in the 128-byte-
// swizzled K-major layout, and the six products h*h, h*m, m*h, h*l, m*m, l*h accumulated in
// FP32 in tensor memory (error near FP32 rounding).
//
// One operand of each pass is the plan's constant K: it is split once, when the plan is
// made, into tiles of 128 rows x 64 columns laid out exactly as the kernel keeps them in
// shared memory, and a tile's three planes arrive with one bulk asynchronous copy whose
// bytes an mbarrier counts.  The other operand (the image or the intermediate) is read from
// global memory and split by all threads, each chunk's loads issued before the previous
// chunk's MMAs are waited for.  K runs in chunks of 64 through one shared-memory
// stage, refilled once the MMAs that read it have committed; two CTAs share an SM (96 KB of
// shared memory and at most 128 registers each), so one CTA's loads overlap the other's MMAs
// and epilogue.  A row-major result goes out through the stage (free by then) so that each
// warp stores whole 512-byte rows.  One thread issues the MMAs.  Every mbarrier wait is
// bounded: a timeout sets a status bit and the tile is abandoned, after a bounded wait for
// the work in flight.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mci_internal.h"
#include "tc_ptx.cuh"

namespace mci {

constexpr int kGemmThreads = 256;
constexpr int kTileM = 128;
constexpr int kTileN = 128;
constexpr int kChunkK = 64;                               // one 128-byte swizzle atom of BF16
constexpr int kPlane = kTileM * kChunkK * 2;              // bytes of one 128 x 64 BF16 plane
constexpr int kTileBytes = 3 * kPlane;                    // one operand tile: planes h, m, l
constexpr int kStage = 2 * kTileBytes;                    // A tile, then B tile
constexpr int kGemmSmem = kStage + 1024;                  // one stage + alignment
constexpr int kCPitch = kTileN + 4;                       // staged result row (floats)
static_assert(kTileM * kCPitch * 4 <= kStage, "the result tile fits in the stage");

// Split four FP32 values into three BF16 planes (h, m, l) and store them.
__device__ __forceinline__ void split_store(const float4 v, char* plane_h, uint32_t off)
{
    float x[4] = {v.x, v.y, v.z, v.w};
    float h[4], m[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = __bfloat162float(__float2bfloat16_rn(x[i]));
        const float r1 = x[i] - h[i];
        m[i] = __bfloat162float(__float2bfloat16_rn(r1));
        l[i] = r1 - m[i];
    }
    *reinterpret_cast<uint2*>(plane_h + off) = make_uint2(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]));
    *reinterpret_cast<uint2*>(plane_h + kPlane + off) =
        make_uint2(pack_bf16(m[0], m[1]), pack_bf16(m[2], m[3]));
    *reinterpret_cast<uint2*>(plane_h + 2 * kPlane + off) =
        make_uint2(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]));
}

// Pre-split tiles of a constant rows x cols matrix: tile (rt, kc) (rows 128 rt.., columns
// 64 kc..) at byte (rt (cols / 64) + kc) kTileBytes of `out`.
__global__ void gemm_presplit_kernel(const float* __restrict__ K, int cols, char* __restrict__ out)
{
    const int tile = blockIdx.x, kcs = cols / kChunkK;
    const int rt = tile / kcs, kc = tile - rt * kcs;
    char* dst = out + (size_t)tile * kTileBytes;
    for (int i = threadIdx.x; i < kTileM * (kChunkK / 4); i += blockDim.x) {
        const int r = i / (kChunkK / 4), k = (i % (kChunkK / 4)) * 4;
        const float4 v = *reinterpret_cast<const float4*>(K + (size_t)(rt * kTileM + r) * cols + kc * kChunkK + k);
        split_store(v, dst, sw128_offset(r, k));
    }
}

// Bulk asynchronous copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on mbarrier `bar` by its byte count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Rows r0 .. r0 + 127, columns k0 .. k0 + 63 of a row-major FP32 operand: 2048 16-byte
// vectors, eight per thread, loaded into registers (all in flight at once) and then split
// into the three planes at dst.
constexpr int kPer = kTileM * (kChunkK / 4) / kGemmThreads;

__device__ __forceinline__ void load_chunk(const float* X, int64_t ld, int r0, int k0, float4 (&v)[kPer])
{
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = threadIdx.x + j * kGemmThreads;
        const int r = i / (kChunkK / 4), k = (i % (kChunkK / 4)) * 4;
        v[j] = __ldg(reinterpret_cast<const float4*>(X + (int64_t)(r0 + r) * ld + k0 + k));
    }
}

__device__ __forceinline__ void split_chunk(const float4 (&v)[kPer], char* dst)
{
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = threadIdx.x + j * kGemmThreads;
        const int r = i / (kChunkK / 4), k = (i % (kChunkK / 4)) * 4;
        split_store(v[j], dst, sw128_offset(r, k));
    }
}

// ---------------------------------------------------------------------------
// kernel: one CTA per 128 x 128 tile of one job
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGemmThreads, 2) gemm_split3_kernel(const GemmJob* __restrict__ jobs,
                                                                   const int* __restrict__ tile0,
                                                                   int n_jobs, int* status)
{
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar_mma, bar_ld;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort, s_drained;

    // job of this tile (tile0 is the non-decreasing tile prefix, n_jobs + 1 entries)
    int lo = 0, hi = n_jobs - 1;
    const int t = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    GemmJob J = jobs[lo];
    if (J.a_off) J.A += J.a_off[J.img];
    if (J.c_off) J.C += J.c_off[J.img];
    const bool a_const = J.a_planes != nullptr, b_const = J.b_planes != nullptr;
    // exactly one operand comes pre-split; the other and the row-major output move as
    // 16-byte vectors
    if (a_const == b_const || (!a_const && ((reinterpret_cast<uintptr_t>(J.A) & 15) || (J.lda & 3))) ||
        (!b_const && ((reinterpret_cast<uintptr_t>(J.B) & 15) || (J.ldb & 3))) ||
        (!J.transpose_c && (reinterpret_cast<uintptr_t>(J.C) & 15))) {
        if (threadIdx.x == 0) atomicOr(status, kStatusBadOffset);
        return;
    }
    const int tiles_n = J.N / kTileN;
    const int tt = t - tile0[lo];
    const int m0 = (tt / tiles_n) * kTileM, n0 = (tt % tiles_n) * kTileN;
    const int chunks = J.K / kChunkK;
    // the pre-split operand's tiles for this tile's rows, and the data operand
    const char* cst = a_const ? J.a_planes + (size_t)(m0 / kTileM) * chunks * kTileBytes
                              : J.b_planes + (size_t)(n0 / kTileN) * chunks * kTileBytes;
    const float* X = a_const ? J.B : J.A;
    const int64_t ldx = a_const ? J.ldb : J.lda;
    const int rx = a_const ? n0 : m0;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(kTileN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar_mma), 1);
        mbar_init(smem_u32(&bar_ld), 1);
        s_abort = 0;
        s_drained = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_bf16_f32(kTileM, kTileN);

    int last_copy = -1, waited_copy = -1, last_commit = -1;   // thread 0's record of work in flight
    char* A = base;
    char* B = base + kTileBytes;
    float4 v[kPer];
    load_chunk(X, ldx, rx, 0, v);
    for (int ch = 0; ch < chunks; ++ch) {
        // the MMAs of chunk ch - 1 read the stage
        if (ch >= 1 && !mbar_wait(smem_u32(&bar_mma), (ch - 1) & 1)) {
            atomicOr(status, kStatusTimeout);
            s_abort = 1;
        }
        if (threadIdx.x == 0) {
            bulk_g2s(smem_u32(a_const ? A : B), cst + (size_t)ch * kTileBytes, kTileBytes, smem_u32(&bar_ld));
            last_copy = ch;
        }
        split_chunk(v, a_const ? B : A);
        // the next chunk's data is in flight while the tensor core works on this one
        if (ch + 1 < chunks) load_chunk(X, ldx, rx, (ch + 1) * kChunkK, v);
        // make the generic-proxy stores visible to the tensor core, then issue
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_abort) break;
        if (threadIdx.x == 0) {
            const bool ok = mbar_wait(smem_u32(&bar_ld), ch & 1);
            if (!ok) {
                atomicOr(status, kStatusTimeout);
                s_abort = 1;
            } else {
                waited_copy = ch;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // pairs (a, b) with a + b <= 2: hh, hm, mh, hl, mm, lh
                const int pa[6] = {0, 0, 1, 0, 1, 2};
                const int pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
                for (int pr = 0; pr < 6; ++pr) {
                    const uint32_t a0 = smem_u32(A + pa[pr] * kPlane), b0 = smem_u32(B + pb[pr] * kPlane);
#pragma unroll
                    for (int kk = 0; kk < kChunkK / 16; ++kk)  // K = 16 per MMA: 32 bytes into the atom
                        mma_bf16(tmem, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(b0 + kk * 32), idesc,
                                 ch > 0 || pr > 0 || kk > 0);
                }
                mma_commit(smem_u32(&bar_mma));
                last_commit = ch;
            }
        }
    }
    __syncthreads();
    // the last commit completes when every MMA of the tile has
    if (!s_abort && !mbar_wait(smem_u32(&bar_mma), (chunks - 1) & 1)) {
        atomicOr(status, kStatusTimeout);
        s_abort = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: warp w holds accumulator rows 32 (w mod 4) .. + 31 (its TMEM lanes) and
    // columns 64 (w / 4) .. + 63, 32 per load
    if (!s_abort) {
        const int lr = (warp & 3) * 32, row = m0 + lr + lane;
#pragma unroll 1
        for (int c0 = (warp >> 2) * 64; c0 < (warp >> 2) * 64 + 64; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)lr << 16) + (uint32_t)c0, v);
            if (J.transpose_c) {
                // C^T: column n of the tile is row n of the output, rows consecutive across lanes
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    J.C[(int64_t)(n0 + c0 + j) * J.ldc + row] = __uint_as_float(v[j]);
            } else {
                // into the stage, rows kCPitch floats apart (a quarter warp's eight rows hit all
                // 32 banks)
                float4* srow = reinterpret_cast<float4*>(reinterpret_cast<float*>(base) + (lr + lane) * kCPitch + c0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    srow[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                          __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
            }
        }
        if (!J.transpose_c) {
            __syncthreads();
            // warp w stores rows w, w + 8, ..: lane l writes 16 bytes at column 4 l
            for (int r = warp; r < kTileM; r += kGemmThreads / 32) {
                const float4 x = reinterpret_cast<const float4*>(reinterpret_cast<float*>(base) + r * kCPitch)[lane];
                reinterpret_cast<float4*>(J.C + (int64_t)(m0 + r) * J.ldc + n0)[lane] = x;
            }
        }
    }
    // after a timeout, copies and MMAs may still be writing shared and tensor memory: wait for
    // them once more (bounded) and free the tensor memory only once they are done; if they never
    // finish it stays allocated (the status word already reports the timeout)
    if (s_abort && threadIdx.x == 0) {
        bool ok = true;
        if (last_copy > waited_copy) ok = mbar_wait(smem_u32(&bar_ld), last_copy & 1) && ok;
        if (last_commit >= 0) ok = mbar_wait(smem_u32(&bar_mma), last_commit & 1) && ok;
        s_drained = ok ? 1 : 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0 && (!s_abort || s_drained)) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTileN)
                     : "memory");
    }
}

int gemm_smem_bytes() { return kGemmSmem; }

int prepare_gemm()
{
    cudaError_t e = cudaFuncSetAttribute(gemm_split3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    // two CTAs per SM: the largest shared-memory carveout
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_split3_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return (int)e;
}

int64_t gemm_plane_bytes(int rows, int cols) { return (int64_t)(rows / kTileM) * (cols / kChunkK) * kTileBytes; }

int presplit_gemm(const float* K, int rows, int cols, char* out, void* stream)
{
    if (rows % kTileM || cols % kChunkK) return (int)cudaErrorInvalidValue;
    gemm_presplit_kernel<<<(rows / kTileM) * (cols / kChunkK), 256, 0, (cudaStream_t)stream>>>(K, cols, out);
    return (int)cudaGetLastError();
}

int launch_gemm(const GemmJob* jobs, const int* tile0, int n_jobs, int n_tiles, int* status, void* stream)
{
    if (n_tiles <= 0) return 0;
    gemm_split3_kernel<<<n_tiles, kGemmThreads, kGemmSmem, (cudaStream_t)stream>>>(jobs, tile0, n_jobs,
                                                                                    status);
    return (int)cudaGetLastError();
}

}  // namespace mci
