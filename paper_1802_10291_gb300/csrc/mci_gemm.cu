// Tensor-core (tcgen05) GEMM for the small-P image path.
//
// For a fixed size class (P, T) in derivative-channel mode, one 1-D
// interpolation is a real linear map out = K in with K a T x P matrix (a
// phase-interleaved circulant, built by the plan from the FP64 weights).  A
// batch of images then needs two GEMMs per image: the row pass Y^T = K_w X^T
// and the column pass HR = K_h Y.  Both run here as jobs of
//     C[M x N] = sum over split pairs  A_a[M x K] * B_b[N x K]^T
// where A and B are FP32 in global memory, read in K-chunks of 64, split on
// the fly into three BF16 planes (x = x_h + x_m + x_l) and stored in shared
// memory in the 128-byte-swizzled K-major layout; the six products
// h*h, h*m, m*h, h*l, m*m, l*h accumulate in FP32 in tensor memory (error near
// FP32 rounding).  One thread issues the MMAs; completion is tracked by an
// mbarrier whose waits are bounded (a timeout sets a status bit and the tile
// is abandoned, so no wait can hang).  The epilogue reads the accumulator
// with tcgen05.ld and stores C row-major or transposed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mci_internal.h"
#include "tc_ptx.cuh"

namespace mci {

constexpr int kGemmThreads = 128;
constexpr int kTileM = 128;
constexpr int kTileN = 128;
constexpr int kChunkK = 64;                               // one 128-byte swizzle atom of BF16
constexpr int kPlane = kTileM * kChunkK * 2;              // bytes of one 128 x 64 BF16 plane
constexpr int kGemmSmem = 6 * kPlane + 1024;              // 3 A planes + 3 B planes + alignment

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

// ---------------------------------------------------------------------------
// kernel: one CTA per 128 x 128 tile of one job
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGemmThreads) gemm_split3_kernel(const GemmJob* __restrict__ jobs,
                                                                   const int* __restrict__ tile0,
                                                                   int n_jobs, int* status)
{
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    char* A = base;                 // planes h, m, l
    char* B = base + 3 * kPlane;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;

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
    // operands and the row-major output are read and written with 16-byte vectors
    if (((reinterpret_cast<uintptr_t>(J.A) | reinterpret_cast<uintptr_t>(J.B)) & 15) ||
        (!J.transpose_c && (reinterpret_cast<uintptr_t>(J.C) & 15))) {
        if (threadIdx.x == 0) atomicOr(status, kStatusBadOffset);
        return;
    }
    const int tiles_n = J.N / kTileN;
    const int tt = t - tile0[lo];
    const int m0 = (tt / tiles_n) * kTileM, n0 = (tt % tiles_n) * kTileN;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(kTileN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_bf16_f32(kTileM, kTileN);

    uint32_t phase = 0;
    const int chunks = J.K / kChunkK;
    for (int ch = 0; ch < chunks; ++ch) {
        const int k0 = ch * kChunkK;
        // load and split: 128 rows x 64 columns of A and of B; each step issues eight
        // 16-byte loads before the first split so their latencies overlap
        constexpr int kVec = kTileM * (kChunkK / 4);  // float4 per operand and chunk
        constexpr int kBatch = 4;
#pragma unroll 1
        for (int i0 = threadIdx.x; i0 < kVec; i0 += kBatch * kGemmThreads) {
            float4 va[kBatch], vb[kBatch];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const int i = i0 + j * kGemmThreads;
                const int r = i / (kChunkK / 4), k = (i % (kChunkK / 4)) * 4;
                va[j] = __ldg(reinterpret_cast<const float4*>(J.A + (int64_t)(m0 + r) * J.lda + k0 + k));
                vb[j] = __ldg(reinterpret_cast<const float4*>(J.B + (int64_t)(n0 + r) * J.ldb + k0 + k));
            }
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const int i = i0 + j * kGemmThreads;
                const int r = i / (kChunkK / 4), k = (i % (kChunkK / 4)) * 4;
                split_store(va[j], A, sw128_offset(r, k));
                split_store(vb[j], B, sw128_offset(r, k));
            }
        }
        // make the generic-proxy stores visible to the tensor core, then issue
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
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
            mma_commit(smem_u32(&bar));
        }
        // the MMAs must finish reading shared memory before the next chunk overwrites it
        if (!mbar_wait(smem_u32(&bar), phase)) {
            atomicOr(status, kStatusTimeout);
            s_abort = 1;
        }
        phase ^= 1;
        __syncthreads();
        if (s_abort) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: warp w holds accumulator rows 32w .. 32w + 31 (TMEM lanes), 32 columns per load
    if (!s_abort) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < kTileN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                  "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                  "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (J.transpose_c) {
                // C^T: column n of the tile is row n of the output, rows consecutive across lanes
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    J.C[(int64_t)(n0 + c0 + j) * J.ldc + row] = __uint_as_float(v[j]);
            } else {
                float4* dst = reinterpret_cast<float4*>(J.C + (int64_t)row * J.ldc + n0 + c0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                         __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
            }
        }
    }
    // after a timeout the committed MMAs may still write the accumulator: wait for their
    // commit once more (bounded) and free the tensor memory only once they are done; if they
    // never finish it stays allocated (the status word already reports the timeout)
    __shared__ int s_drained;
    if (s_abort) {
        if (threadIdx.x == 0) s_drained = mbar_wait(smem_u32(&bar), phase ^ 1) ? 1 : 0;
        __syncthreads();
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
    return (int)cudaFuncSetAttribute(gemm_split3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kGemmSmem);
}

int launch_gemm(const GemmJob* jobs, const int* tile0, int n_jobs, int n_tiles, int* status, void* stream)
{
    if (n_tiles <= 0) return 0;
    gemm_split3_kernel<<<n_tiles, kGemmThreads, kGemmSmem, (cudaStream_t)stream>>>(jobs, tile0, n_jobs,
                                                                                    status);
    return (int)cudaGetLastError();
}

}  // namespace mci
