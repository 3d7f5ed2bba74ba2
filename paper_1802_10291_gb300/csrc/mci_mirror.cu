// Mirror (half-sample-symmetric) image boundaries for the separable 2-D path.
//
// The method interpolates 2 pi-periodic signals (Section 2), so an image is treated as one
// period of a periodic image and its left and right (top and bottom) edges meet: content
// that differs across them rings near the borders.  mci_upsample_2d_mirror reflects each
// h x w image about its edges to 2h x 2w (sample P + n repeats sample P - 1 - n), runs the
// periodic path of mci_upsample_2d on the extension, and keeps the s h x s w block over the
// original image.  The per-image sizes travel in the kernels' parameters; the caller
// provides both scratch buffers, so nothing is allocated.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mci.h"

namespace {

constexpr int kMirrorMaxImages = 256;

struct MirrorDims {
    int n;
    int h[kMirrorMaxImages];
    int w[kMirrorMaxImages];
    int s[kMirrorMaxImages];
};

// image i's offset in a packed array of images of f * (h_j w_j) pixels, j < i
__device__ __forceinline__ int64_t packed_offset(const MirrorDims& d, int i, bool hr, int f)
{
    int64_t off = 0;
    for (int j = 0; j < i; ++j) off += (int64_t)d.h[j] * d.w[j] * (hr ? d.s[j] * d.s[j] : 1);
    return off * f;
}

// Extension of image blockIdx.y: row r of 2h is row r (r < h) or 2h - 1 - r of the image,
// column x of 2w likewise.
__global__ void mirror_extend_kernel(const float* __restrict__ lr, float* __restrict__ ext, const MirrorDims d)
{
    const int i = blockIdx.y;
    if (i >= d.n) return;
    const int h = d.h[i], w = d.w[i];
    const float* src0 = lr + packed_offset(d, i, false, 1);
    float* dst0 = ext + packed_offset(d, i, false, 4);
    for (int r = blockIdx.x; r < 2 * h; r += gridDim.x) {
        const float* src = src0 + (int64_t)(r < h ? r : 2 * h - 1 - r) * w;
        float* dst = dst0 + (int64_t)r * 2 * w;
        for (int x = threadIdx.x; x < 2 * w; x += blockDim.x) dst[x] = src[x < w ? x : 2 * w - 1 - x];
    }
}

// The s h x s w block at the top left of image blockIdx.y's interpolated extension (rows of
// 2 s w pixels) into the packed output.
__global__ void mirror_crop_kernel(const float* __restrict__ ext_hr, float* __restrict__ hr, const MirrorDims d)
{
    const int i = blockIdx.y;
    if (i >= d.n) return;
    const int H = d.s[i] * d.h[i], W = d.s[i] * d.w[i];
    const float* src0 = ext_hr + packed_offset(d, i, true, 4);
    float* dst0 = hr + packed_offset(d, i, true, 1);
    for (int r = blockIdx.x; r < H; r += gridDim.x) {
        const float* src = src0 + (int64_t)r * 2 * W;
        float* dst = dst0 + (int64_t)r * W;
        for (int x = threadIdx.x; x < W; x += blockDim.x) dst[x] = src[x];
    }
}

}  // namespace

extern "C" mci_status mci_upsample_2d_mirror(mci_plan_t plan, const float* lr, const int* h, const int* w,
                                             const int* scale, float* hr, int64_t n_img, float* ext_lr,
                                             float* ext_hr, mci_stream_t stream)
{
    if (!plan || n_img < 0) return MCI_ERR_INVALID_ARG;
    if (n_img == 0) return MCI_OK;
    if (n_img > kMirrorMaxImages) return MCI_ERR_UNSUPPORTED_SIZE;
    if (!lr || !h || !w || !scale || !hr || !ext_lr || !ext_hr) return MCI_ERR_INVALID_ARG;
    // the kernels below read and write these four directly: device (or managed) memory only
    for (const void* ptr : {(const void*)lr, (const void*)hr, (const void*)ext_lr, (const void*)ext_hr}) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
            cudaGetLastError();
            return MCI_ERR_INVALID_ARG;
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return MCI_ERR_INVALID_ARG;
    }
    MirrorDims d{};
    d.n = (int)n_img;
    std::vector<int> h2((size_t)n_img), w2((size_t)n_img);
    int max_rows = 1, max_hr_rows = 1;
    for (int64_t i = 0; i < n_img; ++i) {
        if (h[i] <= 0 || w[i] <= 0 || scale[i] <= 0 || h[i] > (1 << 20) || w[i] > (1 << 20))
            return MCI_ERR_INVALID_ARG;
        d.h[i] = h[i];
        d.w[i] = w[i];
        d.s[i] = scale[i];
        h2[(size_t)i] = 2 * h[i];
        w2[(size_t)i] = 2 * w[i];
        max_rows = std::max(max_rows, 2 * h[i]);
        max_hr_rows = std::max(max_hr_rows, scale[i] * h[i]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    mirror_extend_kernel<<<dim3((unsigned)std::min(max_rows, 4096), (unsigned)n_img), 256, 0, s>>>(lr, ext_lr, d);
    if (cudaGetLastError() != cudaSuccess) return MCI_ERR_CUDA;
    const mci_status st =
        mci_upsample_2d(plan, ext_lr, nullptr, h2.data(), w2.data(), scale, ext_hr, nullptr, n_img, stream);
    if (st != MCI_OK) return st;
    mirror_crop_kernel<<<dim3((unsigned)std::min(max_hr_rows, 4096), (unsigned)n_img), 256, 0, s>>>(ext_hr, hr, d);
    return cudaGetLastError() == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}
