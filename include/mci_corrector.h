/*
 * mci_corrector.h -- learned residual corrector on top of MCI image upsampling,
 * and the on-device generator of its synthetic training images.
 *
 * The paper has no trained component; its closing list of limitations
 * (Section 5.2) suggests using MCI inside learning-based super-resolution.
 * This is that: a 5-layer 3x3 convolutional network f with channels
 * 1 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU between layers, bias, periodic padding,
 * applied to an MCI reconstruction x:  pred = x + f(x).  Weights are BF16 in
 * the convolutions (FP32 master copies), activations and accumulation FP32; the
 * 32 -> 32 convolutions run on the tensor cores with each FP32 activation split
 * into two BF16 terms (hi + lo), the others on the CUDA cores.
 * Training minimises the mean squared error of pred against the HR image with
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8).  Plain MCI stays the fallback: with
 * the last layer's weights and bias zero, pred = x exactly.
 *
 * Parameter layout (flat FP32, mci_corrector_num_params() values): for layer
 * l = 0..4, weights [cout][cin][3][3] then bias [cout].
 *
 * All image buffers are DEVICE pointers, [batch][h][w] FP32 row-major; calls
 * are stream-ordered unless stated.  Status codes as in mci.h.
 */
#ifndef MCI_CORRECTOR_H
#define MCI_CORRECTOR_H

#include "mci.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mci_corrector_s* mci_corrector_t;

/* Floats of generator parameters per image (see mci_generate_images). */
#define MCI_IMAGE_PARAMS 192

/* Number of trainable parameters (28353). */
int mci_corrector_num_params(void);

/* Create a corrector for batches of up to max_pixels = batch * h * w pixels.
 * init_params: host array of mci_corrector_num_params() floats, or NULL for zeros.
 * Allocates device memory (parameters, Adam moments, activations); synchronises. */
mci_status mci_corrector_create(mci_corrector_t* net, int64_t max_pixels, const float* init_params,
                                mci_stream_t stream);

/* out = mci + f(mci) (inference). */
mci_status mci_corrector_forward(mci_corrector_t net, const float* mci, float* out, int batch, int h,
                                 int w, mci_stream_t stream);

/* Loss L = mean (mci + f(mci) - hr)^2 over all pixels and its gradient with respect
 * to every parameter (device grad_out of num_params floats, device loss_out scalar;
 * either may be NULL). */
mci_status mci_corrector_loss_grad(mci_corrector_t net, const float* mci, const float* hr, int batch,
                                   int h, int w, float* grad_out, float* loss_out, mci_stream_t stream);

/* One Adam step on L with learning rate lr; loss_out (device, may be NULL) receives L
 * before the step. */
mci_status mci_corrector_train_step(mci_corrector_t net, const float* mci, const float* hr, int batch,
                                    int h, int w, float lr, float* loss_out, mci_stream_t stream);

/* Checkpoint: host buffer of 3 * num_params floats (master weights, first and second
 * moments) and the Adam step count.  Both synchronise the device. */
mci_status mci_corrector_get_state(mci_corrector_t net, float* host, int* step);
mci_status mci_corrector_set_state(mci_corrector_t net, const float* host, int step);

/* Device-side error word of the corrector's kernels since the last call: bit 0 = a
 * tensor-core completion wait gave up (the tile was skipped; outputs are invalid).
 * Synchronises the device and clears the word. */
mci_status mci_corrector_status(mci_corrector_t net, int* status);

mci_status mci_corrector_destroy(mci_corrector_t net);

/* Synthetic grayscale images in [0, 1]: 0.5 + 20 anisotropic Gaussian blobs + 10 straight
 * edges + 8 low-frequency waves, clipped.  params: device, n * MCI_IMAGE_PARAMS floats per
 * image: blobs (cy, cx, 1/sigma_major, 1/sigma_minor, angle, amplitude) x 20, edges
 * (py, px, angle, step) x 10, waves (cycles_y, cycles_x, phase, amplitude) x 8, in pixels. */
mci_status mci_generate_images(const float* params, float* img, int n, int h, int w,
                               mci_stream_t stream);

/* Pure decimation lr[y][x] = hr[s y][s x] of n images h x w (h, w multiples of s;
 * 1 <= n <= 65535). */
mci_status mci_decimate(const float* hr, float* lr, int n, int h, int w, int s, mci_stream_t stream);

/* The degradation of the paper's super-resolution experiment (Section 5.2): blur by the
 * taps x taps Gaussian of standard deviation sigma (pixels; normalised outer product of
 * w_k = exp(-k^2 / (2 sigma^2)), |k| <= taps / 2; periodic boundary), then decimate by s:
 * lr[y][x] = sum_{i,j} w_i w_j hr[(s y - i) mod h][(s x - j) mod w].  taps odd, 1 .. 255,
 * sigma > 0; otherwise as mci_decimate.  FP32 accumulation. */
mci_status mci_degrade(const float* hr, float* lr, int n, int h, int w, int s, int taps, double sigma,
                       mci_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MCI_CORRECTOR_H */
