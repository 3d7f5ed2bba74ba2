/*
 * mci.h -- C ABI of the GB300-native FFT multichannel interpolation library.
 *
 * Method: Cheng & Kou, "FFT multichannel interpolation and application to
 * image super-resolution".  A periodic signal f on [0, 2 pi) is observed
 * through M linear systems with Fourier multipliers b_m(n) (Section 3,
 * Eq. (sysfunction)); each response g_m is sampled P times at t_p = 2 pi p / P
 * (the paper calls P "L").  The library reconstructs f -- or its circular
 * Hilbert transform, or its derivative -- on the grid t_j = 2 pi j / T from
 * those M*P samples, assuming f is bandlimited to the band
 * {N1, ..., N1 + M*P - 1} (Eq. (bandsignal)), or approximating it there when it
 * is not (operator T_N, Eq. (appxi operator)).  The computation follows the
 * FFT form of Theorem (MCIeq), Eq. (DFTexpression): an FFT of every channel,
 * a per-residue solve with the inverse of the M x M system matrix H_n of
 * Eq. (defH) (Eq. (matrixeqn1)), and an inverse FFT that evaluates the
 * result.  Images are processed separably, rows then columns (Section 5.2).
 *
 * Conventions shared by every entry point:
 *   - All sample and pixel buffers are DEVICE pointers owned by the caller.
 *     The library never frees them and never keeps them past a call.
 *   - Streams are cudaStream_t values passed as void*; NULL is the legacy
 *     default stream.  Every call except mci_plan, mci_plan_info and
 *     mci_destroy is asynchronous and stream-ordered: it only enqueues work.
 *   - Errors are returned as mci_status.  A call that returns an error has
 *     enqueued nothing.  Errors that only the device can see (a size class
 *     index out of range, an image size the plan does not hold) make the
 *     kernels skip the affected signal or image and set a device status word
 *     that mci_plan_info reports.
 *   - No call allocates device memory except mci_plan (tables and workspace), and
 *     mci_interp_1d_host when it stages buffers for a plan made with host_access 0 (its
 *     first such call allocates the chunk buffers; a plan made with host_access 1 holds
 *     them from mci_plan on).
 *   - The result of a real-sample reconstruction is the real part of the
 *     band-limited interpolant, as in the experiments of Section 5.1.
 */
#ifndef MCI_H
#define MCI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mci_plan_s* mci_plan_t;   /* opaque; owned by the library */
typedef void* mci_stream_t;              /* a cudaStream_t */

typedef enum {
    MCI_OK = 0,
    MCI_ERR_INVALID_ARG = -1,      /* null pointer, bad enum, inconsistent sizes */
    MCI_ERR_UNSUPPORTED_SIZE = -2, /* P, T or a buffer the kernels cannot take */
    MCI_ERR_SINGULAR = -3,         /* a system matrix is singular under MCI_SINGULAR_ERROR */
    MCI_ERR_CUDA = -4,             /* a CUDA runtime call failed */
    MCI_ERR_OOM = -5,              /* device allocation failed in mci_plan */
    MCI_ERR_TIMEOUT = -6,          /* a device-side bounded wait gave up */
    MCI_ERR_DEVICE = -7            /* a device-side check failed (see mci_plan_info) */
} mci_status;

/* Linear systems (the paper's h_m / b_m(n), Eq. (sysfunction)). */
enum {
    MCI_SYS_IDENTITY = 0, /* b(n) = 1                                   */
    MCI_SYS_DERIV = 1,    /* b(n) = (i n)^order, order >= 1 (Example 2)  */
    MCI_SYS_HILBERT = 2,  /* b(n) = -i sgn(n) (Examples 3, 5)            */
    MCI_SYS_SHIFT = 3,    /* b(n) = e^{i n tau}                          */
    MCI_SYS_CUSTOM = 4    /* b(n) from a host table, see mci_system      */
};

typedef struct {
    int kind;             /* MCI_SYS_*                                                   */
    int order;            /* MCI_SYS_DERIV: derivative order (1 or more)                 */
    double tau;           /* MCI_SYS_SHIFT: shift                                        */
    const double* custom; /* MCI_SYS_CUSTOM: host table read during mci_plan only: for
                             each size class c in order, 2*M*P_c doubles (re, im) of b(n)
                             for n = N1_c .. N1_c + M*P_c - 1                            */
} mci_system;

/* Output operators applied to the reconstruction (Example 6, and the remark
 * closing Section 3 on reconstructing Q(f)).  OR-able; outputs are stored in
 * the order F, HILBERT, DERIV. */
enum {
    MCI_OUT_F = 1,       /* f itself                       */
    MCI_OUT_HILBERT = 2, /* circular Hilbert transform of f (Section 2) */
    MCI_OUT_DERIV = 4    /* f'                             */
};

enum { MCI_FP32 = 0, MCI_FP64 = 1 };

/* What to do where H_n is singular (Remark (aequal0)). */
enum {
    MCI_SINGULAR_PINV = 0,  /* Moore-Penrose pseudo-inverse: minimum-norm solution of
                               A_n H_n = D_n (Eq. (matrixeqn1)); default            */
    MCI_SINGULAR_ERROR = 1, /* mci_plan fails with MCI_ERR_SINGULAR                  */
    MCI_SINGULAR_ZERO = 2   /* q_{mk}(n) = 0 at that residue, as Remark (aequal0)     */
};

/* Where the channels come from. */
enum {
    MCI_CHANNELS_MEASURED = 0, /* the caller passes all M channels' samples            */
    MCI_CHANNELS_FD = 1        /* the caller passes one channel (system 0, which must be
                                  the identity); the others are its three-point centred
                                  differences (Section 5.2): first derivative
                                  (x[p+1] - x[p-1]) / (2h), second derivative
                                  (x[p+1] - 2x[p] + x[p-1]) / h^2, h = 2 pi / P, periodic.
                                  Only MCI_SYS_IDENTITY and MCI_SYS_DERIV (order 1, 2). */
};

#define MCI_MAX_CHANNELS 8
#define MCI_MAX_SIZES 32

typedef struct {
    int M;                   /* channels, 1 .. MCI_MAX_CHANNELS                            */
    const mci_system* sys;   /* M systems (host, read during mci_plan only)                */
    int n_sizes;             /* size classes, 1 .. MCI_MAX_SIZES                           */
    const int* P;            /* n_sizes samples-per-channel values (host)                  */
    const int* T;            /* n_sizes output lengths (host); each a positive multiple of
                                its P                                                      */
    const int64_t* N1;       /* n_sizes band starts (host), or NULL for -floor(M*P/2)      */
    unsigned out_flags;      /* OR of MCI_OUT_*; 2-D requires exactly MCI_OUT_F            */
    int precision;           /* MCI_FP32 or MCI_FP64: type of samples and outputs          */
    int singular_policy;     /* MCI_SINGULAR_*                                             */
    double singular_rtol;    /* residue singular when sigma_min < rtol * sigma_max;
                                <= 0 selects 1e-13                                         */
    int channel_mode;        /* MCI_CHANNELS_*                                             */
    int64_t max_batch;       /* most signals one mci_interp_1d call passes (>= 1)          */
    int64_t max_images;      /* most images one mci_upsample_2d call passes (0: no 2-D)    */
    int64_t max_intermediate;/* most row-pass pixels one mci_upsample_2d call needs:
                                sum over images of h * s * w (0: no 2-D)                   */
    int autotune;            /* 0: tile height G (signals per CTA) from a fixed shared-memory
                                budget; 1: mci_plan times candidate G for every size class
                                on a scratch batch (zeros, about 64 MB of device memory held
                                during the call) and keeps the fastest.  Results do not
                                depend on G; plan creation takes longer (milliseconds per
                                class).  There is no counterpart in the paper.           */
    int complex_signal;      /* 0: real signals; samples and outputs are real, the output is
                                the real part of the interpolant (Section 5.1 examples).
                                1: complex signals (Examples 4, 5): samples and outputs are
                                complex, interleaved (re, im) in the precision's type, input
                                [M][P] complex per signal, output [n_out][T] complex, and no
                                real part is taken.  Requires MCI_CHANNELS_MEASURED and no
                                2-D (max_images = 0); P a power of two up to 4096 or 3 * 2^a
                                from 6 to 3072, and one signal's max(M, s * n_out) buffers of
                                P complex values must fit in shared memory (else
                                MCI_ERR_UNSUPPORTED_SIZE; e.g. FP64 M = 3, s = 2, P = 4096). */
    int blur_taps;           /* 0: no blur.  Otherwise an odd tap count, 1 .. 255: the blur-aware
                                channel model that Section 5.2 leaves as an open extension.
                                Every channel is taken to be its system's response circularly
                                convolved, before sampling, with the normalised Gaussian
                                w_k = exp(-k^2 / (2 blur_sigma^2)) / sum_j (same), |k| <= taps/2,
                                on the output grid (spacing 2 pi / T of the size class; in 2-D
                                along each axis, i.e. the separable taps x taps Gaussian of the
                                paper's degradation).  Its multiplier beta(n) = sum_k w_k
                                e^{-2 pi i n k / T} then multiplies every b_m(n).            */
    double blur_sigma;       /* standard deviation in output samples, > 0 when blur_taps > 0  */
    double blur_lambda;      /* >= 0.  0: exact model, the unblurred model's reconstruction
                                divided by beta(n) (where |beta(n)| < singular_rtol the factor
                                follows singular_policy: 0 for PINV and ZERO, MCI_ERR_SINGULAR
                                for ERROR; such frequencies add to n_singular).  > 0: Wiener-
                                type regularisation, the unblurred model's reconstruction times
                                (1 + lambda) conj beta(n) / (|beta(n)|^2 + lambda), which is 1
                                at n = 0.  Plans with a blur take no mci_averaged_error.    */
    int host_access;         /* mci_interp_1d_host only.  0: when both buffers are page-locked
                                and mapped into the device address space (cudaHostAlloc /
                                cudaHostRegister, as reported by cudaPointerGetAttributes), the
                                kernels can read the input and write the output in host memory
                                directly over the host link, without staging copies; the first
                                three such calls on the plan time that route and the staged
                                one (the second call stages untimed) and the plan keeps the
                                faster per byte (mci_plan_stats.host_route; the plan keeps
                                that state, so one plan's host calls must not run from several
                                host threads at once); other buffers are staged.
                                1: always stage through device chunks.  */
} mci_desc;

typedef struct {
    int n_singular;          /* singular residues over all size classes                   */
    double max_cond;         /* largest sigma_max / sigma_min over non-singular residues  */
    int device_status;       /* device status word since the last query (0: clean);
                                bit 0 bad size class, bit 1 bad image size, bit 2 bad
                                offset / alignment, bit 3 batch above max_batch,
                                bit 4 intermediate above max_intermediate, bit 5 a
                                device-side kernel launch failed                          */
    int signals_per_cta[MCI_MAX_SIZES]; /* tile height chosen per size class              */
    int threads_per_cta;
    int smem_bytes;          /* dynamic shared memory per CTA                             */
    int64_t table_bytes;     /* device bytes of per-residue tables and twiddles           */
    int64_t workspace_bytes; /* device bytes of the 1-D and 2-D workspace                 */
    unsigned fused_mask;     /* bit c: size class c runs on the fused radix-8 kernel      */
    int persistent_ctas;     /* grid of the one persistent launch that serves uneven
                                batches when every class is fused (0: one launch per class) */
    unsigned fused3_mask;    /* bit c: the image columns of size class c (N = 3 N') run on
                                the fused factor-3 column kernel                            */
    int host_route;          /* mci_interp_1d_host with device-mapped buffers (host_access
                                0): 0 still measuring, 1 zero copy, 2 staged                */
} mci_plan_stats;

/*
 * mci_plan -- build a plan: validate the description, form every per-residue
 * system matrix H_r[j][k] = b_k(N1 + r + j P) of every size class in FP64
 * (Eq. (defH)), invert it by a singular value decomposition (pseudo-inverse
 * or zero or error where singular, Remark (aequal0)), fold the inverse, the
 * output operator and the evaluation phases into per-bin tables, round them to
 * the plan's precision and upload them, and allocate the workspace.
 * *plan receives the plan on success.  Synchronises the stream.  Supported
 * sizes: P even with P = 2^a (4 <= P <= 8192) or 3 * 2^a (12 <= P <= 6144),
 * T a multiple of P, and the per-CTA working set within shared memory;
 * otherwise MCI_ERR_UNSUPPORTED_SIZE.
 */
mci_status mci_plan(mci_plan_t* plan, const mci_desc* desc, mci_stream_t stream);

/*
 * mci_interp_1d -- reconstruct a batch of 1-D signals (Theorem (MCIeq),
 * Eq. (DFTexpression); operator T_N of Eq. (appxi operator)).
 *   in         device, samples of signal b: in + in_off[b] holds M_in x P_c values
 *              (channel-major: channel m at [m * P_c + p]); M_in = M for measured
 *              channels, 1 for MCI_CHANNELS_FD.  Element type per precision.
 *   in_off     device int64 element offsets, or NULL: signals packed back to back
 *   out        device, out + out_off[b] receives n_out x T_c values (n_out = number
 *              of bits in out_flags), output-major, out[o * T_c + j] = value at
 *              t_j = 2 pi j / T_c
 *   out_off    device int64 element offsets, or NULL: packed back to back
 *   size_class int per signal (0 .. n_sizes-1), or NULL when n_sizes == 1.  In
 *              DEVICE memory the batch is grouped by size class on the device and
 *              each class's kernel is launched from there (stream-capturable;
 *              class indices out of range set device_status bit 0).  In HOST
 *              memory the call groups the batch on the host (reading the array
 *              before it returns), uploads the grouping from pinned staging and
 *              launches each class from the host on plan-owned streams forked
 *              from and joined into `stream` -- the faster path; an index out of
 *              range returns MCI_ERR_INVALID_ARG; not for stream capture.
 *   batch      number of signals, 0 .. max_batch
 * Offsets that are multiples of 4 elements (FP32) or 2 (FP64) take the
 * vectorised path; others work but run slower.
 */
mci_status mci_interp_1d(mci_plan_t plan, const void* in, const int64_t* in_off, void* out,
                         const int64_t* out_off, const int* size_class, int64_t batch,
                         mci_stream_t stream);

/*
 * mci_upsample_2d -- separable 2-D interpolation of Section 5.2: every row of
 * an h x w image is interpolated from w samples to s*w, then every column of
 * that h x (s w) intermediate from h samples to s*h.  Channels come from the
 * plan's channel mode (FD derivatives of the pixel row/column, or M = 1).
 * The plan must hold a size class (w, s*w) and a class (h, s*h) for every
 * image (the same class serves both when h == w).
 *   lr       device float, image i at lr + lr_off[i], h_i x w_i row-major
 *   lr_off   device int64 element offsets, or NULL (packed)
 *   h, w     int arrays of image heights and widths
 *   scale    int array of scale factors s_i >= 1.  h, w and scale all in DEVICE
 *            memory: the batch is grouped on the device; the size classes are launched
 *            from the host with grids bounded by the plan's limits (extra CTAs exit at
 *            once) when those bounds are small, else from the device
 *            (stream-capturable either way; bad sizes set device_status bits).  All in HOST
 *            memory: grouping on the host, one upload from pinned staging,
 *            exact-grid launches per class from the host -- the faster path;
 *            an image size the plan does not hold returns
 *            MCI_ERR_UNSUPPORTED_SIZE; not for stream capture.
 *   hr       device float, image i at hr + hr_off[i], (s h) x (s w) row-major
 *   hr_off   device int64 element offsets, or NULL (packed)
 *   n_img    number of images, 0 .. max_images
 * Only MCI_FP32 plans.  Uses the plan's workspace for the intermediate, so
 * calls on one plan must not overlap on the device.
 */
mci_status mci_upsample_2d(mci_plan_t plan, const float* lr, const int64_t* lr_off, const int* h,
                           const int* w, const int* scale, float* hr, const int64_t* hr_off,
                           int64_t n_img, mci_stream_t stream);

/*
 * mci_upsample_2d_mirror -- mci_upsample_2d with mirror image boundaries.  The method
 * interpolates periodic signals (Section 2), so mci_upsample_2d treats an image as one period
 * and its opposite edges meet; here each h x w image is first reflected about its edges to
 * 2h x 2w (row or column P + n repeats P - 1 - n), that extension is interpolated as a
 * periodic image, and the (s h) x (s w) block over the original image is written to hr.  The
 * paper leaves the image boundary open; mirror extension is the usual remedy for the ringing
 * of the periodic wrap.
 *   lr       device float, packed h_i x w_i images
 *   h, w     HOST int arrays; the plan must hold the classes (2 w, 2 s w) and (2 h, 2 s h),
 *            max_images >= n_img and max_intermediate >= sum 4 s_i h_i w_i
 *   scale    HOST int array of scale factors
 *   hr       device float, packed (s h) x (s w) images
 *   n_img    0 .. 256 (MCI_ERR_UNSUPPORTED_SIZE above)
 *   ext_lr   device float scratch of sum 4 h_i w_i elements (the extended images)
 *   ext_hr   device float scratch of sum 4 s_i^2 h_i w_i elements (their interpolation)
 * The caller owns both scratch buffers (the call allocates nothing); they, the plan's
 * workspace and hr are written on `stream`, so calls on one plan or one scratch must not
 * overlap.  Errors: as mci_upsample_2d; MCI_ERR_INVALID_ARG when lr, hr or a scratch
 * buffer is not device (or managed) memory.
 */
mci_status mci_upsample_2d_mirror(mci_plan_t plan, const float* lr, const int* h, const int* w,
                                  const int* scale, float* hr, int64_t n_img, float* ext_lr,
                                  float* ext_hr, mci_stream_t stream);

/*
 * mci_interp_1d_noalloc -- the same computation as mci_interp_1d, with the
 * same arguments except that size_class must be in DEVICE (or managed)
 * memory, for callers that cannot allocate device memory at the time
 * they know their batch: code running under global-mode stream capture (where
 * cudaMalloc is refused), and code whose device memory is handed out up front
 * by a framework or a fixed budget.  Such a caller creates its plan once at
 * start-up (max_batch may then be 1) and passes batches of up to
 * MCI_NOALLOC_MAX_BATCH signals here.  The paper has no counterpart: this is
 * an interface of this library only.
 *   Scratch (the signal grouping and packed offsets of uneven batches) lives in
 *   one static device array of about 1.5 MiB that every GPU loading the library
 *   holds until exit; no call allocates or frees device memory.  The first call
 *   on a device looks up that array's device address (cudaGetSymbolAddress)
 *   and caches it, so make the first call on each device before any stream
 *   capture.  All calls share the array: calls that overlap on the GPU (other
 *   streams, other threads) race on it and must be serialised by the caller.
 *   Every call rewrites all of the scratch it reads, so nothing needs clearing.
 *   The cached address belongs to the device's current context: after
 *   cudaDeviceReset the module may load elsewhere, so a process that resets a
 *   device must not call this entry point on that device again.
 *   batch > MCI_NOALLOC_MAX_BATCH returns MCI_ERR_UNSUPPORTED_SIZE; a plan
 *   with several size classes and a NULL or host-memory size_class returns
 *   MCI_ERR_INVALID_ARG.
 */
#define MCI_NOALLOC_MAX_BATCH 65536
mci_status mci_interp_1d_noalloc(mci_plan_t plan, const void* in, const int64_t* in_off, void* out,
                                 const int64_t* out_off, const int* size_class, int64_t batch,
                                 mci_stream_t stream);

/*
 * mci_interp_1d_host -- mci_interp_1d on HOST buffers (packed signals).  With
 * mci_desc.host_access = 0 and both buffers page-locked and device-mapped, the kernels
 * access them in place (zero copy).  Otherwise the library copies the input to the device,
 * interpolates and copies the output back: the batch is cut into chunks of consecutive
 * signals (about 16 MB of input each) that move through three internal streams -- copy
 * in, compute, copy out -- so that transfers in both directions overlap each other and
 * the compute.
 *   in, out      HOST, packed as in mci_interp_1d with NULL offsets; page-locked memory
 *                (cudaHostAlloc / registered) lets the copies run asynchronously.
 *   size_class   HOST array of batch class indices (NULL for a one-class plan).
 * The chunk buffers (three slots of input and output) belong to the plan: with
 * host_access 1 mci_plan allocates them, sized for any batch (a chunk holds at most
 * max(16 MB, one signal) of input), so no call allocates; with host_access 0 the first
 * call that stages allocates them and keeps them with the plan.  Work already queued on
 * `stream` runs first; the call returns when `out` holds the result (synchronous).
 * Errors: as mci_interp_1d; MCI_ERR_OOM when the chunk buffers cannot be allocated
 * (host_access 0 only; with host_access 1 mci_plan reports it).
 * There is no counterpart in the paper.
 */
mci_status mci_interp_1d_host(mci_plan_t plan, const void* in, void* out, const int* size_class, int64_t batch,
                              mci_stream_t stream);

/*
 * mci_averaged_error -- the phase-averaged approximation error eps(f, N) of Eq.
 * (averageerror) (Section 4, Theorem (error)) for a batch of signals given by their
 * Fourier coefficients, and the Cauchy-Schwarz bound of Eq. (errorestimate):
 *   eps^2 = sum_{n not in I} |a(n)|^2 (1 + sum_{l=1..M} |sum_m r_m(n + (l-k)P) b_m(n)|^2),
 *   bound^2 = sum_{n not in I} |a(n)|^2 + M (sum_m Omega_m) sum_{n not in I} sum_m |a(n) b_m(n)|^2,
 * with r_m the plan's per-residue inverse (Eq. (defrm)) of class size_class, k the block
 * of n and Omega_m = sup_i |r_m(i)|^2 (the bound reads the square on Omega in Eq.
 * (errorestimate) as a slip: Cauchy-Schwarz gives sum_m Omega_m).  FP64 throughout.
 *   coeffs  DEVICE, batch x (2 n_max + 1) complex values (re, im interleaved, FP64):
 *           a(n) for n = -n_max .. n_max; coefficients beyond n_max are taken as 0.
 *   n_max   must cover the band I of the class (and stay below 2^29).
 *   eps     DEVICE, batch doubles (output); bound DEVICE, batch doubles or NULL.
 * Requires measured channels (MCI_CHANNELS_MEASURED) and no MCI_SYS_CUSTOM system
 * (its multiplier is known only inside the band): otherwise MCI_ERR_INVALID_ARG.
 * Stream-ordered; the plan's precision does not matter (its FP64 inverses are used).
 */
mci_status mci_averaged_error(mci_plan_t plan, int size_class, const double* coeffs, int64_t n_max,
                              int64_t batch, double* eps, double* bound, mci_stream_t stream);

/* mci_plan_info -- fill *stats; synchronises the plan's last stream to read the
 * device status word, then clears it. */
mci_status mci_plan_info(mci_plan_t plan, mci_plan_stats* stats);

/* mci_destroy -- release the plan's device tables, workspace and streams
 * (synchronises its streams first).  NULL is a no-op. */
mci_status mci_destroy(mci_plan_t plan);

/* mci_error_string -- static description of a status code. */
const char* mci_error_string(mci_status status);

/*
 * mci_debug_fail_allocation -- test hook: the device and page-locked allocations made by
 * mci_plan and mci_interp_1d_host succeed `after` more times, then one is refused as if the
 * device were out of memory (the call returns MCI_ERR_OOM and frees what it had allocated);
 * after that, allocations succeed again.  A negative value switches the hook off (the default).
 * Process-wide; not for use while other threads create plans.  The paper has no counterpart:
 * it lets the out-of-memory paths be tested without exhausting a GPU.
 */
void mci_debug_fail_allocation(int after);

/*
 * mci_tune_cache_save / mci_tune_cache_load -- the tile heights picked by the plan-time
 * autotuner (mci_desc.autotune) are kept process-wide, keyed by kernel kind, precision, real
 * or complex signals, P, T, input channels, output phases and device (name and
 * multiprocessor count); a plan whose class has an entry uses it without timing.  save writes
 * them to `path` as a flat JSON object {"key": tile_height, ...}; load merges such a file
 * (keys as save writes them, values 1 .. 64).  Host only: no device work.  Errors:
 * MCI_ERR_INVALID_ARG for a NULL path, a file that cannot be opened or a malformed file
 * (nothing is merged then).  The paper has no counterpart: an interface of this library.
 */
mci_status mci_tune_cache_save(const char* path);
mci_status mci_tune_cache_load(const char* path);

#ifdef __cplusplus
}
#endif
#endif /* MCI_H */
