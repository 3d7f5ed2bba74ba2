// Internal structures shared by the host plan code and the CUDA kernels.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

#include "mci.h"

#ifdef __CUDACC__
#define MCI_HD __host__ __device__
#else
#define MCI_HD
#endif

namespace mci {

constexpr int kThreads = 256;      // threads per CTA of the interpolation kernels
constexpr int kMaxTile = 64;       // most signals (rows, columns) per CTA tile
constexpr int kSmemBudget = 64 * 1024;  // preferred dynamic shared memory per CTA

// Padded shared-memory index of complex element e of one FFT buffer: two
// complex of padding after every 32 keep strided Stockham stores free of bank
// conflicts and keep even elements 16-byte aligned (vector loads of pairs).
MCI_HD constexpr int pad16(int e) { return e + 2 * (e >> 5); }

// Division by a small runtime divisor d without a divide: n / d = (n * m) >> 32 with
// m = ceil(2^32 / d), exact for 0 <= n with n * d < 2^32 (buffer and item indices of a tile).
MCI_HD constexpr uint64_t fastdiv_magic(int d) { return ((1ull << 32) + (uint64_t)d - 1) / (uint64_t)d; }
MCI_HD inline int fastdiv(int n, uint64_t m) { return (int)(((uint64_t)(unsigned)n * m) >> 32); }
MCI_HD constexpr int padded_len(int n) { return ((pad16(n) + 1) / 2) * 2; }

// Radix plan of a length-n FFT, shared by the host (twiddle tables) and the
// kernels: E elements per thread; radix 16/8/4/2 on the power-of-two part and
// one radix-3 pass last where n has a factor 3.
MCI_HD constexpr int elems_per_thread(int n)
{
    return n % 3 == 0 ? (n >= 12 ? 12 : n) : (n >= 16 ? 16 : n);
}
MCI_HD constexpr int pick_radix(int rem, int E)
{
    return rem == 3 ? 3
         : (rem % 16 == 0 && E % 16 == 0) ? 16
         : (rem % 8 == 0 && E % 8 == 0) ? 8
         : (rem % 4 == 0 && E % 4 == 0) ? 4
         : 2;
}
// Shared-memory twiddles of a length-n FFT: for every pass with stride NS > 1 the
// NS values w^{jm} = e^{-2 pi i jm / (NS RAD)}, jm < NS, one pass after the other.
// smem_twiddle_offset(n, NS) is the first entry of the pass that starts at NS;
// smem_twiddle_count(n) the total.
MCI_HD constexpr int smem_twiddle_offset(int n, int NS)
{
    int off = 0, ns = 1;
    while (ns < NS) {
        const int rad = pick_radix(n / ns, elems_per_thread(n));
        if (ns > 1) off += ns;
        ns *= rad;
    }
    return off;
}
MCI_HD constexpr int smem_twiddle_count(int n) { return smem_twiddle_offset(n, n); }

// ---------------------------------------------------------------------------
// Fused radix-8 path (mci_fast.cu) for real FP32 classes with N = P/2 a power of
// two in [kFastMinN, kFastMaxN]: N/8 threads per signal, 2048/N signals per CTA.
// A transform of length N = 2^n takes ceil(n/3) passes of radix 8; the leftover
// factor 2^(n mod 3) is the first forward pass and the last inverse pass.
constexpr int kFastMinN = 128;
constexpr int kFastMaxN = 2048;
MCI_HD constexpr int ilog2(int n)
{
    int k = 0;
    while ((2 << k) <= n) ++k;
    return k;
}
MCI_HD constexpr int fast_passes(int N) { return (ilog2(N) + 2) / 3; }
MCI_HD constexpr int fast_radix(int N, int inv, int p)
{
    return ilog2(N) % 3 == 0 ? 8 : (p == (inv ? fast_passes(N) - 1 : 0) ? (1 << (ilog2(N) % 3)) : 8);
}
// stride NS of pass p: the product of the radices of the passes before it
MCI_HD constexpr int fast_ns(int N, int inv, int p)
{
    int ns = 1;
    for (int i = 0; i < p; ++i) ns *= fast_radix(N, inv, i);
    return ns;
}
// Per-class table of the fused path (complex, after the class's bin weights):
// e^{-2 pi i k / P} for k = 0..N, then for the forward (inv = 0) and the inverse
// (inv = 1) transform the NS entries e^{-2 pi i jm / (NS R)}, jm < NS, of every
// pass p >= 1 in order.  fast_tw_offset(N, 2, 0) is the table length.
MCI_HD constexpr int fast_tw_offset(int N, int inv, int p)
{
    int off = N + 1;
    for (int t = 0; t < 2; ++t)
        for (int q = 1; q < fast_passes(N); ++q) {
            if (t == inv && q == p) return off;
            off += fast_ns(N, t, q);
        }
    return off;
}
MCI_HD constexpr int fast_tw_count(int N) { return fast_tw_offset(N, 2, 0); }

// One size class as the kernels see it.
struct ClassDev {
    int P;       // samples per channel
    int N;       // FFT length P/2 (real transforms of length P packed as complex of N)
    int T;       // output samples
    int s;       // T / P
    int M_in;    // channels read from the input (M, or 1 in FD mode)
    int Q;       // output phases: s * n_out
    int QM;      // FFT buffers per signal in shared memory: max(M_in, Q)
    int G;       // signals per tile
    int n_out;   // outputs per signal
    int npad;    // padded FFT buffer length (complex elements)
    int sstride; // shared-memory stride between the tile's signals (complex elements):
                 // QM * npad rounded up to 2 mod 16, so that the buffers of consecutive
                 // signals start on different banks (16-byte aligned)
    int64_t w_off;   // offset of this class's bin weights W[k][m][q], k = 0..N
    uint64_t mag_min, mag_q, mag_nout;   // fastdiv_magic of M_in, Q and n_out
    int cplx;            // complex signals: FFT length N = P, complex samples and outputs
    int chan_len;        // reals per input channel: P, or 2 P for complex signals
    int64_t in_len;      // reals per signal: M_in * chan_len
    int64_t out_len;     // reals per signal: n_out * T (x 2 for complex signals)
    int fast;            // fused radix-8 kernel (mci_fast.cu): 1 + its variant index, or 0
    int tw_rel;          // fused path: offset (complex) of the class table after its weights
    int fast3;           // image columns on the fused factor-3 kernel (N = 3 N'), else 0
    int Gc;              // signals per column tile (G, or the factor-3 kernel's 2048 / N')
};

// Grouping of one mci_interp_1d call (uneven batches), built on the device or on the host.
struct Sched1D {
    int start[MCI_MAX_SIZES];          // first position of each class in the sorted list
    int count[MCI_MAX_SIZES];          // signals per class
    unsigned next_tile;                // work counter of the persistent launch (zero per call)
};

// What the device-side scheduler needs to launch one size class.
struct ClassLaunch {
    ClassDev c;
    const void* W;
    int prec;
    int smem;
    int smem_cols;   // dynamic shared memory of the class's column kernel
};

enum StatusBits {
    kStatusBadClass = 1,
    kStatusBadImage = 2,
    kStatusBadOffset = 4,
    kStatusBatch = 8,
    kStatusIntermediate = 16,
    kStatusLaunch = 32,
    kStatusTimeout = 64,
};

// One GEMM of the small-P image path: C[M x N] = A[M x K] * B[N x K]^T (FP32 operands,
// split into BF16 planes on the tensor cores), C stored row-major or transposed.
struct GemmJob {
    const float* A;          // plus a_off[img] when a_off is set
    const float* B;
    float* C;                // plus c_off[img] when c_off is set
    const int64_t* a_off;    // device per-image offsets, or NULL
    const int64_t* c_off;
    int64_t lda, ldb, ldc;
    int M, N, K;
    int img;
    int transpose_c;
    const char* a_planes;    // A (or B) pre-split into BF16 plane tiles at plan time, or NULL
    const char* b_planes;    // (at most one of the two)
};

// Device-built work lists of one mci_upsample_2d call: per size class, the
// row-pass and column-pass items (image, tile) in one list.
struct Sched2D {
    int row_start[MCI_MAX_SIZES];
    int row_count[MCI_MAX_SIZES];
    int col_start[MCI_MAX_SIZES];
    int col_count[MCI_MAX_SIZES];
};

// Arguments of the averaged-error evaluator (Eq. (averageerror), Eq. (errorestimate)).
struct ErrArgs {
    const double2* G;        // per residue r: G_r[m][m'] = sum_l conj(r_m) r_m' over the M
                             // aliases, at G[(r * M + m) * M + m']
    const double2* coeffs;   // [batch][2 n_max + 1]: a(n), n = -n_max .. n_max
    double* eps;             // [batch]
    double* bound;           // [batch] or NULL
    int64_t N1, mu, n_max, batch;
    int M, P;
    int kind[MCI_MAX_CHANNELS], order[MCI_MAX_CHANNELS];
    double tau[MCI_MAX_CHANNELS];
    double omega_sum;        // sum over m of Omega_m = sup_i |r_m(i)|^2
};
int launch_averaged_error(const ErrArgs& a, void* stream);

enum KernelMode { kModeUniform = 0, kModeSorted = 1, kModeRows = 2, kModeCols = 3 };

// Arguments of one size-class launch (passed by value).
struct KArgs {
    ClassDev c;              // this launch's size class
    int cls;                 // its index
    int mode;                // KernelMode
    const void* in;          // 1-D: samples; rows: LR images; cols: intermediate
    void* out;               // 1-D: outputs; rows: intermediate; cols: HR images
    const void* W;           // this class's bin weights (cpx<R>)
    // 1-D
    const int64_t* in_off;   // per signal, or NULL (packed)
    const int64_t* out_off;
    int64_t batch;
    int uniform_items;
    int qchunks;             // > 1: the phases of every tile are spread over gridDim.y CTAs
    const int64_t* sorted;   // signals sorted by class
    const Sched1D* sched1;
    // 2-D
    const int2* items;       // (image, tile) lists of all classes
    const Sched2D* sched2;
    const int* h;
    const int* w;
    const int* scale;
    const int64_t* img_in_off;   // LR image offsets
    const int64_t* img_out_off;  // HR image offsets
    const int64_t* inter_off;    // intermediate image offsets
    int* status;
};

// Kernel for (precision, column pattern, FFT length), or NULL when not compiled.
const void* kernel_lookup(int precision, bool cols, int N);
// Fused radix-8 kernel for (N, input channels, scale, outputs), or NULL when not compiled;
// *variant (if not NULL) receives its index in the persistent kernel's dispatch.
const void* fast_kernel_lookup(int N, int M_in, int s, int n_out, int* variant = nullptr);
// Its column-pass counterpart for image plans (separable 2-D), or NULL.
const void* fast_cols_kernel_lookup(int N, int M_in, int s, int n_out);
// Variants 0 .. kFastPersistentVariants - 1 are the ones the persistent kernel dispatches.
constexpr int kFastPersistentVariants = 5;
// Image columns of length P = 6 N' (N = 3 N', N' a power of two) on the fused factor-3
// kernel: its table layout after the class weights is e^{-2 pi i k / P} (k = 0..N), the
// per-pass twiddles of the length-N' transforms (as fast_tw_offset(N', ..) lays them out
// after N' + 1 entries), then e^{-2 pi i k / N} for k < N'.
const void* fast3_cols_kernel_lookup(int N, int M_in, int s, int n_out);
MCI_HD constexpr int fast3_table_count(int Nq) { return 3 * Nq + 1 + fast_tw_count(Nq) - (Nq + 1) + Nq; }
constexpr int kFastMaxImageN = 512;   // image rows and columns on the fused path: N <= 512

// One persistent launch over an uneven batch whose classes are all on the fused path: the
// CTAs take tiles from sched->next_tile (zero at launch), classes in `order` (largest P
// first), the signals of class c at sorted[start[c] ..], offsets in_off / out_off.
struct PersistArgs {
    const ClassLaunch* cl;
    const int* order;
    int n_classes;
    Sched1D* sched;
    const int64_t* sorted;
    const float* in;
    float* out;
    const int64_t* in_off;
    const int64_t* out_off;
};
const void* fast_persistent_kernel();

int launch_sched_1d(const int* size_class, int64_t batch, int n_classes, const ClassLaunch* cl,
                    const int* order, int64_t* sorted, Sched1D* st, int64_t* in_pref,
                    int64_t* out_pref, const KArgs& tmpl, void* stream, int persist);
int launch_sched_2d(int64_t n_img, int n_classes, const ClassLaunch* cl, int64_t max_inter,
                    int64_t max_items, int64_t* inter_off, int64_t* lr_pref, int64_t* hr_pref,
                    int* row_cls, int* col_cls, int2* items, Sched2D* st, const KArgs& rows_tmpl,
                    const KArgs& cols_tmpl, void* stream, int child);

// Tensor-core GEMM (mci_gemm.cu): tile0 is the tile prefix over jobs (n_jobs + 1).
int launch_gemm(const GemmJob* jobs, const int* tile0, int n_jobs, int n_tiles, int* status,
                void* stream);
int prepare_gemm();
int gemm_smem_bytes();
// Plane tiles of a constant rows x cols matrix (rows % 128 == 0, cols % 64 == 0).
int64_t gemm_plane_bytes(int rows, int cols);
int presplit_gemm(const float* K, int rows, int cols, char* out, void* stream);

// Static scratch of mci_interp_1d_noalloc (mci_noalloc.cu).
struct NoAllocScratch;
NoAllocScratch* noalloc_scratch(cudaError_t* err);
int64_t* noalloc_sorted(NoAllocScratch* s);
int64_t* noalloc_in_pref(NoAllocScratch* s);
int64_t* noalloc_out_pref(NoAllocScratch* s);
Sched1D* noalloc_sched(NoAllocScratch* s);

}  // namespace mci
