// Host side of the C ABI: plan construction in FP64 and the stream-ordered
// entry points.  See include/mci.h for the contract of every function.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mci_internal.h"
#include "mci_linalg.h"

using cd = std::complex<double>;

namespace mci {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// e^{2 pi i q / den}, q reduced modulo den in integers first.
cd cis_frac(int64_t q, int64_t den)
{
    q %= den;
    if (q < 0) q += den;
    const double a = kTwoPi * (double)q / (double)den;
    return cd(std::cos(a), std::sin(a));
}

int sgn(int64_t n) { return (n > 0) - (n < 0); }

// Fourier multiplier b(n) of one system (Eq. (sysfunction); Examples 2, 3, 5).
cd system_multiplier(const mci_system& s, const double* custom_class, int64_t N1, int64_t n)
{
    switch (s.kind) {
    case MCI_SYS_IDENTITY: return 1.0;
    case MCI_SYS_DERIV: {
        cd v = 1.0;
        for (int i = 0; i < s.order; ++i) v *= cd(0.0, (double)n);
        return v;
    }
    case MCI_SYS_HILBERT: return cd(0.0, -(double)sgn(n));
    case MCI_SYS_SHIFT: return cd(std::cos((double)n * s.tau), std::sin((double)n * s.tau));
    case MCI_SYS_CUSTOM: {
        const int64_t i = n - N1;
        return cd(custom_class[2 * i], custom_class[2 * i + 1]);
    }
    }
    return 0.0;
}

// Output operators (Example 6): f, Hilbert transform, derivative.
cd output_multiplier(int op, int64_t n)
{
    if (op == MCI_OUT_HILBERT) return cd(0.0, -(double)sgn(n));
    if (op == MCI_OUT_DERIV) return cd(0.0, (double)n);
    return 1.0;
}

// Blur-aware channel model (the extension Section 5.2 leaves open): each channel is
// blurred before sampling by the normalised Gaussian w_k, |k| <= K, on the T-grid, whose
// multiplier is beta(n) = sum_k w_k e^{-2 pi i n k / T}.  Returns the factor the unblurred
// model's reconstruction is multiplied by at frequency n: 1 / beta(n) (lambda = 0) or
// (1 + lambda) conj beta / (|beta|^2 + lambda); *singular set where lambda = 0 and
// |beta(n)| < rtol (the factor is then 0).
cd blur_output_factor(const mci_desc& d, const std::vector<double>& w, int T, int64_t n, double rtol,
                      bool* singular)
{
    const int K = d.blur_taps / 2;
    cd beta = 0.0;
    for (int k = -K; k <= K; ++k) beta += w[k + K] * cis_frac(-n * (int64_t)k, T);
    *singular = false;
    if (d.blur_lambda > 0.0) return (1.0 + d.blur_lambda) * std::conj(beta) / (std::norm(beta) + d.blur_lambda);
    if (std::abs(beta) < rtol) {
        *singular = true;
        return 0.0;
    }
    return 1.0 / beta;
}

std::vector<double> blur_taps_of(const mci_desc& d)
{
    const int K = d.blur_taps / 2;
    std::vector<double> w(2 * K + 1);
    double sum = 0.0;
    for (int k = -K; k <= K; ++k) sum += (w[k + K] = std::exp(-(double)k * k / (2.0 * d.blur_sigma * d.blur_sigma)));
    for (double& v : w) v /= sum;
    return w;
}

// One-sided (Hestenes) Jacobi SVD of an M x M complex matrix, row-major:
// on return A holds U * diag(sigma) column-wise, V the right singular vectors.
void jacobi_svd(int M, std::vector<cd>& A, std::vector<cd>& V)
{
    V.assign(M * M, 0.0);
    for (int i = 0; i < M; ++i) V[i * M + i] = 1.0;
    for (int sweep = 0; sweep < 80; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < M - 1; ++i)
            for (int j = i + 1; j < M; ++j) {
                double alpha = 0.0, beta = 0.0;
                cd gamma = 0.0;
                for (int r = 0; r < M; ++r) {
                    alpha += std::norm(A[r * M + i]);
                    beta += std::norm(A[r * M + j]);
                    gamma += std::conj(A[r * M + i]) * A[r * M + j];
                }
                const double g = std::abs(gamma);
                if (g == 0.0 || alpha == 0.0 || beta == 0.0) continue;
                off = std::max(off, g / std::sqrt(alpha * beta));
                if (g <= 1e-300) continue;
                const cd ph = gamma / g;  // e^{i phi}
                const double zeta = (beta - alpha) / (2.0 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int r = 0; r < M; ++r) {
                    const cd ai = A[r * M + i], aj = A[r * M + j] * std::conj(ph);
                    A[r * M + i] = c * ai - s * aj;
                    A[r * M + j] = s * ai + c * aj;
                    const cd vi = V[r * M + i], vj = V[r * M + j] * std::conj(ph);
                    V[r * M + i] = c * vi - s * vj;
                    V[r * M + j] = s * vi + c * vj;
                }
            }
        if (off < 1e-16) break;
    }
}

struct ResidueInverse {
    std::vector<cd> Q;  // P x M x M: Q[(r*M + m)*M + j], channel m, alias j
    int n_singular = 0;
    double max_cond = 1.0;
};

// H_r[j][k] = b_k(N1 + r + j P) (Eq. (defH)); Q_r = H_r^{-1} or its pseudo-inverse.
mci_status invert_residues(const mci_desc& d, int P, int64_t N1, const double* const* custom,
                           double rtol, ResidueInverse& out)
{
    const int M = d.M;
    out.Q.assign((size_t)P * M * M, 0.0);
    std::vector<cd> H(M * M);
    for (int r = 0; r < P; ++r) {
        const int64_t n = N1 + r;
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < M; ++k)
                H[j * M + k] = system_multiplier(d.sys[k], custom[k], N1, n + (int64_t)j * P);
        bool singular = false;
        double cond = 1.0;
        const mci_status st = invert_system(M, H, rtol, d.singular_policy, &out.Q[(size_t)r * M * M],
                                            &singular, &cond);
        if (st != MCI_OK) return st;
        if (singular) ++out.n_singular;
        else out.max_cond = std::max(out.max_cond, cond);
    }
    return MCI_OK;
}

// Complex signals use a length-P complex FFT (no packing): P must be a kernel FFT length.
bool supported_complex_p(int P)
{
    if (P < 2) return false;
    int q = P;
    bool three = false;
    if (q % 3 == 0) {
        q /= 3;
        three = true;
    }
    if (q & (q - 1)) return false;
    if (three) return P >= 6 && P <= 3072;
    return P <= 4096;
}

bool supported_p(int P)
{
    if (P < 4 || P % 2) return false;
    int q = P;
    bool three = false;
    if (q % 3 == 0) {
        q /= 3;
        three = true;
    }
    if (q & (q - 1)) return false;  // remaining part must be a power of two
    if (three) return P >= 12 && P <= 6144;
    return P <= 8192;
}

struct HostClass {
    int P, T, s, N;
    int64_t N1;
};

}  // namespace

// Q = H^{-1} of one M x M system matrix (row-major H[j * M + k]), or its Moore-Penrose
// pseudo-inverse V Sigma^+ U^H where sigma_min < rtol sigma_max (Remark (aequal0)); Q[m * M + j].
mci_status invert_system(int M, std::vector<cd> H, double rtol, int policy, cd* Q, bool* singular,
                         double* cond)
{
    std::vector<cd> V;
    for (int i = 0; i < M * M; ++i) Q[i] = 0.0;
    jacobi_svd(M, H, V);
    std::vector<double> sig(M);
    double smax = 0.0;
    for (int k = 0; k < M; ++k) {
        double nn = 0.0;
        for (int row = 0; row < M; ++row) nn += std::norm(H[row * M + k]);
        sig[k] = std::sqrt(nn);
        smax = std::max(smax, sig[k]);
    }
    double smin = smax;
    for (int k = 0; k < M; ++k) smin = std::min(smin, sig[k]);
    *singular = !(smax > 0.0) || smin < rtol * smax;
    *cond = smax > 0.0 && smin > 0.0 ? smax / smin : 0.0;
    if (*singular) {
        if (policy == MCI_SINGULAR_ERROR) return MCI_ERR_SINGULAR;
        if (policy == MCI_SINGULAR_ZERO || !(smax > 0.0)) return MCI_OK;  // Q = 0
    }
    // U[:,k] = H[:,k] / sigma_k
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < M; ++j) {
            cd acc = 0.0;
            for (int k = 0; k < M; ++k) {
                if (!(sig[k] > rtol * smax) || sig[k] == 0.0) continue;
                const cd u_jk = H[j * M + k] / sig[k];
                acc += V[m * M + k] * std::conj(u_jk) / sig[k];
            }
            Q[m * M + j] = acc;
        }
    return MCI_OK;
}

}  // namespace mci

using namespace mci;

struct mci_plan_s {
    mci_desc desc{};
    std::vector<mci_system> sys;
    std::vector<HostClass> cls;
    std::vector<ClassDev> cdev;
    std::vector<ClassLaunch> launch;  // host copy of d_launch
    std::vector<const void*> kern;    // per class host kernel (contiguous pattern)
    std::vector<const void*> kern_cols;
    std::vector<int> csmem;           // per class dynamic shared memory
    std::vector<int> csmem_cols;      // per class dynamic shared memory of the column kernel
    int n_sm = 0;                     // multiprocessors of the plan's device
    int persist = 0;                  // uneven batches: one persistent launch (all classes fused)
    int persist_ctas = 0;             // its grid: resident CTAs per SM x SMs
    int persist_smem = 0;
    int n_out = 0;
    int M_in = 0;
    int smem = 0;                     // largest per-class shared memory
    int n_singular = 0;
    double max_cond = 1.0;
    std::vector<int> order;           // class ids by descending P
    size_t elem = 4;                  // sizeof(real)
    int64_t max_items = 0;            // 2-D work-list capacity
    // device memory
    void* d_tables = nullptr;         // launch info | order | W
    ClassLaunch* d_launch = nullptr;
    int* d_order = nullptr;
    void* d_W = nullptr;
    int64_t table_bytes = 0;
    void* d_work = nullptr;           // 1-D and 2-D workspace
    int64_t work_bytes = 0;
    int* d_status = nullptr;
    int64_t* d_sorted = nullptr;
    int64_t* d_in_pref = nullptr;
    int64_t* d_out_pref = nullptr;
    Sched1D* d_sched1 = nullptr;
    float* d_inter = nullptr;
    int64_t* d_inter_off = nullptr;
    int64_t* d_lr_pref = nullptr;
    int64_t* d_hr_pref = nullptr;
    int* d_row_cls = nullptr;
    int* d_col_cls = nullptr;
    int2* d_items = nullptr;
    Sched2D* d_sched2 = nullptr;
    cudaStream_t last_stream = nullptr;
    // host-grouped uneven batches: per-class streams, fork/join events, pinned staging
    std::vector<cudaStream_t> cstreams;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    char* h_stage[2] = {nullptr, nullptr};   // mirrors the device block d_sorted .. d_sched1
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    size_t off_in_pref = 0, off_out_pref = 0, off_sched1 = 0;  // offsets inside the block
    int stage_cur = 0;
    // host-grouped 2-D: staging mirrors the device block d_inter_off .. end of d_hws
    int* d_hws = nullptr;                    // device copies of h, w, scale (3 x max_images)
    char* h_stage2[2] = {nullptr, nullptr};
    cudaEvent_t ev_stage2[2] = {nullptr, nullptr};
    size_t stage2_bytes = 0;
    size_t o2_lrp = 0, o2_hrp = 0, o2_it = 0, o2_s2 = 0, o2_hws = 0;
    int stage2_cur = 0;
    // tensor-core image path: per class offset of the T x P matrix in gemm_tab (-1: none)
    std::vector<float> gemm_tab;
    std::vector<int64_t> gemm_off;
    std::vector<const float*> d_kmap;
    void* d_gemm = nullptr;
    void* d_kplanes = nullptr;          // each class's K pre-split into BF16 plane tiles
    std::vector<const char*> d_kp;
    GemmJob* d_jobs = nullptr;
    int* d_tile0 = nullptr;
    size_t o2_jobs = 0, o2_tile0 = 0;
    // averaged-error evaluator: per class and residue the M x M matrix G_r (FP64 complex)
    // and the sum of Omega_m
    std::vector<double> rtab;            // host staging
    std::vector<int64_t> rtab_off;       // per class offset in complex elements
    std::vector<double> omega_sum;
    void* d_rtab = nullptr;
    // host-buffer entry point: chunk buffers and the copy-in / compute / copy-out pipeline
    static constexpr int kSlots = 3;
    void* d_chunk = nullptr;             // kSlots x (chunk input | chunk output)
    size_t chunk_in_bytes = 0, chunk_out_bytes = 0;
    // host_access 0 with device-mapped buffers: 0 times the zero-copy route next, 1 runs the
    // staged route untimed (it may allocate), 2 times it, 3 decided (host_zero_copy)
    int host_trial = 0;
    bool host_zero_copy = true;
    double host_rate[2] = {0.0, 0.0};    // bytes per second: zero copy, staged
    cudaStream_t hs[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_in[kSlots] = {}, ev_comp[kSlots] = {}, ev_free[kSlots] = {};
};

namespace {

// Test hook of mci_debug_fail_allocation: allocations left before one is refused (-1: off).
std::atomic<int> g_fail_after{-1};

bool refuse_allocation()
{
    int c = g_fail_after.load();
    while (c >= 0 && !g_fail_after.compare_exchange_weak(c, c - 1)) {
    }
    return c == 0;
}

// device-grouped 2-D batches: classes are launched from the host with bounded grids when the
// bounds of all classes add up to at most this many CTAs
constexpr int64_t kBoundedCtas = 16384;

// host-buffer path: input bytes per chunk of consecutive signals (one signal may exceed it)
constexpr int64_t kChunkIn = (int64_t)16 << 20;

cudaError_t dev_malloc(void** ptr, size_t bytes)
{
    if (refuse_allocation()) return cudaErrorMemoryAllocation;
    return cudaMalloc(ptr, bytes);
}

cudaError_t pinned_alloc(void** ptr, size_t bytes)
{
    if (refuse_allocation()) return cudaErrorMemoryAllocation;
    return cudaHostAlloc(ptr, bytes, cudaHostAllocDefault);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

mci_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return MCI_OK;
    if (e == cudaErrorMemoryAllocation) return MCI_ERR_OOM;
    return MCI_ERR_CUDA;
}

mci_status validate(const mci_desc* d)
{
    if (!d || d->M < 1 || d->M > MCI_MAX_CHANNELS || !d->sys) return MCI_ERR_INVALID_ARG;
    if (d->n_sizes < 1 || d->n_sizes > MCI_MAX_SIZES || !d->P || !d->T) return MCI_ERR_INVALID_ARG;
    if (d->out_flags == 0 || (d->out_flags & ~7u)) return MCI_ERR_INVALID_ARG;
    if (d->precision != MCI_FP32 && d->precision != MCI_FP64) return MCI_ERR_INVALID_ARG;
    if (d->singular_policy < 0 || d->singular_policy > 2) return MCI_ERR_INVALID_ARG;
    if (d->channel_mode != MCI_CHANNELS_MEASURED && d->channel_mode != MCI_CHANNELS_FD)
        return MCI_ERR_INVALID_ARG;
    if (d->max_batch < 1 || d->max_images < 0 || d->max_intermediate < 0) return MCI_ERR_INVALID_ARG;
    for (int k = 0; k < d->M; ++k) {
        const mci_system& s = d->sys[k];
        if (s.kind < MCI_SYS_IDENTITY || s.kind > MCI_SYS_CUSTOM) return MCI_ERR_INVALID_ARG;
        if (s.kind == MCI_SYS_DERIV && s.order < 1) return MCI_ERR_INVALID_ARG;
        if (s.kind == MCI_SYS_CUSTOM && !s.custom) return MCI_ERR_INVALID_ARG;
        if (d->channel_mode == MCI_CHANNELS_FD) {
            if (k == 0 && s.kind != MCI_SYS_IDENTITY) return MCI_ERR_INVALID_ARG;
            if (k > 0 && !(s.kind == MCI_SYS_DERIV && (s.order == 1 || s.order == 2)))
                return MCI_ERR_INVALID_ARG;
        }
    }
    if (d->blur_taps < 0 || d->blur_taps > 255 || (d->blur_taps > 0 && d->blur_taps % 2 == 0))
        return MCI_ERR_INVALID_ARG;
    if (d->blur_taps > 0 && !(d->blur_sigma > 0.0 && std::isfinite(d->blur_sigma) &&
                              d->blur_lambda >= 0.0 && std::isfinite(d->blur_lambda)))
        return MCI_ERR_INVALID_ARG;
    if (d->complex_signal != 0 && d->complex_signal != 1) return MCI_ERR_INVALID_ARG;
    if (d->host_access != 0 && d->host_access != 1) return MCI_ERR_INVALID_ARG;
    if (d->complex_signal && (d->channel_mode != MCI_CHANNELS_MEASURED || d->max_images > 0))
        return MCI_ERR_INVALID_ARG;
    for (int c = 0; c < d->n_sizes; ++c) {
        if (!(d->complex_signal ? supported_complex_p(d->P[c]) : supported_p(d->P[c])))
            return MCI_ERR_UNSUPPORTED_SIZE;
        if (d->T[c] < d->P[c] || d->T[c] % d->P[c]) return MCI_ERR_UNSUPPORTED_SIZE;
        for (int c2 = 0; c2 < c; ++c2)
            if (d->P[c2] == d->P[c] && d->T[c2] == d->T[c] &&
                (!d->N1 || d->N1[c2] == d->N1[c]))
                return MCI_ERR_INVALID_ARG;  // duplicate size class
    }
    if (d->max_images > 0 && d->precision != MCI_FP32) return MCI_ERR_INVALID_ARG;
    if (d->max_images > 0 && d->out_flags != MCI_OUT_F) return MCI_ERR_INVALID_ARG;
    if (d->max_images > 0 && d->channel_mode == MCI_CHANNELS_MEASURED && d->M != 1)
        return MCI_ERR_INVALID_ARG;
    return MCI_OK;
}

// FD spectral factor of system k on bin k of a length-P real DFT (Section 5.2 centred differences).
cd fd_factor(const mci_system& s, int P, int k)
{
    if (s.kind == MCI_SYS_IDENTITY) return 1.0;
    const double h = kTwoPi / P;
    const cd e = cis_frac(k, P);
    if (s.order == 1) return (e - std::conj(e)) / (2.0 * h);           // i sin(2 pi k/P) / h
    return (e - 2.0 + std::conj(e)) / (h * h);                          // (2 cos - 2) / h^2
}

template <typename R>
void push_cpx(std::vector<R>& v, cd z)
{
    v.push_back((R)z.real());
    v.push_back((R)z.imag());
}

// Image size classes small enough for the tensor-core path: the T x P matrix of the
// linear map is formed by the plan, and both passes of an image run as GEMMs when
// its row and column classes are both eligible.
// Image classes served by the tensor-core route (two dense products per image).  Its work
// grows with P * T while the FFT route's grows with T log P; measured per batch (GEMM vs
// FFT route, M = 2): 64 x 128^2 x2 0.055 vs 0.073 ms, 64 x 128^2 x4 0.111 vs 0.115 ms,
// 64 x 256^2 x2 0.226 vs 0.152 ms, 16 x 256^2 x3 0.133 vs 0.093 ms, 32 x 256^2 x4 0.349 vs
// 0.202 ms -- so it takes P = 128 with T <= 512 only.  Its FP32 accumulation error is
// also several times that of the FFT route: 4.4e-6 x RMS with M = 2 systems {f, f'} but
// 1.06e-5 x RMS with M = 3 {f, f', f''} (over the 1e-5 FP32 tolerance; the FFT route gives
// 1.0e-6 per pass) on a 256^2 -> 768^2 image, so it takes M <= 2 only.
bool gemm_eligible(const mci_plan_s* p, const HostClass& hc)
{
    const mci_desc& d = p->desc;
    return d.max_images > 0 && d.precision == MCI_FP32 && p->M_in == 1 && d.M <= 2 && p->n_out == 1 &&
           hc.P == 128 && hc.T % 128 == 0 && hc.T <= 512;
}

template <typename R>
mci_status build_tables(mci_plan_s* p, std::vector<R>& W)
{
    const mci_desc& d = p->desc;
    const int M = d.M, Min = p->M_in, nout = p->n_out;
    const double rtol = d.singular_rtol > 0 ? d.singular_rtol : 1e-13;
    std::vector<int> ops;
    for (int o : {MCI_OUT_F, MCI_OUT_HILBERT, MCI_OUT_DERIV})
        if (d.out_flags & o) ops.push_back(o);
    size_t custom_off = 0;
    for (size_t c = 0; c < p->cls.size(); ++c) {
        const HostClass& hc = p->cls[c];
        const int P = hc.P, N = hc.N, s = hc.s, T = hc.T, Q = s * nout;
        std::vector<const double*> custom(M, nullptr);
        for (int k = 0; k < M; ++k)
            if (d.sys[k].kind == MCI_SYS_CUSTOM) custom[k] = d.sys[k].custom + custom_off;
        custom_off += (size_t)2 * M * P;
        ResidueInverse inv;
        mci_status st = invert_residues(d, P, hc.N1, custom.data(), rtol, inv);
        if (st != MCI_OK) return st;
        p->n_singular += inv.n_singular;
        p->max_cond = std::max(p->max_cond, inv.max_cond);
        // averaged-error evaluator: with r_m(N1 + l P + r) = Q_r[m][l] (Eq. (defrm)),
        // sum_l |sum_m r_m(n + (l - k) P) b_m(n)|^2 = b^H G_r b for n in residue r, with
        // G_r[m][m'] = sum_l conj(Q_r[m][l]) Q_r[m'][l]; stored per r (M x M complex)
        p->rtab_off[c] = (int64_t)(p->rtab.size() / 2);
        for (int r = 0; r < P; ++r)
            for (int m = 0; m < M; ++m)
                for (int m2 = 0; m2 < M; ++m2) {
                    cd acc = 0.0;
                    for (int l = 0; l < M; ++l)
                        acc += std::conj(inv.Q[((size_t)r * M + m) * M + l]) * inv.Q[((size_t)r * M + m2) * M + l];
                    p->rtab.push_back(acc.real());
                    p->rtab.push_back(acc.imag());
                }
        double osum = 0.0;   // sum over m of Omega_m = sup |r_m|^2 (bound of Eq. (errorestimate))
        for (int m = 0; m < M; ++m) {
            double om = 0.0;
            for (int j = 0; j < M; ++j)
                for (int r = 0; r < P; ++r) om = std::max(om, std::norm(inv.Q[((size_t)r * M + m) * M + j]));
            osum += om;
        }
        p->omega_sum[c] = osum;
        std::vector<cd> omega;   // blur factor over the band, n = N1 .. N1 + M P - 1
        if (d.blur_taps > 0) {
            const std::vector<double> w = blur_taps_of(d);
            omega.resize((size_t)M * P);
            for (int64_t i = 0; i < (int64_t)M * P; ++i) {
                bool sing = false;
                omega[i] = blur_output_factor(d, w, T, hc.N1 + i, rtol, &sing);
                if (sing) {
                    ++p->n_singular;
                    if (d.singular_policy == MCI_SINGULAR_ERROR) return MCI_ERR_SINGULAR;
                }
            }
        }
        ClassDev& cd_ = p->cdev[c];
        if ((W.size() / 2) % 2) push_cpx(W, cd(0.0));  // 16-byte aligned class region
        cd_.w_off = (int64_t)(W.size() / 2);
        // W_r[m][q] = (1/P) sum_j Q_r[m][j] o(n_j) omega(n_j) e^{2 pi i n_j u / T},
        // n_j = N1 + r + j P (omega = 1 without a blur)
        auto Wfull = [&](int r, int m, int q) {
            const int o = ops[q / s], u = q % s;
            cd acc = 0.0;
            for (int j = 0; j < M; ++j) {
                const int64_t n = hc.N1 + r + (int64_t)j * P;
                const cd om = omega.empty() ? cd(1.0) : omega[(size_t)(r + (int64_t)j * P)];
                acc += inv.Q[((size_t)r * M + m) * M + j] * output_multiplier(o, n) * om *
                       cis_frac(n * (int64_t)u, T);
            }
            return acc / (double)P;
        };
        auto res = [&](int k) { return (int)((((int64_t)k - hc.N1) % P + P) % P); };
        std::vector<cd> Wk((size_t)M * Q);
        const bool gemm = gemm_eligible(p, hc);
        std::vector<cd> w1;  // single-input-channel weights per bin, phase (GEMM matrix)
        if (gemm) w1.assign((size_t)(N + 1) * Q, 0.0);
        if (d.complex_signal) {
            // complex signals: every bin k < P on its own, no symmetrisation; plane (m, q)
            // holds W[k][m][q] = Wfull(residue of k, m, q) for k = 0..P-1
            std::vector<cd> cplanes((size_t)Min * Q * P);
            for (int k = 0; k < P; ++k) {
                const int r = res(k);
                for (int m = 0; m < Min; ++m)
                    for (int q = 0; q < Q; ++q) cplanes[((size_t)m * Q + q) * P + k] = Wfull(r, m, q);
            }
            for (const cd& z : cplanes) push_cpx(W, z);
            continue;
        }
        // stored as planes: plane (m, q) holds W[k][m][q] for k = 0..N contiguously, so the
        // threads of a warp (consecutive bins) read consecutive elements of a plane
        std::vector<cd> planes((size_t)Min * Q * (N + 1));
        for (int k = 0; k <= N; ++k) {
            const int ra = res(k), rb = res((P - k) % P);
            for (int m = 0; m < M; ++m)
                for (int q = 0; q < Q; ++q)
                    Wk[(size_t)m * Q + q] = 0.5 * (Wfull(ra, m, q) + std::conj(Wfull(rb, m, q)));
            if (d.channel_mode == MCI_CHANNELS_FD) {
                for (int q = 0; q < Q; ++q) {
                    cd acc = 0.0;
                    for (int m = 0; m < M; ++m) acc += fd_factor(d.sys[m], P, k) * Wk[(size_t)m * Q + q];
                    planes[(size_t)q * (N + 1) + k] = acc;
                    if (gemm) w1[(size_t)k * Q + q] = acc;
                }
            } else {
                for (int m = 0; m < Min; ++m)
                    for (int q = 0; q < Q; ++q) planes[((size_t)m * Q + q) * (N + 1) + k] = Wk[(size_t)m * Q + q];
                if (gemm)
                    for (int q = 0; q < Q; ++q) w1[(size_t)k * Q + q] = Wk[q];
            }
        }
        for (const cd& z : planes) push_cpx(W, z);
        if (cd_.fast) {
            // fused-path table: e^{-2 pi i k / P}, k = 0..N, then the per-pass twiddles
            // e^{-2 pi i jm / (NS R)}, jm < NS, of the forward and the inverse transform
            if ((W.size() / 2) % 2) push_cpx(W, cd(0.0));
            cd_.tw_rel = (int)((int64_t)(W.size() / 2) - cd_.w_off);
            for (int k = 0; k <= N; ++k) push_cpx(W, cis_frac(-(int64_t)k, P));
            for (int inv = 0; inv < 2; ++inv)
                for (int ps = 1; ps < fast_passes(N); ++ps) {
                    const int ns = fast_ns(N, inv, ps), rad = fast_radix(N, inv, ps);
                    for (int jm = 0; jm < ns; ++jm) push_cpx(W, cis_frac(-(int64_t)jm, (int64_t)ns * rad));
                }
        }
        if (cd_.fast3) {
            // factor-3 column table: e^{-2 pi i k / P}, k = 0..N; the per-pass twiddles of the
            // length-N' transforms (N' = N / 3); e^{-2 pi i k / N}, k < N'
            const int Nq = N / 3;
            if ((W.size() / 2) % 2) push_cpx(W, cd(0.0));
            cd_.tw_rel = (int)((int64_t)(W.size() / 2) - cd_.w_off);
            for (int k = 0; k <= N; ++k) push_cpx(W, cis_frac(-(int64_t)k, P));
            for (int inv = 0; inv < 2; ++inv)
                for (int ps = 1; ps < fast_passes(Nq); ++ps) {
                    const int ns = fast_ns(Nq, inv, ps), rad = fast_radix(Nq, inv, ps);
                    for (int jm = 0; jm < ns; ++jm) push_cpx(W, cis_frac(-(int64_t)jm, (int64_t)ns * rad));
                }
            for (int k = 0; k < Nq; ++k) push_cpx(W, cis_frac(-(int64_t)k, N));
        }
        if (gemm) {
            // out[s l + u] = sum_p kappa_u[(l - p) mod P] x[p], kappa_u[d] = sum over all P bins of
            // W_k[u] e^{2 pi i k d / P} with W_{P-k} = conj W_k (the kernel's real inverse FFT)
            p->gemm_off[c] = (int64_t)p->gemm_tab.size();
            std::vector<double> kappa((size_t)s * P);
            for (int u = 0; u < s; ++u)
                for (int dd = 0; dd < P; ++dd) {
                    double acc = w1[(size_t)0 * Q + u].real() + w1[(size_t)N * Q + u].real() * ((dd & 1) ? -1.0 : 1.0);
                    for (int k = 1; k < N; ++k) acc += 2.0 * (w1[(size_t)k * Q + u] * cis_frac((int64_t)k * dd, P)).real();
                    kappa[(size_t)u * P + dd] = acc;
                }
            for (int j = 0; j < T; ++j) {
                const int l = j / s, u = j % s;
                for (int q = 0; q < P; ++q)
                    p->gemm_tab.push_back((float)kappa[(size_t)u * P + (((l - q) % P) + P) % P]);
            }
        }
    }
    return MCI_OK;
}

}  // namespace

// One persistent launch over the grouped batch (sorted, st in device memory; st->next_tile is
// zero when it starts).  tiles < 0: not known on the host (grouped on the device).
static cudaError_t launch_persistent(mci_plan_t p, const KArgs& a, const int64_t* sorted, Sched1D* st,
                                     const int64_t* in_off, const int64_t* out_off, int64_t tiles,
                                     cudaStream_t s)
{
    PersistArgs pa{};
    pa.cl = p->d_launch;
    pa.order = p->d_order;
    pa.n_classes = (int)p->cls.size();
    pa.sched = st;
    pa.sorted = sorted;
    pa.in = static_cast<const float*>(a.in);
    pa.out = static_cast<float*>(a.out);
    pa.in_off = in_off;
    pa.out_off = out_off;
    int64_t grid = p->persist_ctas;
    if (tiles >= 0) grid = std::min(grid, tiles);
    if (grid <= 0) return cudaSuccess;
    void* args[] = {&pa};
    return cudaLaunchKernel(fast_persistent_kernel(), dim3((unsigned)grid), dim3(kThreads), args,
                            (size_t)p->persist_smem, s);
}

// Uneven batch whose size classes are in host memory: stable grouping on the host
// into a pinned staging block (two blocks alternate; a block is reused only after
// its previous upload has completed), one upload, then every non-empty class is
// launched from the host with its exact grid on its own stream, forked from and
// joined back into the caller's stream.
static mci_status interp_1d_host_grouped(mci_plan_t p, KArgs a, const int* size_class, int64_t batch,
                                         cudaStream_t s)
{
    const int n = (int)p->cls.size();
    char* blk = p->h_stage[p->stage_cur];
    cudaEvent_t ev = p->ev_stage[p->stage_cur];
    if (cudaEventSynchronize(ev) != cudaSuccess) return MCI_ERR_CUDA;
    int64_t* sorted = (int64_t*)blk;
    int64_t* in_pref = (int64_t*)(blk + p->off_in_pref);
    int64_t* out_pref = (int64_t*)(blk + p->off_out_pref);
    Sched1D* st = (Sched1D*)(blk + p->off_sched1);
    std::vector<int64_t> cnt(n, 0), pos(n, 0);
    for (int64_t b = 0; b < batch; ++b) {
        const int c = size_class[b];
        if (c < 0 || c >= n) return MCI_ERR_INVALID_ARG;
        ++cnt[c];
    }
    int64_t acc = 0;
    for (int oi = 0; oi < n; ++oi) {
        const int c = p->order[oi];
        pos[c] = acc;
        st->start[c] = (int)acc;
        st->count[c] = (int)cnt[c];
        acc += cnt[c];
    }
    int64_t pin = 0, pout = 0;
    for (int64_t b = 0; b < batch; ++b) {
        const int c = size_class[b];
        sorted[pos[c]++] = b;
        in_pref[b] = pin;
        out_pref[b] = pout;
        pin += p->cdev[c].in_len;
        pout += p->cdev[c].out_len;
    }
    st->next_tile = 0;
    cudaError_t e = cudaMemcpyAsync(p->d_sorted, blk, p->stage_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    p->stage_cur ^= 1;
    if (!a.in_off) a.in_off = p->d_in_pref;
    if (!a.out_off) a.out_off = p->d_out_pref;
    a.mode = kModeSorted;
    if (p->persist) {
        int64_t tiles = 0;
        for (int c = 0; c < n; ++c) tiles += (cnt[c] + p->cdev[c].G - 1) / p->cdev[c].G;
        if (e == cudaSuccess) e = launch_persistent(p, a, p->d_sorted, p->d_sched1, a.in_off, a.out_off, tiles, s);
        return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
    }
    // several non-empty classes run concurrently on their own streams (fork/join through
    // events); a single one goes straight onto s (four API calls fewer)
    int busy = 0;
    for (int c = 0; c < n; ++c) busy += cnt[c] > 0;
    if (e == cudaSuccess && busy > 1) e = cudaEventRecord(p->ev_fork, s);
    for (int oi = 0; oi < n && e == cudaSuccess; ++oi) {
        const int c = p->order[oi];
        if (cnt[c] == 0) continue;
        const int64_t grid = (cnt[c] + p->cdev[c].G - 1) / p->cdev[c].G;
        KArgs ac = a;
        ac.c = p->cdev[c];
        ac.cls = c;
        ac.W = p->launch[c].W;
        void* args[] = {&ac};
        cudaStream_t cs = busy > 1 ? p->cstreams[c] : s;
        if (busy > 1) e = cudaStreamWaitEvent(cs, p->ev_fork, 0);
        if (e == cudaSuccess)
            e = cudaLaunchKernel(p->kern[c], dim3((unsigned)grid), dim3(kThreads), args, (size_t)p->csmem[c], cs);
        if (busy > 1 && e == cudaSuccess) e = cudaEventRecord(p->ev_join[c], cs);
        if (busy > 1 && e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join[c], 0);
    }
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

// Launch every non-empty class of one pass from the host, each on its own stream,
// forked from and joined back into s (a pass with one class: on s).
static cudaError_t launch_classes(mci_plan_t p, const KArgs& tmpl, bool cols, const int* counts,
                                  cudaStream_t s)
{
    const int n = (int)p->cls.size();
    int busy = 0;
    for (int c = 0; c < n; ++c) busy += counts[c] > 0;
    cudaError_t e = busy > 1 ? cudaEventRecord(p->ev_fork, s) : cudaSuccess;
    for (int oi = 0; oi < n && e == cudaSuccess; ++oi) {
        const int c = p->order[oi];
        if (counts[c] == 0) continue;
        KArgs ac = tmpl;
        ac.c = p->cdev[c];
        ac.cls = c;
        ac.W = p->launch[c].W;
        void* args[] = {&ac};
        const void* k = cols ? p->kern_cols[c] : p->kern[c];
        cudaStream_t cs = busy > 1 ? p->cstreams[c] : s;   // a single class: straight onto s
        if (busy > 1) e = cudaStreamWaitEvent(cs, p->ev_fork, 0);
        if (e == cudaSuccess)
            e = cudaLaunchKernel(k, dim3((unsigned)counts[c]), dim3(kThreads), args,
                                 (size_t)(cols ? p->csmem_cols[c] : p->csmem[c]), cs);
        if (busy > 1 && e == cudaSuccess) e = cudaEventRecord(p->ev_join[c], cs);
        if (busy > 1 && e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join[c], 0);
    }
    return e;
}

// 2-D batch whose image sizes are in host memory: per-class (image, tile) lists,
// offsets and a device copy of the sizes are built on the host in pinned staging
// (two alternating blocks), uploaded in one copy, then the row pass and the
// column pass are launched per class from the host with exact grids.
static mci_status upsample_2d_host_grouped(mci_plan_t p, KArgs rows, KArgs cols, const int* h,
                                           const int* w, const int* scale, bool pack_lr,
                                           bool pack_hr, int64_t n_img, cudaStream_t s)
{
    const int n = (int)p->cls.size();
    char* blk = p->h_stage2[p->stage2_cur];
    cudaEvent_t ev = p->ev_stage2[p->stage2_cur];
    if (cudaEventSynchronize(ev) != cudaSuccess) return MCI_ERR_CUDA;
    int64_t* inter_off = (int64_t*)blk;
    int64_t* lr_pref = (int64_t*)(blk + p->o2_lrp);
    int64_t* hr_pref = (int64_t*)(blk + p->o2_hrp);
    int2* items = (int2*)(blk + p->o2_it);
    Sched2D* st = (Sched2D*)(blk + p->o2_s2);
    int* hws = (int*)(blk + p->o2_hws);
    const int64_t I = p->desc.max_images;
    auto lookup = [&](int P, int64_t T) {
        for (int c = 0; c < n; ++c)
            if (p->cdev[c].P == P && p->cdev[c].T == T) return c;
        return -1;
    };
    std::vector<int> rc(n_img), cc(n_img), rcnt(n, 0), ccnt(n, 0);
    std::vector<char> by_gemm(n_img, 0);
    GemmJob* jobs = (GemmJob*)(blk + p->o2_jobs);     // row jobs, then column jobs at + I
    int* tile0 = (int*)(blk + p->o2_tile0);            // row prefix, then column prefix at + I + 1
    int n_gemm = 0, row_tiles = 0, col_tiles = 0;
    int64_t inter = 0, lr = 0, hrp = 0;
    for (int64_t i = 0; i < n_img; ++i) {
        const int hi = h[i], wi = w[i], si = scale[i];
        if (hi <= 0 || wi <= 0 || si <= 0) return MCI_ERR_INVALID_ARG;
        rc[i] = lookup(wi, (int64_t)si * wi);
        cc[i] = lookup(hi, (int64_t)si * hi);
        if (rc[i] < 0 || cc[i] < 0) return MCI_ERR_UNSUPPORTED_SIZE;
        if (p->d_kmap[rc[i]] && p->d_kmap[cc[i]]) {
            // both passes on the tensor cores: Y^T = (X K_w^T)^T into the intermediate, HR = K_h Y
            by_gemm[i] = 1;
            GemmJob& r = jobs[n_gemm];
            r.A = (const float*)rows.in + (pack_lr ? lr : 0);
            r.a_off = pack_lr ? nullptr : rows.img_in_off;
            r.B = p->d_kmap[rc[i]];
            r.a_planes = nullptr;
            r.b_planes = p->d_kp[rc[i]];
            r.C = p->d_inter + inter;
            r.c_off = nullptr;
            r.lda = wi;
            r.ldb = wi;
            r.ldc = hi;
            r.M = hi;
            r.N = si * wi;
            r.K = wi;
            r.img = (int)i;
            r.transpose_c = 1;
            GemmJob& q = jobs[I + n_gemm];
            q.A = p->d_kmap[cc[i]];
            q.a_planes = p->d_kp[cc[i]];
            q.b_planes = nullptr;
            q.a_off = nullptr;
            q.B = p->d_inter + inter;
            q.C = (float*)cols.out + (pack_hr ? hrp : 0);
            q.c_off = pack_hr ? nullptr : cols.img_out_off;
            q.lda = hi;
            q.ldb = hi;
            q.ldc = (int64_t)si * wi;
            q.M = si * hi;
            q.N = si * wi;
            q.K = hi;
            q.img = (int)i;
            q.transpose_c = 0;
            tile0[n_gemm] = row_tiles;
            tile0[I + 1 + n_gemm] = col_tiles;
            row_tiles += (r.M / 128) * (r.N / 128);
            col_tiles += (q.M / 128) * (q.N / 128);
            ++n_gemm;
        } else {
            rcnt[rc[i]] += (hi + p->cdev[rc[i]].G - 1) / p->cdev[rc[i]].G;
            ccnt[cc[i]] += (int)(((int64_t)si * wi + p->cdev[cc[i]].Gc - 1) / p->cdev[cc[i]].Gc);
        }
        inter_off[i] = inter;
        lr_pref[i] = lr;
        hr_pref[i] = hrp;
        inter += (int64_t)hi * si * wi;
        lr += (int64_t)hi * wi;
        hrp += (int64_t)si * si * hi * wi;
        hws[i] = hi;
        hws[I + i] = wi;
        hws[2 * I + i] = si;
    }
    if (inter > p->desc.max_intermediate) return MCI_ERR_UNSUPPORTED_SIZE;
    int64_t pos = 0;
    std::vector<int64_t> rcur(n), ccur(n);
    for (int c = 0; c < n; ++c) {
        st->row_start[c] = (int)pos;
        st->row_count[c] = rcnt[c];
        rcur[c] = pos;
        pos += rcnt[c];
    }
    for (int c = 0; c < n; ++c) {
        st->col_start[c] = (int)pos;
        st->col_count[c] = ccnt[c];
        ccur[c] = pos;
        pos += ccnt[c];
    }
    if (pos > p->max_items) return MCI_ERR_UNSUPPORTED_SIZE;
    tile0[n_gemm] = row_tiles;
    tile0[I + 1 + n_gemm] = col_tiles;
    for (int64_t i = 0; i < n_img; ++i) {
        if (by_gemm[i]) continue;
        const int nr = (h[i] + p->cdev[rc[i]].G - 1) / p->cdev[rc[i]].G;
        const int nc = (int)(((int64_t)scale[i] * w[i] + p->cdev[cc[i]].Gc - 1) / p->cdev[cc[i]].Gc);
        for (int t = 0; t < nr; ++t) items[rcur[rc[i]]++] = make_int2((int)i, t);
        for (int t = 0; t < nc; ++t) items[ccur[cc[i]]++] = make_int2((int)i, t);
    }
    // upload the used part in one copy: offsets, schedule, sizes, GEMM jobs and the filled items
    const size_t head = p->o2_it + sizeof(int2) * (size_t)pos;
    cudaError_t e = cudaMemcpyAsync(p->d_inter_off, blk, head, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    p->stage2_cur ^= 1;
    for (KArgs* a : {&rows, &cols}) {
        a->h = p->d_hws;
        a->w = p->d_hws + I;
        a->scale = p->d_hws + 2 * I;
        if (pack_lr) a->img_in_off = p->d_lr_pref;
        if (pack_hr) a->img_out_off = p->d_hr_pref;
    }
    rows.mode = kModeRows;
    cols.mode = kModeCols;
    if (e == cudaSuccess && n_gemm)
        e = (cudaError_t)launch_gemm(p->d_jobs, p->d_tile0, n_gemm, row_tiles, p->d_status, s);
    if (e == cudaSuccess) e = launch_classes(p, rows, false, rcnt.data(), s);
    if (e == cudaSuccess && n_gemm)
        e = (cudaError_t)launch_gemm(p->d_jobs + I, p->d_tile0 + I + 1, n_gemm, col_tiles, p->d_status, s);
    if (e == cudaSuccess) e = launch_classes(p, cols, true, ccnt.data(), s);
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

extern "C" {

const char* mci_error_string(mci_status s)
{
    switch (s) {
    case MCI_OK: return "success";
    case MCI_ERR_INVALID_ARG: return "invalid argument";
    case MCI_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case MCI_ERR_SINGULAR: return "singular system matrix";
    case MCI_ERR_CUDA: return "CUDA runtime error";
    case MCI_ERR_OOM: return "device out of memory";
    case MCI_ERR_TIMEOUT: return "device wait timed out";
    case MCI_ERR_DEVICE: return "device-side check failed";
    }
    return "unknown status";
}

mci_status mci_destroy(mci_plan_t p)
{
    if (!p) return MCI_OK;
    cudaDeviceSynchronize();
    for (cudaStream_t cs : p->cstreams)
        if (cs) cudaStreamDestroy(cs);
    for (cudaEvent_t ev : p->ev_join)
        if (ev) cudaEventDestroy(ev);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    for (int i = 0; i < 2; ++i) {
        if (p->ev_stage[i]) cudaEventDestroy(p->ev_stage[i]);
        if (p->h_stage[i]) cudaFreeHost(p->h_stage[i]);
        if (p->ev_stage2[i]) cudaEventDestroy(p->ev_stage2[i]);
        if (p->h_stage2[i]) cudaFreeHost(p->h_stage2[i]);
    }
    if (p->d_tables) cudaFree(p->d_tables);
    if (p->d_work) cudaFree(p->d_work);
    if (p->d_gemm) cudaFree(p->d_gemm);
    if (p->d_kplanes) cudaFree(p->d_kplanes);
    if (p->d_rtab) cudaFree(p->d_rtab);
    if (p->d_chunk) cudaFree(p->d_chunk);
    for (cudaStream_t hs : p->hs)
        if (hs) cudaStreamDestroy(hs);
    for (int i = 0; i < mci_plan_s::kSlots; ++i) {
        if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
        if (p->ev_comp[i]) cudaEventDestroy(p->ev_comp[i]);
        if (p->ev_free[i]) cudaEventDestroy(p->ev_free[i]);
    }
    delete p;
    return MCI_OK;
}

// Plan-time tile autotuner: for every size class, time the uniform 1-D launch of a
// scratch batch for each candidate tile height G (signals per CTA; the candidates come
// from shared-memory budgets of 16 .. 144 KB per CTA, i.e. 1 .. 12 CTAs per SM) and keep
// the fastest.  The results of a launch do not depend on G.
// Tile heights chosen by the autotuner, process-wide, keyed by the kernel kind, the class
// shape, the precision and the device (name and multiprocessor count); saved to and loaded
// from a JSON object {"key": G, ...} by mci_tune_cache_save / mci_tune_cache_load.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;

static std::string tune_key(const ClassDev& c, int prec, const cudaDeviceProp& prop)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "generic-1d|%s|%s|P=%d|T=%d|Min=%d|Q=%d|%s|sm=%d",
                  prec == MCI_FP64 ? "fp64" : "fp32", c.cplx ? "complex" : "real", c.P, c.T, c.M_in, c.Q,
                  prop.name, prop.multiProcessorCount);
    return buf;
}

static cudaError_t autotune_tiles(mci_plan_s* p, int smem_cap, cudaStream_t s)
{
    const int n = (int)p->cls.size();
    const int csz = (int)(2 * p->elem);
    const size_t scratch_bytes = (size_t)64 << 20;
    void* scratch = nullptr;
    cudaError_t e = dev_malloc((void**)&scratch, scratch_bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(scratch, 0, scratch_bytes, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    cudaDeviceProp prop{};
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
    for (int c = 0; c < n && e == cudaSuccess; ++c) {
        ClassDev cd = p->cdev[c];
        if (cd.fast) continue;   // the fused kernel's tile is fixed by N
        const int per = cd.sstride * csz;
        const std::string key = tune_key(cd, p->desc.precision, prop);
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tune.find(key);
            const int twb0 = smem_twiddle_count(cd.N) * csz;
            if (it != g_tune.end() && it->second >= 1 && it->second <= kMaxTile &&
                it->second * per + twb0 <= smem_cap) {   // tuned before: no timing
                p->cdev[c].G = it->second;
                p->csmem[c] = it->second * per + twb0;
                continue;
            }
        }
        const int twb = smem_twiddle_count(cd.N) * csz;
        const int64_t sig_bytes = (cd.in_len + cd.out_len) * (int64_t)p->elem;
        const int64_t nsig = std::max<int64_t>(1, std::min<int64_t>((int64_t)scratch_bytes / sig_bytes, 8192));
        std::vector<int> cand;
        for (int budget : {16 << 10, 24 << 10, 32 << 10, 48 << 10, 64 << 10, 96 << 10, 144 << 10}) {
            const int G = std::max(1, std::min(kMaxTile, (budget - twb) / per));
            if (G * per + twb <= smem_cap && std::find(cand.begin(), cand.end(), G) == cand.end())
                cand.push_back(G);
        }
        int bestG = cd.G;
        float best = 1e30f;
        for (int G : cand) {
            cd.G = G;
            KArgs a{};
            a.c = cd;
            a.cls = c;
            a.mode = kModeUniform;
            a.W = p->launch[c].W;
            a.in = scratch;
            a.out = (char*)scratch + nsig * cd.in_len * (int64_t)p->elem;
            a.batch = nsig;
            a.status = p->d_status;
            const int64_t items = (nsig + G - 1) / G;
            a.uniform_items = (int)items;
            void* args[] = {&a};
            const size_t smem = (size_t)G * per + twb;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)   // warm-up
                e = cudaLaunchKernel(p->kern[c], dim3((unsigned)items), dim3(kThreads), args, smem, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep)
                e = cudaLaunchKernel(p->kern[c], dim3((unsigned)items), dim3(kThreads), args, smem, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                bestG = G;
            }
        }
        p->cdev[c].G = bestG;
        p->csmem[c] = bestG * per + twb;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = bestG;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaError_t ef = cudaFree(scratch);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) {
        p->smem = 0;
        for (int c = 0; c < n; ++c) {
            if (!p->cdev[c].fast3) {   // columns share the rows' tile
                p->cdev[c].Gc = p->cdev[c].G;
                p->csmem_cols[c] = p->csmem[c];
            }
            p->smem = std::max(p->smem, p->csmem[c]);
            p->launch[c].c = p->cdev[c];
            p->launch[c].smem = p->csmem[c];
            p->launch[c].smem_cols = p->csmem_cols[c];
        }
        e = cudaMemcpyAsync(p->d_launch, p->launch.data(), sizeof(ClassLaunch) * n, cudaMemcpyHostToDevice, s);
    }
    return e;
}

mci_status mci_plan(mci_plan_t* out, const mci_desc* desc, mci_stream_t stream)
{
    if (!out) return MCI_ERR_INVALID_ARG;
    *out = nullptr;
    mci_status st = validate(desc);
    if (st != MCI_OK) return st;
    mci_plan_s* p = new (std::nothrow) mci_plan_s();
    if (!p) return MCI_ERR_OOM;
    p->desc = *desc;
    p->sys.assign(desc->sys, desc->sys + desc->M);
    p->desc.sys = p->sys.data();
    p->desc.P = nullptr;  // host arrays are not kept
    p->desc.T = nullptr;
    p->desc.N1 = nullptr;
    const mci_desc& d = p->desc;
    p->elem = d.precision == MCI_FP64 ? 8 : 4;
    p->M_in = d.channel_mode == MCI_CHANNELS_FD ? 1 : d.M;
    p->n_out = __builtin_popcount(d.out_flags);
    const int n = desc->n_sizes;
    p->cls.resize(n);
    p->cdev.resize(n);
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        delete p;
        return MCI_ERR_CUDA;
    }
    const int smem_cap = (int)prop.sharedMemPerBlockOptin - 2048;  // static shared memory margin
    p->n_sm = prop.multiProcessorCount;
    const int csz = (int)(2 * p->elem);
    int need = 0;
    int Pmax = 0, Tmax = 0;
    for (int c = 0; c < n; ++c) {
        HostClass& hc = p->cls[c];
        hc.P = desc->P[c];
        hc.T = desc->T[c];
        hc.s = hc.T / hc.P;
        hc.N = d.complex_signal ? hc.P : hc.P / 2;   // complex FFT length
        hc.N1 = desc->N1 ? desc->N1[c] : -(int64_t)((int64_t)d.M * hc.P / 2);
        Pmax = std::max(Pmax, hc.P);
        Tmax = std::max(Tmax, hc.T);
        ClassDev& cd_ = p->cdev[c];
        cd_.P = hc.P;
        cd_.N = hc.N;
        cd_.T = hc.T;
        cd_.s = hc.s;
        cd_.M_in = p->M_in;
        cd_.n_out = p->n_out;
        cd_.Q = hc.s * p->n_out;
        cd_.QM = std::max(cd_.M_in, cd_.Q);
        cd_.npad = padded_len(hc.N);
        cd_.sstride = cd_.QM * cd_.npad + (((2 - cd_.QM * cd_.npad) % 16) + 16) % 16;
        cd_.mag_min = fastdiv_magic(cd_.M_in);
        cd_.mag_q = fastdiv_magic(cd_.Q);
        cd_.mag_nout = fastdiv_magic(cd_.n_out);
        cd_.cplx = d.complex_signal;
        cd_.chan_len = hc.P * (d.complex_signal ? 2 : 1);
        cd_.in_len = (int64_t)cd_.M_in * cd_.chan_len;
        cd_.out_len = (int64_t)cd_.n_out * hc.T * (d.complex_signal ? 2 : 1);
        // fused radix-8 kernel: real FP32 1-D classes with N a power of two in its range and a
        // compiled (channels, scale, outputs) variant; its tile and shared memory are fixed
        // image plans: rows and columns both on the fused path (one tile height for both
        // passes), N up to kFastMaxImageN, where a column variant is compiled
        int var = -1;
        const bool img = d.max_images > 0;
        cd_.fast = d.precision == MCI_FP32 && !d.complex_signal && hc.N >= kFastMinN &&
                           hc.N <= (img ? kFastMaxImageN : kFastMaxN) && (hc.N & (hc.N - 1)) == 0 &&
                           fast_kernel_lookup(hc.N, cd_.M_in, hc.s, p->n_out, &var) != nullptr &&
                           (!img || fast_cols_kernel_lookup(hc.N, cd_.M_in, hc.s, p->n_out) != nullptr)
                       ? 1 + var
                       : 0;
        // image columns of a class with N = 3 N' (N' a power of two): the fused factor-3 column
        // kernel (its own tile of 2048 / N' columns); the rows stay on the generic kernel
        cd_.fast3 = !cd_.fast && img && d.precision == MCI_FP32 && !d.complex_signal &&
                    fast3_cols_kernel_lookup(hc.N, cd_.M_in, hc.s, p->n_out) != nullptr;
        if (cd_.fast) continue;
        const int per = cd_.sstride * csz + smem_twiddle_count(hc.N) * csz;
        if (per > smem_cap) {
            delete p;
            return MCI_ERR_UNSUPPORTED_SIZE;
        }
        need = std::max(need, per);
    }
    const int budget = std::max(need, std::min(kSmemBudget, smem_cap));
    p->csmem.resize(n);
    p->csmem_cols.resize(n);
    for (int c = 0; c < n; ++c) {
        ClassDev& cd_ = p->cdev[c];
        if (cd_.fast) {   // 2048 / N signals of QM buffers of N complex values
            cd_.G = cd_.Gc = 2048 / cd_.N;
            p->csmem[c] = p->csmem_cols[c] = cd_.G * cd_.QM * cd_.N * csz;
            p->smem = std::max(p->smem, p->csmem[c]);
            continue;
        }
        const int per = cd_.sstride * csz;
        const int twb = smem_twiddle_count(cd_.N) * csz;   // FFT twiddles after the buffers
        cd_.G = std::max(1, std::min(kMaxTile, (budget - twb) / per));
        p->csmem[c] = cd_.G * per + twb;
        if (p->csmem[c] > smem_cap) {
            delete p;
            return MCI_ERR_UNSUPPORTED_SIZE;
        }
        p->smem = std::max(p->smem, p->csmem[c]);
        cd_.Gc = cd_.G;
        p->csmem_cols[c] = p->csmem[c];
        if (cd_.fast3) {   // 2048 / N' columns of N complex values
            cd_.Gc = 2048 / (cd_.N / 3);
            p->csmem_cols[c] = cd_.Gc * cd_.N * csz;
            p->smem = std::max(p->smem, p->csmem_cols[c]);
        }
    }
    p->order.resize(n);
    for (int c = 0; c < n; ++c) p->order[c] = c;
    std::stable_sort(p->order.begin(), p->order.end(),
                     [&](int a, int b) { return p->cls[a].P > p->cls[b].P; });

    // FP64 tables
    p->gemm_off.assign(n, -1);
    p->rtab_off.assign(n, 0);
    p->omega_sum.assign(n, 0.0);
    std::vector<float> W32;
    std::vector<double> W64;
    st = d.precision == MCI_FP64 ? build_tables<double>(p, W64) : build_tables<float>(p, W32);
    if (st != MCI_OK) {
        delete p;
        return st;
    }
    const void* W_src = d.precision == MCI_FP64 ? (const void*)W64.data() : (const void*)W32.data();
    const size_t W_bytes = (d.precision == MCI_FP64 ? W64.size() : W32.size()) * p->elem;
    const size_t launch_bytes = align_up(sizeof(ClassLaunch) * n, 256);
    const size_t order_bytes = align_up(sizeof(int) * n, 256);
    const size_t total = launch_bytes + order_bytes + align_up(W_bytes, 256);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = dev_malloc((void**)&p->d_tables, total);
    if (e != cudaSuccess) {
        delete p;
        return cuda_status(e);
    }
    p->table_bytes = (int64_t)total;
    char* base = (char*)p->d_tables;
    p->d_launch = (ClassLaunch*)base;
    p->d_order = (int*)(base + launch_bytes);
    p->d_W = base + launch_bytes + order_bytes;
    p->launch.resize(n);
    p->kern.resize(n);
    p->kern_cols.resize(n);
    for (int c = 0; c < n; ++c) {
        ClassLaunch& L = p->launch[c];
        L.c = p->cdev[c];
        L.W = (const char*)p->d_W + p->cdev[c].w_off * 2 * p->elem;
        L.prec = d.precision;
        L.smem = p->csmem[c];
        L.smem_cols = p->csmem_cols[c];
        p->kern[c] = p->cdev[c].fast ? fast_kernel_lookup(p->cdev[c].N, p->cdev[c].M_in, p->cdev[c].s, p->n_out)
                                     : kernel_lookup(d.precision, false, p->cdev[c].N);
        p->kern_cols[c] = d.precision != MCI_FP32 ? nullptr
                          : p->cdev[c].fast ? fast_cols_kernel_lookup(p->cdev[c].N, p->cdev[c].M_in, p->cdev[c].s, p->n_out)
                          : p->cdev[c].fast3 ? fast3_cols_kernel_lookup(p->cdev[c].N, p->cdev[c].M_in, p->cdev[c].s, p->n_out)
                                             : kernel_lookup(d.precision, true, p->cdev[c].N);
        if (p->cdev[c].fast && d.max_images > 0 && !p->kern_cols[c]) e = cudaErrorInvalidDeviceFunction;
        if (!p->kern[c]) e = cudaErrorInvalidDeviceFunction;
        // The dynamic shared-memory limit is an attribute of the kernel function, which
        // size classes of one FFT length (in this plan or another) share: it is set to
        // the device maximum once; each launch states what it uses.  Largest carveout.
        for (const void* k : {p->kern[c], p->kern_cols[c]}) {
            if (!k || e != cudaSuccess) continue;
            cudaFuncAttributes fa{};
            e = cudaFuncGetAttributes(&fa, k);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)prop.sharedMemPerBlockOptin - (int)fa.sharedSizeBytes);
            // the fused kernel runs two CTAs per SM (registers): shared memory for exactly
            // those, the rest of the SM's storage to L1 (the bin weights and twiddles are read
            // through it; measured 10% faster than the largest carveout); others: largest
            int carve = cudaSharedmemCarveoutMaxShared;
            if (p->cdev[c].fast || (p->cdev[c].fast3 && k == p->kern_cols[c])) {
                const int need = 2 * ((k == p->kern_cols[c] ? p->csmem_cols[c] : p->csmem[c]) + (int)fa.sharedSizeBytes + 1024);
                carve = std::min(100, (100 * need + (int)prop.sharedMemPerMultiprocessor - 1) /
                                          (int)prop.sharedMemPerMultiprocessor);
            }
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
        }
    }
    // uneven batches whose classes are all on the fused path: one persistent launch
    p->persist = n > 1 && fast_persistent_kernel() != nullptr;
    for (int c = 0; c < n; ++c) {
        p->persist = p->persist && p->cdev[c].fast >= 1 && p->cdev[c].fast <= kFastPersistentVariants;
        p->persist_smem = std::max(p->persist_smem, p->csmem[c]);
    }
    if (e == cudaSuccess && p->persist) {
        const void* k = fast_persistent_kernel();
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, k);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, p->persist_smem);
        const int need = 2 * (p->persist_smem + (int)fa.sharedSizeBytes + 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     std::min(100, (100 * need + (int)prop.sharedMemPerMultiprocessor - 1) /
                                                       (int)prop.sharedMemPerMultiprocessor));
        int per_sm = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, kThreads, p->persist_smem);
        p->persist_ctas = per_sm * prop.multiProcessorCount;
        if (e == cudaSuccess && p->persist_ctas <= 0) p->persist = 0;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_launch, p->launch.data(), sizeof(ClassLaunch) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_order, p->order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_W, W_src, W_bytes, cudaMemcpyHostToDevice, s);
    p->d_kmap.assign(n, nullptr);
    if (e == cudaSuccess && !p->gemm_tab.empty()) {
        e = dev_malloc((void**)&p->d_gemm, sizeof(float) * p->gemm_tab.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_gemm, p->gemm_tab.data(), sizeof(float) * p->gemm_tab.size(),
                                cudaMemcpyHostToDevice, s);
        for (int c = 0; c < n; ++c)
            if (p->gemm_off[c] >= 0) p->d_kmap[c] = (const float*)p->d_gemm + p->gemm_off[c];
        if (e == cudaSuccess) e = (cudaError_t)prepare_gemm();
        p->table_bytes += (int64_t)(sizeof(float) * p->gemm_tab.size());
        // the constant operand of both GEMM passes, split once into the kernel's plane tiles
        int64_t kp_bytes = 0;
        std::vector<int64_t> kp_off(n, -1);
        for (int c = 0; c < n; ++c)
            if (p->gemm_off[c] >= 0) {
                kp_off[c] = kp_bytes;
                kp_bytes += gemm_plane_bytes(p->cls[c].T, p->cls[c].P);
            }
        if (e == cudaSuccess) e = dev_malloc(&p->d_kplanes, (size_t)kp_bytes);
        p->d_kp.assign(n, nullptr);
        for (int c = 0; c < n && e == cudaSuccess; ++c)
            if (kp_off[c] >= 0) {
                p->d_kp[c] = (const char*)p->d_kplanes + kp_off[c];
                e = (cudaError_t)presplit_gemm(p->d_kmap[c], p->cls[c].T, p->cls[c].P,
                                               (char*)p->d_kplanes + kp_off[c], s);
            }
        p->table_bytes += kp_bytes;
    }

    if (e == cudaSuccess && !p->rtab.empty()) {
        e = dev_malloc((void**)&p->d_rtab, sizeof(double) * p->rtab.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_rtab, p->rtab.data(), sizeof(double) * p->rtab.size(), cudaMemcpyHostToDevice,
                                s);
        p->table_bytes += (int64_t)(sizeof(double) * p->rtab.size());
    }

    // workspace
    const int64_t B = d.max_batch, I = d.max_images, X = d.max_intermediate;
    p->max_items = I * (int64_t)(Pmax + Tmax);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_status = carve(sizeof(int) * 4);
    const size_t o_sorted = carve(sizeof(int64_t) * B);
    const size_t o_inp = carve(sizeof(int64_t) * B);
    const size_t o_outp = carve(sizeof(int64_t) * B);
    const size_t o_s1 = carve(sizeof(Sched1D));
    size_t o_inter = 0, o_ioff = 0, o_lrp = 0, o_hrp = 0, o_rc = 0, o_cc = 0, o_it = 0, o_s2 = 0,
           o_hws = 0, o_jobs = 0, o_tile0 = 0;
    if (I > 0) {
        o_inter = carve(sizeof(float) * (size_t)X);
        o_ioff = carve(sizeof(int64_t) * I);
        o_lrp = carve(sizeof(int64_t) * I);
        o_hrp = carve(sizeof(int64_t) * I);
        // the host-grouped path uploads [o_ioff, o_it + used items) in one copy
        o_s2 = carve(sizeof(Sched2D));
        o_hws = carve(sizeof(int) * 3 * I);
        o_jobs = carve(sizeof(GemmJob) * 2 * I);
        o_tile0 = carve(sizeof(int) * 2 * (I + 1));
        o_rc = carve(sizeof(int) * I);
        o_cc = carve(sizeof(int) * I);
        o_it = carve(sizeof(int2) * (size_t)p->max_items);
    }
    if (e == cudaSuccess) e = dev_malloc((void**)&p->d_work, off);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        mci_destroy(p);
        return cuda_status(e);
    }
    p->work_bytes = (int64_t)off;
    // a plan that always stages host buffers (host_access 1) gets its chunk buffers now: a
    // chunk holds at most max(kChunkIn, one signal) bytes of input, so at most that times the
    // largest output/input ratio of the classes of output
    if (e == cudaSuccess && d.host_access == 1 && B > 0) {
        int64_t max_li = 0;
        double ratio = 0.0;
        for (const ClassDev& c : p->cdev) {
            max_li = std::max(max_li, c.in_len * (int64_t)p->elem);
            ratio = std::max(ratio, (double)c.out_len / (double)c.in_len);
        }
        const int64_t bin = std::max(kChunkIn, max_li);
        const size_t need_in = align_up((size_t)bin, 256);
        const size_t need_out = align_up((size_t)std::ceil((double)bin * ratio), 256);
        e = dev_malloc((void**)&p->d_chunk, mci_plan_s::kSlots * (need_in + need_out));
        if (e != cudaSuccess) {
            cudaStreamSynchronize(s);
            mci_destroy(p);
            return cuda_status(e);
        }
        p->chunk_in_bytes = need_in;
        p->chunk_out_bytes = need_out;
        p->work_bytes += (int64_t)(mci_plan_s::kSlots * (need_in + need_out));
    }
    char* w = (char*)p->d_work;
    p->d_status = (int*)(w + o_status);
    p->d_sorted = (int64_t*)(w + o_sorted);
    p->d_in_pref = (int64_t*)(w + o_inp);
    p->d_out_pref = (int64_t*)(w + o_outp);
    p->d_sched1 = (Sched1D*)(w + o_s1);
    if (I > 0) {
        p->d_inter = (float*)(w + o_inter);
        p->d_inter_off = (int64_t*)(w + o_ioff);
        p->d_lr_pref = (int64_t*)(w + o_lrp);
        p->d_hr_pref = (int64_t*)(w + o_hrp);
        p->d_row_cls = (int*)(w + o_rc);
        p->d_col_cls = (int*)(w + o_cc);
        p->d_items = (int2*)(w + o_it);
        p->d_sched2 = (Sched2D*)(w + o_s2);
        p->d_hws = (int*)(w + o_hws);
        p->d_jobs = (GemmJob*)(w + o_jobs);
        p->d_tile0 = (int*)(w + o_tile0);
    }
    // host-grouped path: one stream per class, fork/join events, two pinned staging blocks
    p->stage_bytes = o_s1 + sizeof(Sched1D) - o_sorted;
    p->off_in_pref = o_inp - o_sorted;
    p->off_out_pref = o_outp - o_sorted;
    p->off_sched1 = o_s1 - o_sorted;
    if (n > 1 && e == cudaSuccess) {
        p->cstreams.assign(n, nullptr);
        p->ev_join.assign(n, nullptr);
        for (int c = 0; c < n && e == cudaSuccess; ++c) {
            e = cudaStreamCreateWithFlags(&p->cstreams[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[c], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = pinned_alloc((void**)&p->h_stage[i], p->stage_bytes);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_stage[i], cudaEventDisableTiming);
        }
    }
    if (I > 0 && e == cudaSuccess) {
        p->stage2_bytes = o_it + sizeof(int2) * (size_t)p->max_items - o_ioff;
        p->o2_jobs = o_jobs - o_ioff;
        p->o2_tile0 = o_tile0 - o_ioff;
        p->o2_lrp = o_lrp - o_ioff;
        p->o2_hrp = o_hrp - o_ioff;
        p->o2_it = o_it - o_ioff;
        p->o2_s2 = o_s2 - o_ioff;
        p->o2_hws = o_hws - o_ioff;
        if (p->cstreams.empty()) {
            p->cstreams.assign(n, nullptr);
            p->ev_join.assign(n, nullptr);
            for (int c = 0; c < n && e == cudaSuccess; ++c) {
                e = cudaStreamCreateWithFlags(&p->cstreams[c], cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[c], cudaEventDisableTiming);
            }
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        }
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = pinned_alloc((void**)&p->h_stage2[i], p->stage2_bytes);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_stage2[i], cudaEventDisableTiming);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int) * 4, s);
    if (e == cudaSuccess && d.autotune) e = autotune_tiles(p, smem_cap, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int) * 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        mci_destroy(p);
        return cuda_status(e);
    }
    p->last_stream = s;
    *out = p;
    return MCI_OK;
}

mci_status mci_interp_1d(mci_plan_t p, const void* in, const int64_t* in_off, void* out,
                         const int64_t* out_off, const int* size_class, int64_t batch,
                         mci_stream_t stream)
{
    if (!p || batch < 0 || batch > p->desc.max_batch) return MCI_ERR_INVALID_ARG;
    if (batch == 0) return MCI_OK;
    if (!in || !out) return MCI_ERR_INVALID_ARG;
    const int n = (int)p->cls.size();
    if (n > 1 && !size_class) return MCI_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    KArgs a{};
    a.in = in;
    a.out = out;
    a.in_off = in_off;
    a.out_off = out_off;
    a.batch = batch;
    a.sorted = p->d_sorted;
    a.sched1 = p->d_sched1;
    a.status = p->d_status;
    cudaError_t e;
    if (n == 1) {
        // uniform batch: launched from the host, one CTA per tile
        a.c = p->cdev[0];
        a.cls = 0;
        a.mode = kModeUniform;
        a.W = p->launch[0].W;
        const int64_t items = (batch + p->cdev[0].G - 1) / p->cdev[0].G;
        if (items > 0x7fffffff) return MCI_ERR_UNSUPPORTED_SIZE;
        a.uniform_items = (int)items;
        // few tiles with many output phases (e.g. one short signal evaluated on a long grid):
        // spread each tile's phases over several CTAs (at least 8 phases each)
        const ClassDev& c0 = p->cdev[0];
        int qch = 1;
        if (!c0.fast && !c0.cplx && c0.Q >= 16 && items < p->n_sm)
            qch = (int)std::max<int64_t>(1, std::min<int64_t>(c0.Q / 8, 2 * p->n_sm / items));
        a.qchunks = qch;
        void* args[] = {&a};
        e = cudaLaunchKernel(p->kern[0], dim3((unsigned)items, (unsigned)qch), dim3(kThreads), args,
                             (size_t)p->csmem[0], s);
    } else {
        cudaPointerAttributes attr{};
        if (cudaPointerGetAttributes(&attr, size_class) != cudaSuccess) {
            cudaGetLastError();  // clear the sticky-free error of an unknown pointer
            attr.type = cudaMemoryTypeUnregistered;
        }
        const bool on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
        if (!on_device) return interp_1d_host_grouped(p, a, size_class, batch, s);
        e = (cudaError_t)launch_sched_1d(size_class, batch, n, p->d_launch, p->d_order, p->d_sorted,
                                         p->d_sched1, in_off ? nullptr : p->d_in_pref,
                                         out_off ? nullptr : p->d_out_pref, a, s, p->persist);
        if (e == cudaSuccess && p->persist)
            e = launch_persistent(p, a, p->d_sorted, p->d_sched1, in_off ? in_off : p->d_in_pref,
                                  out_off ? out_off : p->d_out_pref, -1, s);
    }
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_upsample_2d(mci_plan_t p, const float* lr, const int64_t* lr_off, const int* h,
                           const int* w, const int* scale, float* hr, const int64_t* hr_off,
                           int64_t n_img, mci_stream_t stream)
{
    if (!p || n_img < 0) return MCI_ERR_INVALID_ARG;
    if (p->desc.max_images <= 0 || n_img > p->desc.max_images) return MCI_ERR_INVALID_ARG;
    if (n_img == 0) return MCI_OK;
    if (!lr || !hr || !h || !w || !scale) return MCI_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    KArgs rows{};
    rows.in = lr;
    rows.out = p->d_inter;
    rows.items = p->d_items;
    rows.sched2 = p->d_sched2;
    rows.h = h;
    rows.w = w;
    rows.scale = scale;
    rows.img_in_off = lr_off ? lr_off : p->d_lr_pref;
    rows.img_out_off = hr_off ? hr_off : p->d_hr_pref;
    rows.inter_off = p->d_inter_off;
    rows.status = p->d_status;
    KArgs cols = rows;
    cols.in = p->d_inter;
    cols.out = hr;
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, h) != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return upsample_2d_host_grouped(p, rows, cols, h, w, scale, !lr_off, !hr_off, n_img, s);
    // Device grouping.  Each class's tile count is known only on the device, but bounded by
    // the plan: rows: n_img ceil(P_max / G) and max_intermediate / (P G) + n_img; columns:
    // n_img ceil(T_max / Gc) and max_intermediate / (P Gc) + n_img.  When the bounds add up
    // to few CTAs, every class is launched from the host with its bound as the grid (the
    // CTAs beyond the count leave at once): no launches from the device, whose latency
    // dominates small batches.  Otherwise the scheduler launches the classes itself.
    const int n = (int)p->cls.size();
    int Pmax = 0, Tmax = 0;
    for (const HostClass& hc : p->cls) {
        Pmax = std::max(Pmax, hc.P);
        Tmax = std::max(Tmax, hc.T);
    }
    const int64_t X = p->desc.max_intermediate;
    std::vector<int64_t> brow(n), bcol(n);
    int64_t total = 0;
    for (int c = 0; c < n; ++c) {
        const ClassDev& cd = p->cdev[c];
        brow[c] = std::min<int64_t>(n_img * ((Pmax + cd.G - 1) / cd.G), X / ((int64_t)cd.P * cd.G) + n_img);
        bcol[c] = std::min<int64_t>(n_img * ((Tmax + cd.Gc - 1) / cd.Gc), X / ((int64_t)cd.P * cd.Gc) + n_img);
        total += brow[c] + bcol[c];
    }
    const bool host_launch = total <= kBoundedCtas;
    int e = launch_sched_2d(n_img, n, p->d_launch, X, p->max_items, p->d_inter_off,
                            lr_off ? nullptr : p->d_lr_pref, hr_off ? nullptr : p->d_hr_pref, p->d_row_cls,
                            p->d_col_cls, p->d_items, p->d_sched2, rows, cols, s, host_launch ? 0 : 1);
    for (int pass = 0; pass < 2 && host_launch && e == 0; ++pass) {
        const bool cpass = pass == 1;
        for (int c = 0; c < n && e == 0; ++c) {
            const int64_t grid = cpass ? bcol[c] : brow[c];
            const void* k = cpass ? p->kern_cols[c] : p->kern[c];
            if (grid <= 0 || !k) continue;
            KArgs ac = cpass ? cols : rows;
            ac.c = p->cdev[c];
            ac.cls = c;
            ac.W = p->launch[c].W;
            ac.mode = cpass ? kModeCols : kModeRows;
            void* args[] = {&ac};
            e = (int)cudaLaunchKernel(k, dim3((unsigned)grid), dim3(kThreads), args,
                                      (size_t)(cpass ? p->csmem_cols[c] : p->csmem[c]), s);
        }
    }
    return e ? MCI_ERR_CUDA : MCI_OK;
}

mci_status mci_averaged_error(mci_plan_t p, int size_class, const double* coeffs, int64_t n_max,
                              int64_t batch, double* eps, double* bound, mci_stream_t stream)
{
    if (!p || batch < 0) return MCI_ERR_INVALID_ARG;
    if (batch == 0) return MCI_OK;
    if (!coeffs || !eps || size_class < 0 || size_class >= (int)p->cls.size()) return MCI_ERR_INVALID_ARG;
    const mci_desc& d = p->desc;
    if (d.channel_mode != MCI_CHANNELS_MEASURED) return MCI_ERR_INVALID_ARG;
    for (int m = 0; m < d.M; ++m)
        if (d.sys[m].kind == MCI_SYS_CUSTOM) return MCI_ERR_INVALID_ARG;   // b(n) known only in the band
    if (d.blur_taps > 0) return MCI_ERR_INVALID_ARG;   // the error kernel has no blur factor
    const HostClass& hc = p->cls[size_class];
    const int64_t mu = (int64_t)d.M * hc.P;
    if (n_max < std::max<int64_t>(-hc.N1, hc.N1 + mu - 1)) return MCI_ERR_INVALID_ARG;   // band inside
    if (batch > 0x7fffffff || n_max >= (1 << 29) || mu >= (1 << 29) || hc.N1 <= -(1 << 29))
        return MCI_ERR_UNSUPPORTED_SIZE;
    ErrArgs a{};
    a.G = reinterpret_cast<const double2*>(p->d_rtab) + p->rtab_off[size_class];
    a.coeffs = reinterpret_cast<const double2*>(coeffs);
    a.eps = eps;
    a.bound = bound;
    a.N1 = hc.N1;
    a.mu = mu;
    a.n_max = n_max;
    a.batch = batch;
    a.M = d.M;
    a.P = hc.P;
    for (int m = 0; m < d.M; ++m) {
        a.kind[m] = d.sys[m].kind;
        a.order[m] = d.sys[m].order;
        a.tau[m] = d.sys[m].tau;
    }
    a.omega_sum = p->omega_sum[size_class];
    return launch_averaged_error(a, stream) == 0 ? MCI_OK : MCI_ERR_CUDA;
}

mci_status mci_plan_info(mci_plan_t p, mci_plan_stats* st)
{
    if (!p || !st) return MCI_ERR_INVALID_ARG;
    std::memset(st, 0, sizeof(*st));
    st->n_singular = p->n_singular;
    st->max_cond = p->max_cond;
    for (size_t c = 0; c < p->cdev.size(); ++c) st->signals_per_cta[c] = p->cdev[c].G;
    st->threads_per_cta = kThreads;
    st->smem_bytes = p->smem;
    st->table_bytes = p->table_bytes;
    st->workspace_bytes = p->work_bytes;
    for (size_t c = 0; c < p->cdev.size(); ++c)
        if (p->cdev[c].fast) st->fused_mask |= 1u << c;
    for (size_t c = 0; c < p->cdev.size(); ++c)
        if (p->cdev[c].fast3) st->fused3_mask |= 1u << c;
    st->host_route = p->host_trial < 3 ? 0 : (p->host_zero_copy ? 1 : 2);
    st->persistent_ctas = p->persist ? p->persist_ctas : 0;
    cudaError_t e = cudaStreamSynchronize(p->last_stream);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
    st->device_status = status;
    return cuda_status(e);
}

// Host buffers: packed signals are cut into chunks of consecutive signals (about 16 MB of
// input each); chunk c uses slot c mod 3 of device buffers and moves through three streams:
// copy in -> compute (mci_interp_1d, size classes grouped on the host) -> copy out, so the
// two copy directions and the compute of neighbouring chunks overlap.
// The staged host-buffer route: chunks of consecutive signals through the copy-in, compute
// and copy-out streams.
static mci_status interp_1d_host_staged(mci_plan_t p, const void* in, void* out, const int* size_class,
                                        int64_t batch, mci_stream_t stream)
{
    const int n = (int)p->cls.size();
    auto in_len = [&](int64_t b) { return p->cdev[n > 1 ? size_class[b] : 0].in_len; };
    auto out_len = [&](int64_t b) { return p->cdev[n > 1 ? size_class[b] : 0].out_len; };
    // chunks: consecutive signals up to kChunkIn bytes of input
    std::vector<int64_t> first{0};
    std::vector<int64_t> ioff{0}, ooff{0};
    int64_t cin = 0, cout = 0, max_in = 0, max_out = 0;
    for (int64_t b = 0; b < batch; ++b) {
        const int64_t li = in_len(b) * (int64_t)p->elem, lo = out_len(b) * (int64_t)p->elem;
        if (cin > 0 && cin + li > kChunkIn) {
            first.push_back(b);
            ioff.push_back(ioff.back() + cin);
            ooff.push_back(ooff.back() + cout);
            cin = cout = 0;
        }
        cin += li;
        cout += lo;
        max_in = std::max(max_in, cin);
        max_out = std::max(max_out, cout);
    }
    first.push_back(batch);
    ioff.push_back(ioff.back() + cin);
    ooff.push_back(ooff.back() + cout);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!p->hs[0]) {
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&p->hs[i], cudaStreamNonBlocking);
        for (int i = 0; i < mci_plan_s::kSlots && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_comp[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_free[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(p->ev_free[i], p->hs[2]);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    const size_t need_in = align_up((size_t)max_in, 256), need_out = align_up((size_t)max_out, 256);
    if (need_in > p->chunk_in_bytes || need_out > p->chunk_out_bytes) {
        e = cudaDeviceSynchronize();
        if (e == cudaSuccess && p->d_chunk) e = cudaFree(p->d_chunk);
        p->d_chunk = nullptr;
        if (e == cudaSuccess) e = dev_malloc((void**)&p->d_chunk, mci_plan_s::kSlots * (need_in + need_out));
        if (e != cudaSuccess) {
            p->chunk_in_bytes = p->chunk_out_bytes = 0;
            return cuda_status(e);
        }
        p->chunk_in_bytes = need_in;
        p->chunk_out_bytes = need_out;
    }
    cudaStream_t s_in = p->hs[0], s_cmp = p->hs[1], s_out = p->hs[2];
    // the pipeline starts after the caller's prior work on its stream
    cudaEvent_t ev0 = p->ev_comp[0];
    if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev0, 0);
    const int nch = (int)first.size() - 1;
    for (int c = 0; c < nch && e == cudaSuccess; ++c) {
        const int slot = c % mci_plan_s::kSlots;
        char* din = (char*)p->d_chunk + (size_t)slot * (p->chunk_in_bytes + p->chunk_out_bytes);
        char* dout = din + p->chunk_in_bytes;
        const int64_t b0 = first[c], nb = first[c + 1] - first[c];
        e = cudaStreamWaitEvent(s_in, p->ev_free[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(din, (const char*)in + ioff[c], (size_t)(ioff[c + 1] - ioff[c]),
                                cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[slot], s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_cmp, p->ev_in[slot], 0);
        if (e == cudaSuccess) {
            const mci_status st = mci_interp_1d(p, din, nullptr, dout, nullptr, n > 1 ? size_class + b0 : nullptr,
                                                nb, s_cmp);
            if (st != MCI_OK) return st;
        }
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_comp[slot], s_cmp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, p->ev_comp[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)out + ooff[c], dout, (size_t)(ooff[c + 1] - ooff[c]), cudaMemcpyDeviceToHost,
                                s_out);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_free[slot], s_out);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_out);
    p->last_stream = s;
    return cuda_status(e);
}

mci_status mci_interp_1d_host(mci_plan_t p, const void* in, void* out, const int* size_class, int64_t batch,
                              mci_stream_t stream)
{
    if (!p || batch < 0 || batch > p->desc.max_batch) return MCI_ERR_INVALID_ARG;
    if (batch == 0) return MCI_OK;
    const int n = (int)p->cls.size();
    if (!in || !out || (n > 1 && !size_class)) return MCI_ERR_INVALID_ARG;
    for (int64_t b = 0; b < batch && n > 1; ++b)
        if (size_class[b] < 0 || size_class[b] >= n) return MCI_ERR_INVALID_ARG;
    if (p->desc.host_access == 0) {
        // page-locked, device-mapped buffers on both sides: the kernels can read and write them
        // in place over the host link (the runtime's device addresses of the two buffers).
        // Which of that and the staged route is faster depends on the machine (where the pages
        // sit relative to the GPU): the first calls time both, per byte, and the plan keeps
        // the faster
        cudaPointerAttributes ai{}, ao{};
        const bool qi = cudaPointerGetAttributes(&ai, in) == cudaSuccess;
        const bool qo = qi && cudaPointerGetAttributes(&ao, out) == cudaSuccess;
        if (!qo) cudaGetLastError();
        if (qo && ai.type == cudaMemoryTypeHost && ao.type == cudaMemoryTypeHost && ai.devicePointer &&
            ao.devicePointer) {
            double bytes = 0.0;
            for (int64_t b = 0; b < batch; ++b) {
                const ClassDev& c = p->cdev[n > 1 ? size_class[b] : 0];
                bytes += (double)(c.in_len + c.out_len) * p->elem;
            }
            const int trial = p->host_trial;
            const auto t0 = std::chrono::steady_clock::now();
            mci_status st;
            if (trial == 3 ? p->host_zero_copy : trial == 0) {
                st = mci_interp_1d(p, ai.devicePointer, nullptr, ao.devicePointer, nullptr, size_class, batch, stream);
                if (st == MCI_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) st = MCI_ERR_CUDA;
            } else {
                st = interp_1d_host_staged(p, in, out, size_class, batch, stream);
            }
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (st == MCI_OK && trial < 3) {
                if (trial == 0) p->host_rate[0] = bytes / dt;
                if (trial == 2) {
                    p->host_rate[1] = bytes / dt;
                    p->host_zero_copy = p->host_rate[0] >= p->host_rate[1];
                }
                p->host_trial = trial + 1;
            }
            return st;
        }
    }
    return interp_1d_host_staged(p, in, out, size_class, batch, stream);
}

mci_status mci_interp_1d_noalloc(mci_plan_t p, const void* in, const int64_t* in_off, void* out,
                                 const int64_t* out_off, const int* size_class, int64_t batch,
                                 mci_stream_t stream)
{
    if (!p || batch < 0) return MCI_ERR_INVALID_ARG;
    if (batch > MCI_NOALLOC_MAX_BATCH) return MCI_ERR_UNSUPPORTED_SIZE;
    if (batch == 0) return MCI_OK;
    if (!in || !out) return MCI_ERR_INVALID_ARG;
    const int n = (int)p->cls.size();
    if (n > 1) {
        // the grouping kernel reads size_class on the device: a host array is refused
        // (host-side grouping would need the plan's staging blocks, sized by max_batch)
        if (!size_class) return MCI_ERR_INVALID_ARG;
        cudaPointerAttributes attr{};
        if (cudaPointerGetAttributes(&attr, size_class) != cudaSuccess) {
            cudaGetLastError();  // clear the error of an unknown pointer
            return MCI_ERR_INVALID_ARG;
        }
        if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
            return MCI_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSuccess;
    NoAllocScratch* scratch = noalloc_scratch(&e);
    if (!scratch) return MCI_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    KArgs a{};
    a.in = in;
    a.out = out;
    a.in_off = in_off;
    a.out_off = out_off;
    a.batch = batch;
    a.sorted = noalloc_sorted(scratch);
    a.sched1 = noalloc_sched(scratch);
    a.status = p->d_status;
    if (n == 1) {
        a.c = p->cdev[0];
        a.cls = 0;
        a.mode = kModeUniform;
        a.W = p->launch[0].W;
        const int64_t items = (batch + p->cdev[0].G - 1) / p->cdev[0].G;
        a.uniform_items = (int)items;
        void* args[] = {&a};
        e = cudaLaunchKernel(p->kern[0], dim3((unsigned)items), dim3(kThreads), args,
                             (size_t)p->csmem[0], s);
    } else {
        e = (cudaError_t)launch_sched_1d(size_class, batch, n, p->d_launch, p->d_order,
                                         noalloc_sorted(scratch), noalloc_sched(scratch),
                                         in_off ? nullptr : noalloc_in_pref(scratch),
                                         out_off ? nullptr : noalloc_out_pref(scratch), a, s, p->persist);
        if (e == cudaSuccess && p->persist)
            e = launch_persistent(p, a, noalloc_sorted(scratch), noalloc_sched(scratch),
                                  in_off ? in_off : noalloc_in_pref(scratch),
                                  out_off ? out_off : noalloc_out_pref(scratch), -1, s);
    }
    return e == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

}  // extern "C"

void mci_debug_fail_allocation(int after) { g_fail_after.store(after < 0 ? -1 : after); }

mci_status mci_tune_cache_save(const char* path)
{
    if (!path) return MCI_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "w");
    if (!f) return MCI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::fprintf(f, "{");
    bool first = true;
    for (const auto& kv : g_tune) {
        std::fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
        first = false;
    }
    std::fprintf(f, "%s}\n", first ? "" : "\n");
    return std::fclose(f) == 0 ? MCI_OK : MCI_ERR_INVALID_ARG;
}

mci_status mci_tune_cache_load(const char* path)
{
    if (!path) return MCI_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "r");
    if (!f) return MCI_ERR_INVALID_ARG;
    std::string txt;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, k);
    std::fclose(f);
    // a flat JSON object of string keys (no escapes) and integer values
    std::map<std::string, int> got;
    size_t i = txt.find('{');
    if (i == std::string::npos) return MCI_ERR_INVALID_ARG;
    ++i;
    for (;;) {
        while (i < txt.size() && (txt[i] == ' ' || txt[i] == '\n' || txt[i] == '\r' || txt[i] == '\t' || txt[i] == ','))
            ++i;
        if (i >= txt.size()) return MCI_ERR_INVALID_ARG;
        if (txt[i] == '}') break;
        if (txt[i] != '"') return MCI_ERR_INVALID_ARG;
        const size_t j = txt.find('"', i + 1);
        if (j == std::string::npos) return MCI_ERR_INVALID_ARG;
        const std::string key = txt.substr(i + 1, j - i - 1);
        i = txt.find(':', j);
        if (i == std::string::npos) return MCI_ERR_INVALID_ARG;
        char* end = nullptr;
        const long v = std::strtol(txt.c_str() + i + 1, &end, 10);
        if (end == txt.c_str() + i + 1 || v < 1 || v > kMaxTile) return MCI_ERR_INVALID_ARG;
        got[key] = (int)v;
        i = (size_t)(end - txt.c_str());
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : got) g_tune[kv.first] = kv.second;
    return MCI_OK;
}
