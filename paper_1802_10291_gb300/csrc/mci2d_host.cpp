// Host side of the 2-D MCI interface (include/mci2d.h): validation, FP64 plan tables
// (per-residue inverses, output phase factors, FFT roots) and the entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "mci2d_internal.h"
#include "mci_linalg.h"

using mci2::Dims2;
using mci2::kSmemMax;

namespace {

using cd = std::complex<double>;
constexpr double kTwoPi2 = 6.283185307179586476925286766559;

cd cis2(int64_t q, int64_t den)
{
    q %= den;
    if (q < 0) q += den;
    const double a = kTwoPi2 * (double)q / (double)den;
    return cd(std::cos(a), std::sin(a));
}

cd multiplier2(const mci2_system& s, int64_t ny, int64_t nx)
{
    switch (s.kind) {
    case MCI2_SYS_IDENTITY: return 1.0;
    case MCI2_SYS_PARTIAL: {
        cd v = 1.0;
        for (int i = 0; i < s.order_y; ++i) v *= cd(0.0, (double)ny);
        for (int i = 0; i < s.order_x; ++i) v *= cd(0.0, (double)nx);
        return v;
    }
    case MCI2_SYS_LAPLACIAN: return -((double)ny * (double)ny + (double)nx * (double)nx);
    case MCI2_SYS_SHIFT: {
        const double a = (double)ny * s.tau_y + (double)nx * s.tau_x;
        return cd(std::cos(a), std::sin(a));
    }
    case MCI2_SYS_RIESZ: {
        const double r = std::sqrt((double)ny * ny + (double)nx * nx);
        if (r == 0.0) return 0.0;
        return cd(0.0, -(double)(s.order_y == 0 ? ny : nx) / r);
    }
    }
    return 0.0;
}

bool supported_p2(int P)
{
    if (P < 4 || P > 1024 || P % 2) return false;
    int q = P % 3 == 0 ? P / 3 : P;
    return (q & (q - 1)) == 0;
}

}  // namespace

struct mci2_plan_s {
    mci2_desc d{};
    std::vector<mci2_system> sys;
    Dims2 dims{};
    int64_t N1y = 0, N1x = 0;
    int n_singular = 0;
    double max_cond = 1.0;
    size_t csz = 8;
    void* Qt = nullptr;
    void* Fy = nullptr;
    void* Oy = nullptr;
    void* Fx = nullptr;
    void* roots1 = nullptr;
    void* roots2 = nullptr;
    void* X = nullptr;
    void* Zw = nullptr;
    int64_t ws_bytes = 0;
    size_t smem1 = 0, smem2 = 0, smem3 = 0;
};

namespace {

template <typename R>
void push(std::vector<R>& v, cd z)
{
    v.push_back((R)z.real());
    v.push_back((R)z.imag());
}

template <typename R>
mci_status upload(const std::vector<R>& v, void** dst, cudaStream_t st)
{
    if (cudaMalloc(dst, v.size() * sizeof(R)) != cudaSuccess) return MCI_ERR_OOM;
    if (cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(R), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MCI_ERR_CUDA;
    return MCI_OK;
}

template <typename R>
mci_status build2(mci2_plan_s* p, cudaStream_t st)
{
    const mci2_desc& d = p->d;
    const Dims2& D = p->dims;
    const int M = D.M, P1 = D.P1, P2 = D.P2;
    const double rtol = d.singular_rtol > 0 ? d.singular_rtol : 1e-13;
    // Q table [r2][m][j][r1] with 1 / (2 P1 P2) folded in (bins of one column read
    // consecutive r1)
    std::vector<R> Q((size_t)P1 * P2 * M * M * 2);
    std::vector<cd> H(M * M), q(M * M);
    const double scale = 1.0 / (2.0 * P1 * P2);
    for (int r2 = 0; r2 < P2; ++r2)
        for (int r1 = 0; r1 < P1; ++r1) {
            for (int j = 0; j < M; ++j) {
                const int64_t ny = p->N1y + r1 + (int64_t)(j / D.Mx) * P1;
                const int64_t nx = p->N1x + r2 + (int64_t)(j % D.Mx) * P2;
                for (int k = 0; k < M; ++k) H[j * M + k] = multiplier2(p->sys[k], ny, nx);
            }
            bool sing = false;
            double cond = 1.0;
            const mci_status s = mci::invert_system(M, H, rtol, d.singular_policy, q.data(), &sing, &cond);
            if (s != MCI_OK) return s;
            if (sing) ++p->n_singular;
            else p->max_cond = std::max(p->max_cond, cond);
            for (int i = 0; i < M * M; ++i) {
                const size_t e = (((size_t)r2 * M * M + i) * P1 + r1) * 2;
                Q[e] = (R)(q[i].real() * scale);
                Q[e + 1] = (R)(q[i].imag() * scale);
            }
        }
    // phase factors e^{2 pi i n u / T} per axis: [u][j_axis][r]
    // along y the factor splits as e^{2 pi i (N1y + r) u / T1} e^{2 pi i jy u / s1}
    std::vector<R> Fy, Oy, Fx, ro1, ro2;
    for (int u = 0; u < D.s1; ++u)
        for (int r = 0; r < P1; ++r) push(Fy, cis2((p->N1y + r) * u, D.T1));
    for (int u = 0; u < D.s1; ++u)
        for (int jy = 0; jy < D.My; ++jy) push(Oy, cis2((int64_t)jy * u, D.s1));
    for (int u = 0; u < D.s2; ++u)
        for (int jx = 0; jx < D.Mx; ++jx)
            for (int r = 0; r < P2; ++r) push(Fx, cis2((p->N1x + r + (int64_t)jx * P2) * u, D.T2));
    for (int k = 0; k < P1; ++k) push(ro1, cis2(-k, P1));
    for (int k = 0; k < P2; ++k) push(ro2, cis2(-k, P2));
    mci_status s;
    if ((s = upload(Q, &p->Qt, st)) != MCI_OK) return s;
    if ((s = upload(Fy, &p->Fy, st)) != MCI_OK) return s;
    if ((s = upload(Oy, &p->Oy, st)) != MCI_OK) return s;
    if ((s = upload(Fx, &p->Fx, st)) != MCI_OK) return s;
    if ((s = upload(ro1, &p->roots1, st)) != MCI_OK) return s;
    if ((s = upload(ro2, &p->roots2, st)) != MCI_OK) return s;
    // host tables must stay alive until the copies finish
    return cudaStreamSynchronize(st) == cudaSuccess ? MCI_OK : MCI_ERR_CUDA;
}

void free2(mci2_plan_s* p)
{
    void* bufs[8] = {p->Qt, p->Fy, p->Oy, p->Fx, p->roots1, p->roots2, p->X, p->Zw};
    for (int i = 0; i < 8; ++i)
        if (bufs[i]) cudaFree(bufs[i]);
    delete p;
}

}  // namespace

extern "C" {

mci_status mci2_plan(mci2_plan_t* out, const mci2_desc* d, mci_stream_t stream)
{
    if (!out) return MCI_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d || d->My < 1 || d->Mx < 1 || d->My * d->Mx > 8 || !d->sys) return MCI_ERR_INVALID_ARG;
    if (d->precision != MCI_FP32 && d->precision != MCI_FP64) return MCI_ERR_INVALID_ARG;
    if (d->singular_policy < 0 || d->singular_policy > 2) return MCI_ERR_INVALID_ARG;
    if (d->max_batch < 1 || d->max_batch > 65535) return MCI_ERR_INVALID_ARG;
    const int M = d->My * d->Mx;
    for (int k = 0; k < M; ++k) {
        const mci2_system& s = d->sys[k];
        if (s.kind < MCI2_SYS_IDENTITY || s.kind > MCI2_SYS_RIESZ) return MCI_ERR_INVALID_ARG;
        if (s.kind == MCI2_SYS_PARTIAL && (s.order_y < 0 || s.order_x < 0 || s.order_y + s.order_x > 16))
            return MCI_ERR_INVALID_ARG;
        if (s.kind == MCI2_SYS_RIESZ && s.order_y != 0 && s.order_y != 1) return MCI_ERR_INVALID_ARG;
        if (s.kind == MCI2_SYS_SHIFT && !(std::isfinite(s.tau_y) && std::isfinite(s.tau_x)))
            return MCI_ERR_INVALID_ARG;
    }
    if (!supported_p2(d->P1) || !supported_p2(d->P2)) return MCI_ERR_UNSUPPORTED_SIZE;
    if (d->T1 < d->P1 || d->T2 < d->P2 || d->T1 % d->P1 || d->T2 % d->P2) return MCI_ERR_UNSUPPORTED_SIZE;
    if (d->T1 / d->P1 > 16 || d->T2 / d->P2 > 16) return MCI_ERR_UNSUPPORTED_SIZE;

    mci2_plan_s* p = new (std::nothrow) mci2_plan_s;
    if (!p) return MCI_ERR_OOM;
    p->d = *d;
    p->sys.assign(d->sys, d->sys + M);
    p->d.sys = p->sys.data();
    p->d.N1 = nullptr;
    p->N1y = d->N1 ? d->N1[0] : -(int64_t)((d->My * d->P1) / 2);
    p->N1x = d->N1 ? d->N1[1] : -(int64_t)((d->Mx * d->P2) / 2);
    p->csz = d->precision == MCI_FP64 ? 16 : 8;
    Dims2& D = p->dims;
    D.M = M;
    D.My = d->My;
    D.Mx = d->Mx;
    D.P1 = d->P1;
    D.P2 = d->P2;
    D.H2 = d->P2 / 2;
    D.T1 = d->T1;
    D.T2 = d->T2;
    D.s1 = d->T1 / d->P1;
    D.s2 = d->T2 / d->P2;
    D.N1y_mod = (int)(((p->N1y % D.P1) + D.P1) % D.P1);
    D.N1x_mod = (int)(((p->N1x % D.P2) + D.P2) % D.P2);
    const size_t csz = p->csz;
    // pass 1: G1 rows per CTA (even divisor of P1); shared memory: FFT sequences at stride
    // P2 + 1 (G1 of them with the scratch) and P2 FFT roots, likewise in the other passes
    D.G1 = 2;
    for (int g : {16, 8, 4})
        if (D.P1 % g == 0 && (size_t)g * D.P2 * csz <= 96 * 1024) {
            D.G1 = g;
            break;
        }
    p->smem1 = ((size_t)D.G1 * (D.P2 + 1) + D.P2) * csz;
    // pass 2: 2 M sequences for the spectra, 2 chunk for the phase FFTs (chunk of the s1 s2 output
    // phases per batch), the roots and 2 chunk M phase factors; the largest chunk within 56 KB
    // (four CTAs per SM), or one phase at a time
    auto smem_col = [&](int chunk) {
        return ((size_t)(2 * M + 2 * chunk) * (D.P1 + 1) + D.P1 + (size_t)2 * chunk * M) * csz;
    };
    D.chunk = D.s1 * D.s2;
    while (D.chunk > 1 && smem_col(D.chunk) > (size_t)56 * 1024) --D.chunk;
    p->smem2 = smem_col(D.chunk);
    // pass 3: G3 output rows per CTA (even divisor of T1), G3 s2 sequences with the scratch
    D.G3 = 2;
    for (int g : {8, 4})
        if (D.T1 % g == 0 && (size_t)g * D.s2 * D.P2 * csz <= 96 * 1024) {
            D.G3 = g;
            break;
        }
    p->smem3 = ((size_t)D.G3 * D.s2 * (D.P2 + 1) + D.P2) * csz;
    D.lgG1 = 31 - __builtin_clz((unsigned)D.G1);
    D.lgG3 = 31 - __builtin_clz((unsigned)D.G3);
    if (p->smem1 > (size_t)kSmemMax || p->smem2 > (size_t)kSmemMax ||
        p->smem3 > (size_t)kSmemMax) {
        free2(p);
        return MCI_ERR_UNSUPPORTED_SIZE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    mci_status s = d->precision == MCI_FP64 ? build2<double>(p, st) : build2<float>(p, st);
    if (s == MCI_OK) s = mci2::set_smem(d->precision, p->smem1, p->smem2, p->smem3);
    if (s == MCI_OK) {
        const int64_t xb = d->max_batch * M * (D.H2 + 1) * D.P1 * (int64_t)csz;
        const int64_t zb = d->max_batch * D.s2 * (D.H2 + 1) * D.T1 * (int64_t)csz;
        p->ws_bytes = xb + zb;
        if (cudaMalloc(&p->X, xb) != cudaSuccess || cudaMalloc(&p->Zw, zb) != cudaSuccess) s = MCI_ERR_OOM;
    }
    if (s != MCI_OK) {
        cudaGetLastError();
        free2(p);
        return s;
    }
    *out = p;
    return MCI_OK;
}

mci_status mci2_interp(mci2_plan_t p, const void* in, void* out, int64_t batch, mci_stream_t stream)
{
    if (!p || batch < 0 || batch > p->d.max_batch) return MCI_ERR_INVALID_ARG;
    if (batch == 0) return MCI_OK;
    if (!in || !out || ((uintptr_t)in % 16) || ((uintptr_t)out % 16)) return MCI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const mci2::Tables t{p->Qt, p->Fy, p->Oy, p->Fx, p->roots1, p->roots2, p->X, p->Zw};
    return mci2::launch(p->d.precision, p->dims, t, p->smem1, p->smem2, p->smem3, in, out, batch, st);
}

mci_status mci2_plan_info(mci2_plan_t p, int* n_singular, double* max_cond, int64_t* workspace_bytes)
{
    if (!p) return MCI_ERR_INVALID_ARG;
    if (n_singular) *n_singular = p->n_singular;
    if (max_cond) *max_cond = p->max_cond;
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    return MCI_OK;
}

mci_status mci2_destroy(mci2_plan_t p)
{
    if (!p) return MCI_OK;
    cudaDeviceSynchronize();
    free2(p);
    return MCI_OK;
}

}  // extern "C"
