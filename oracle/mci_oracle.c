/*
 * FP64 CPU oracle for FFT multichannel interpolation (MCI).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes (Cheng & Kou, "FFT multichannel interpolation ..."):
 *   Section 3, band partition:  I^N = {N1, ..., N1 + M*P - 1} cut into M
 *     consecutive blocks of P integers (the paper's L is P here).
 *   Eq. (sysfunction): channel m has the Fourier multiplier b_m(n).
 *   Eq. (defH): per residue n in I_1 the M x M matrix
 *     H_n[j][k] = b_k(n + j*P), j = alias block, k = channel.
 *   Remark (aequal0): where H_n is singular the paper zeroes q_{mk}(n); this
 *     oracle offers that reading and the Moore-Penrose pseudo-inverse
 *     (the minimum-norm solution of A_n H_n = D_n, Eq. (matrixeqn1)).
 *   Eq. (defrm): r_m(N1 + k*P + r) = q_{mk}(N1 + r).
 *   Eq. (ym): y_m(t) = sum_{n in I^N} r_m(n) e^{int}; Example 6 applies an
 *     output operator o(n) to it (identity, Hilbert -i sgn n, derivative in).
 *   Theorem (MCIeq), Eq. (drictexpression), and the operator T_N of
 *     Eq. (appxi operator):
 *       out(t) = Re[ (1/P) sum_m sum_p g_m(t_p) y_m(t - t_p) ],  t_p = 2 pi p / P.
 *     Taking the real part follows the experiments of Section 5.1 (Table 1).
 *
 * The sums are evaluated directly, in the definition's order, with
 * Neumaier-compensated accumulation.  Phases are reduced in integers before
 * calling cos/sin of the C library.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef double complex cplx;

enum { SYS_IDENTITY = 0, SYS_DERIV = 1, SYS_HILBERT = 2, SYS_SHIFT = 3, SYS_CUSTOM = 4 };
enum { OUT_F = 0, OUT_HILBERT = 1, OUT_DERIV = 2 };
enum { POLICY_PINV = 0, POLICY_ERROR = 1, POLICY_ZERO = 2 };

enum { ORC_OK = 0, ORC_BAD_ARG = -1, ORC_SINGULAR = -3, ORC_NOMEM = -5 };

static const double TWO_PI = 6.283185307179586476925286766559;

/* e^{2 pi i q / den} with q reduced modulo den in integers first. */
static cplx cis_frac(int64_t q, int64_t den)
{
    q %= den;
    if (q < 0) q += den;
    double a = TWO_PI * (double)q / (double)den;
    return cos(a) + I * sin(a);
}

static int sgn64(int64_t n) { return (n > 0) - (n < 0); }

/* ---------------------------------------------------------------------------
 * System multipliers b(n) (Eq. (sysfunction); Examples 2, 3, 5) and output
 * operators o(n) (Example 6, Section 3 closing remark on Q(f)).
 * custom: table of 2*mu doubles (re, im) for n = N1 .. N1 + mu - 1.
 * ------------------------------------------------------------------------- */
static cplx sys_mult(int kind, int order, double tau, const double *custom,
                     int64_t N1, int64_t mu, int64_t n)
{
    switch (kind) {
    case SYS_IDENTITY: return 1.0;
    case SYS_DERIV: {
        cplx v = 1.0;
        for (int i = 0; i < order; ++i) v *= I * (double)n;
        return v;
    }
    case SYS_HILBERT: return -I * (double)sgn64(n);
    case SYS_SHIFT: return cos((double)n * tau) + I * sin((double)n * tau);
    case SYS_CUSTOM: {
        int64_t i = n - N1;
        if (!custom || i < 0 || i >= mu) return 0.0;
        return custom[2 * i] + I * custom[2 * i + 1];
    }
    }
    return 0.0;
}

static cplx out_mult(int op, int64_t n)
{
    switch (op) {
    case OUT_F: return 1.0;
    case OUT_HILBERT: return -I * (double)sgn64(n);
    case OUT_DERIV: return I * (double)n;
    }
    return 0.0;
}

/* ---------------------------------------------------------------------------
 * Small dense complex linear algebra (row-major n x n).
 * ------------------------------------------------------------------------- */

/* Gauss-Jordan inversion with partial pivoting.  Returns 0, or 1 when a pivot
 * falls below tol (the matrix is treated as singular). */
static int gj_inverse(int n, const cplx *A, cplx *X, double tol)
{
    cplx *W = malloc(sizeof(cplx) * n * 2 * n);
    if (!W) return -1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            W[i * 2 * n + j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = cabs(W[c * 2 * n + c]);
        for (int i = c + 1; i < n; ++i) {
            double v = cabs(W[i * 2 * n + c]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > tol)) { free(W); return 1; }
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) {
                cplx t = W[c * 2 * n + j];
                W[c * 2 * n + j] = W[piv * 2 * n + j];
                W[piv * 2 * n + j] = t;
            }
        cplx inv = 1.0 / W[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) W[c * 2 * n + j] *= inv;
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            cplx f = W[i * 2 * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) W[i * 2 * n + j] -= f * W[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) X[i * n + j] = W[i * 2 * n + n + j];
    free(W);
    return 0;
}

/* Moore-Penrose pseudo-inverse through a full-rank factorisation A = B C:
 * C = the non-zero rows of the reduced row-echelon form of A, B = the pivot
 * columns of A, and pinv(A) = C^H (C C^H)^{-1} (B^H B)^{-1} B^H
 * (the classical formula for a full-rank factorisation).
 * tol decides which pivots of the echelon form count as zero.
 * Returns the rank, or -1 on allocation failure. */
static int fullrank_pinv(int n, const cplx *A, cplx *X, double tol)
{
    cplx *R = malloc(sizeof(cplx) * n * n);
    int *pc = malloc(sizeof(int) * n);
    if (!R || !pc) { free(R); free(pc); return -1; }
    memcpy(R, A, sizeof(cplx) * n * n);
    int rank = 0;
    for (int c = 0; c < n && rank < n; ++c) {
        int piv = rank;
        double best = cabs(R[rank * n + c]);
        for (int i = rank + 1; i < n; ++i) {
            double v = cabs(R[i * n + c]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > tol)) {
            for (int i = rank; i < n; ++i) R[i * n + c] = 0.0;
            continue;
        }
        if (piv != rank)
            for (int j = 0; j < n; ++j) {
                cplx t = R[rank * n + j];
                R[rank * n + j] = R[piv * n + j];
                R[piv * n + j] = t;
            }
        cplx inv = 1.0 / R[rank * n + c];
        for (int j = 0; j < n; ++j) R[rank * n + j] *= inv;
        for (int i = 0; i < n; ++i) {
            if (i == rank) continue;
            cplx f = R[i * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) R[i * n + j] -= f * R[rank * n + j];
        }
        pc[rank++] = c;
    }
    memset(X, 0, sizeof(cplx) * n * n);
    if (rank == 0) { free(R); free(pc); return 0; }
    int r = rank;
    cplx *B = malloc(sizeof(cplx) * n * r);      /* n x r */
    cplx *CC = malloc(sizeof(cplx) * r * r);     /* C C^H */
    cplx *BB = malloc(sizeof(cplx) * r * r);     /* B^H B */
    cplx *CCi = malloc(sizeof(cplx) * r * r);
    cplx *BBi = malloc(sizeof(cplx) * r * r);
    cplx *Mid = malloc(sizeof(cplx) * r * r);
    if (!B || !CC || !BB || !CCi || !BBi || !Mid) {
        free(B); free(CC); free(BB); free(CCi); free(BBi); free(Mid); free(R); free(pc);
        return -1;
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < r; ++k) B[i * r + k] = A[i * n + pc[k]];
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            cplx s1 = 0.0, s2 = 0.0;
            for (int j = 0; j < n; ++j) {
                s1 += R[a * n + j] * conj(R[b * n + j]);
                s2 += conj(B[j * r + a]) * B[j * r + b];
            }
            CC[a * r + b] = s1;
            BB[a * r + b] = s2;
        }
    gj_inverse(r, CC, CCi, 0.0);
    gj_inverse(r, BB, BBi, 0.0);
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            cplx s = 0.0;
            for (int k = 0; k < r; ++k) s += CCi[a * r + k] * BBi[k * r + b];
            Mid[a * r + b] = s;
        }
    /* X = C^H * Mid * B^H, C = rows 0..r-1 of R */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cplx s = 0.0;
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b)
                    s += conj(R[a * n + i]) * Mid[a * r + b] * conj(B[j * r + b]);
            X[i * n + j] = s;
        }
    free(B); free(CC); free(BB); free(CCi); free(BBi); free(Mid); free(R); free(pc);
    return rank;
}

/* ---------------------------------------------------------------------------
 * Problem description shared by the entry points below.
 * ------------------------------------------------------------------------- */
typedef struct {
    int M;
    const int *kind;      /* M */
    const int *order;     /* M */
    const double *tau;    /* M */
    const double *custom; /* M * 2 * mu doubles, or NULL */
    int64_t P;
    int64_t N1;
} orc_sys;

static cplx orc_b(const orc_sys *s, int k, int64_t n)
{
    int64_t mu = (int64_t)s->M * s->P;
    const double *tab = s->custom ? s->custom + (size_t)k * 2 * mu : NULL;
    return sys_mult(s->kind[k], s->order ? s->order[k] : 1, s->tau ? s->tau[k] : 0.0, tab,
                    s->N1, mu, n);
}

/*
 * oracle_q_table: Q_r = H_r^{-1} (or its pseudo-inverse), r = 0..P-1,
 * H_r[j][k] = b_k(N1 + r + j*P)  (Eq. (defH)).
 * Q is written row-major per residue: Q[((r*M)+m)*M + j] (re, im interleaved),
 * row m = channel, column j = alias block, i.e. q_{m,j+1}(N1 + r).
 * A residue is singular when Gauss-Jordan meets a pivot below
 * rtol * max|H_r|.  policy: 0 pseudo-inverse, 1 return ORC_SINGULAR,
 * 2 zero the residue (Remark aequal0).
 * *n_singular receives the number of singular residues.
 */
int oracle_q_table(int M, const int *kind, const int *order, const double *tau,
                   const double *custom, int64_t P, int64_t N1, int policy, double rtol,
                   double *Q, int *n_singular)
{
    if (M < 1 || P < 1 || !kind || !Q) return ORC_BAD_ARG;
    orc_sys s = {M, kind, order, tau, custom, P, N1};
    cplx *H = malloc(sizeof(cplx) * M * M), *X = malloc(sizeof(cplx) * M * M);
    if (!H || !X) { free(H); free(X); return ORC_NOMEM; }
    int nsing = 0;
    for (int64_t r = 0; r < P; ++r) {
        int64_t n = N1 + r;
        double scale = 0.0;
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < M; ++k) {
                H[j * M + k] = orc_b(&s, k, n + (int64_t)j * P);
                if (cabs(H[j * M + k]) > scale) scale = cabs(H[j * M + k]);
            }
        double tol = rtol * scale;
        int sing = (scale == 0.0) ? 1 : gj_inverse(M, H, X, tol);
        if (sing < 0) { free(H); free(X); return ORC_NOMEM; }
        if (sing) {
            ++nsing;
            if (policy == POLICY_ERROR) { free(H); free(X); if (n_singular) *n_singular = nsing; return ORC_SINGULAR; }
            if (policy == POLICY_ZERO || scale == 0.0) memset(X, 0, sizeof(cplx) * M * M);
            else if (fullrank_pinv(M, H, X, tol) < 0) { free(H); free(X); return ORC_NOMEM; }
        }
        for (int m = 0; m < M; ++m)
            for (int j = 0; j < M; ++j) {
                cplx q = X[m * M + j];
                Q[2 * ((r * M + m) * M + j)] = creal(q);
                Q[2 * ((r * M + m) * M + j) + 1] = cimag(q);
            }
    }
    if (n_singular) *n_singular = nsing;
    free(H); free(X);
    return ORC_OK;
}

/* r_m(n) for n in the band from the Q table (Eq. (defrm)):
 * r[(m*mu) + (n - N1)] with n = N1 + j*P + r  ->  q_{m,j}(N1 + r). */
static void build_r(int M, int64_t P, const double *Q, cplx *rm)
{
    int64_t mu = (int64_t)M * P;
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < M; ++j)
            for (int64_t r = 0; r < P; ++r) {
                const double *q = Q + 2 * ((r * M + m) * M + j);
                rm[(int64_t)m * mu + j * P + r] = q[0] + I * q[1];
            }
}

/* Neumaier-compensated accumulator. */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nval(const nsum *a) { return a->s + a->c; }

static int hw_threads(int req)
{
    if (req > 0) return req;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* ---------------------------------------------------------------------------
 * y_m tabulated on the T-grid (Eq. (ym) with output operator o):
 *   Y[m*T + l] = sum_{n in band} r_m(n) o(n) e^{2 pi i n l / T}
 * ------------------------------------------------------------------------- */
typedef struct {
    int M; int64_t P, T, N1; int op;
    const cplx *rm; const cplx *cis; cplx *Y;
    int64_t l0, l1;
} ytab_job;

static void *ytab_worker(void *arg)
{
    ytab_job *jb = arg;
    int64_t mu = (int64_t)jb->M * jb->P;
    for (int m = 0; m < jb->M; ++m)
        for (int64_t l = jb->l0; l < jb->l1; ++l) {
            nsum re = {0, 0}, im = {0, 0};
            for (int64_t i = 0; i < mu; ++i) {
                int64_t n = jb->N1 + i;
                int64_t q = (n % jb->T) * l % jb->T;
                if (q < 0) q += jb->T;
                cplx v = jb->rm[(int64_t)m * mu + i] * out_mult(jb->op, n) * jb->cis[q];
                nadd(&re, creal(v));
                nadd(&im, cimag(v));
            }
            jb->Y[(int64_t)m * jb->T + l] = nval(&re) + I * nval(&im);
        }
    return NULL;
}

static int build_ytab(int M, int64_t P, int64_t T, int64_t N1, int op, const cplx *rm,
                      cplx *Y, int nthreads)
{
    cplx *cis = malloc(sizeof(cplx) * T);
    if (!cis) return ORC_NOMEM;
    for (int64_t q = 0; q < T; ++q) cis[q] = cis_frac(q, T);
    int nt = hw_threads(nthreads);
    if (nt > T) nt = (int)T;
    pthread_t *th = malloc(sizeof(pthread_t) * nt);
    ytab_job *jobs = malloc(sizeof(ytab_job) * nt);
    if (!th || !jobs) { free(cis); free(th); free(jobs); return ORC_NOMEM; }
    for (int t = 0; t < nt; ++t) {
        jobs[t] = (ytab_job){M, P, T, N1, op, rm, cis, Y, T * t / nt, T * (t + 1) / nt};
        pthread_create(&th[t], NULL, ytab_worker, &jobs[t]);
    }
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs); free(cis);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Direct sum formula (Theorem MCIeq / operator T_N):
 *   out[b][o][j] = Re[ (1/P) sum_m sum_p g[b][m][p] y^{o}_m(t_j - t_p) ],
 *   t_j = 2 pi j / T,  t_p = 2 pi p / P.
 * When P divides T every t_j - t_p lies on the T-grid and the tabulated y is
 * used; otherwise y_m(t_j - t_p) is summed over the band for every pair.
 * g: batch x M x P (real samples).  ops: n_ops output operators.
 * out: batch x n_ops x T.  If idx != NULL only the n_idx grid points idx[]
 * are evaluated and out is batch x n_ops x n_idx.
 * ------------------------------------------------------------------------- */
typedef struct {
    int M; int64_t P, T, N1; int n_ops; const int *ops;
    const cplx *Y;       /* n_ops x M x T, grid route */
    const cplx *rm;      /* M x mu, general route */
    const double *g; double *out;
    const int64_t *idx; int64_t n_idx;
    int64_t b0, b1;
} sum_job;

static void *sum_worker(void *arg)
{
    sum_job *jb = arg;
    const int M = jb->M;
    const int64_t P = jb->P, T = jb->T, mu = (int64_t)M * P;
    const int64_t npts = jb->idx ? jb->n_idx : T;
    for (int64_t b = jb->b0; b < jb->b1; ++b) {
        const double *gb = jb->g + b * M * P;
        for (int o = 0; o < jb->n_ops; ++o)
            for (int64_t ii = 0; ii < npts; ++ii) {
                int64_t j = jb->idx ? jb->idx[ii] : ii;
                nsum acc = {0, 0};
                for (int m = 0; m < M; ++m)
                    for (int64_t p = 0; p < P; ++p) {
                        double y;
                        if (jb->Y) {
                            int64_t l = (j - p * (T / P)) % T;
                            if (l < 0) l += T;
                            y = creal(jb->Y[((int64_t)o * M + m) * T + l]);
                        } else {
                            /* y_m(t_j - t_p), phase n (jP - pT) / (TP) reduced in integers */
                            nsum yr = {0, 0};
                            for (int64_t i = 0; i < mu; ++i) {
                                int64_t n = jb->N1 + i;
                                cplx v = jb->rm[(int64_t)m * mu + i] * out_mult(jb->ops[o], n) *
                                         cis_frac(n * (j * P - p * T), T * P);
                                nadd(&yr, creal(v));
                            }
                            y = nval(&yr);
                        }
                        nadd(&acc, gb[(int64_t)m * P + p] * y);
                    }
                jb->out[(b * jb->n_ops + o) * npts + ii] = nval(&acc) / (double)P;
            }
    }
    return NULL;
}

int oracle_mci_direct(int M, const int *kind, const int *order, const double *tau,
                      const double *custom, int64_t P, int64_t N1, int64_t T, int policy,
                      double rtol, int n_ops, const int *ops, const double *g, int64_t batch,
                      const int64_t *idx, int64_t n_idx, double *out, int nthreads,
                      int *n_singular)
{
    if (M < 1 || P < 1 || T < 1 || n_ops < 1 || !ops || !g || !out || batch < 0)
        return ORC_BAD_ARG;
    int64_t mu = (int64_t)M * P;
    double *Q = malloc(sizeof(double) * 2 * P * M * M);
    cplx *rm = malloc(sizeof(cplx) * M * mu);
    if (!Q || !rm) { free(Q); free(rm); return ORC_NOMEM; }
    int rc = oracle_q_table(M, kind, order, tau, custom, P, N1, policy, rtol, Q, n_singular);
    if (rc) { free(Q); free(rm); return rc; }
    build_r(M, P, Q, rm);
    cplx *Y = NULL;
    if (T % P == 0) {
        Y = malloc(sizeof(cplx) * n_ops * M * T);
        if (!Y) { free(Q); free(rm); return ORC_NOMEM; }
        for (int o = 0; o < n_ops; ++o) {
            rc = build_ytab(M, P, T, N1, ops[o], rm, Y + (int64_t)o * M * T, nthreads);
            if (rc) { free(Q); free(rm); free(Y); return rc; }
        }
    }
    int nt = hw_threads(nthreads);
    if (nt > batch) nt = (int)(batch > 0 ? batch : 1);
    pthread_t *th = malloc(sizeof(pthread_t) * nt);
    sum_job *jobs = malloc(sizeof(sum_job) * nt);
    if (!th || !jobs) { free(Q); free(rm); free(Y); free(th); free(jobs); return ORC_NOMEM; }
    if (batch == 1 && nt == 1) nt = 1;
    for (int t = 0; t < nt; ++t) {
        jobs[t] = (sum_job){M, P, T, N1, n_ops, ops, Y, rm, g, out, idx, n_idx,
                            batch * t / nt, batch * (t + 1) / nt};
        pthread_create(&th[t], NULL, sum_worker, &jobs[t]);
    }
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs); free(Q); free(rm); free(Y);
    return ORC_OK;
}

/* y_m on the T-grid for inspection against the paper's closed forms:
 * Y[(m*T)+l] (re, im interleaved) = sum_n r_m(n) o(n) e^{2 pi i n l / T}. */
int oracle_interp_functions(int M, const int *kind, const int *order, const double *tau,
                            const double *custom, int64_t P, int64_t N1, int64_t T, int policy,
                            double rtol, int op, double *Yout, int nthreads)
{
    if (M < 1 || P < 1 || T < 1 || !Yout) return ORC_BAD_ARG;
    int64_t mu = (int64_t)M * P;
    double *Q = malloc(sizeof(double) * 2 * P * M * M);
    cplx *rm = malloc(sizeof(cplx) * M * mu);
    cplx *Y = malloc(sizeof(cplx) * M * T);
    if (!Q || !rm || !Y) { free(Q); free(rm); free(Y); return ORC_NOMEM; }
    int rc = oracle_q_table(M, kind, order, tau, custom, P, N1, policy, rtol, Q, NULL);
    if (!rc) {
        build_r(M, P, Q, rm);
        rc = build_ytab(M, P, T, N1, op, rm, Y, nthreads);
    }
    if (!rc)
        for (int64_t i = 0; i < (int64_t)M * T; ++i) {
            Yout[2 * i] = creal(Y[i]);
            Yout[2 * i + 1] = cimag(Y[i]);
        }
    free(Q); free(rm); free(Y);
    return rc;
}
