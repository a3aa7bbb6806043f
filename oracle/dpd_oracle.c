/*
 * FP64 reference ("oracle") for the augmented-parallel-Hammerstein (APH) DPD
 * filter of Li et al., "Parallel Digital Predistortion Design on Mobile GPU and
 * Embedded Multicore CPU for Mobile Transmitters".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA library: no headers, no helpers, no tables.  It is written to be read
 * against the paper, not to be fast: plain loops over the definitions, in
 * double precision, with C99 complex arithmetic.
 *
 * Conventions (all arrays interleaved re,im; complex double == double[2]):
 *   x      : input samples x_0 .. x_{N-1}                      (Sec. 2.1)
 *   h      : coefficient vector, stacked as in Sec. 2.2:
 *            [h_1, h_3, ..., h_P, hbar_1, hbar_3, ..., hbar_Q, c],
 *            each h_p = [h_{p,0} .. h_{p,L-1}], L = M + 1 taps.
 *   P, Q   : highest odd order of the main / conjugate branch; Q = 0 means no
 *            conjugate branch (I_Q empty), likewise P = 0.
 *   Samples before x_0 are zero (the zero rows at the top of the basis matrix,
 *   Eq. 2); the output has N samples.
 *
 * The paper's orthogonalising coefficients u_{m,p} are taken as the identity, so
 * that psi_p(x) = |x|^{p-1} x and psibar_q(x) = |x|^{q-1} conj(x) (Sec. 2.1).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_BAD_ARG 1
#define OR_NOT_SPD 6

typedef double complex cplx;

static int nbranch(int order) { return order > 0 ? (order + 1) / 2 : 0; }

static int check_model(int P, int Q, int M)
{
    if (P < 0 || Q < 0 || M < 0) return 0;
    if ((P > 0 && P % 2 == 0) || (Q > 0 && Q % 2 == 0)) return 0;
    if (P == 0 && Q == 0) return 0;
    return 1;
}

int oracle_num_coeffs(int P, int Q, int M)
{
    if (!check_model(P, Q, M)) return -1;
    return (nbranch(P) + nbranch(Q)) * (M + 1) + 1;
}

/* |x|^{p-1} for odd p, formed from low order to high order (Sec. 3.2.1):
 * |x|^{p-1} = (|x|^2)^{(p-1)/2}, one factor |x|^2 per order step. */
static double mag_pow(cplx x, int p)
{
    double r = creal(x) * creal(x) + cimag(x) * cimag(x);
    double w = 1.0;
    for (int o = 1; o < p; o += 2) w *= r;
    return w;
}

/* psi_p(x) = |x|^{p-1} x  (main branch, Sec. 2.1) */
static cplx psi(cplx x, int p) { return mag_pow(x, p) * x; }

/* psibar_q(x) = psi_q(x^*) = |x|^{q-1} x^*  (conjugate branch, Sec. 2.1) */
static cplx psibar(cplx x, int q) { return mag_pow(x, q) * conj(x); }

static cplx sample(const cplx *x, int64_t n, int64_t j) { return (j >= 0 && j < n) ? x[j] : 0.0; }

/*
 * Eq. 1 / Algorithm 1: for every n,
 *   f_p(x_n)    = sum_{k=0}^{L-1} h_{p,k}    psi_p(x_{n-k})       (filtering)
 *   fbar_q(x_n) = sum_{k=0}^{L-1} hbar_{q,k} psibar_q(x_{n-k})
 *   z_n         = sum_p f_p + sum_q fbar_q + c                     (accumulation)
 */
int oracle_apply(int P, int Q, int M, const double *h_, const double *x_, int64_t n,
                 double *y_, int nthreads)
{
    if (!check_model(P, Q, M) || n < 0 || (n > 0 && (!x_ || !y_)) || !h_) return OR_BAD_ARG;
    const cplx *h = (const cplx *)h_;
    const cplx *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
    const int L = M + 1, Bp = nbranch(P), Bq = nbranch(Q);
    const cplx c = h[(Bp + Bq) * L];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
        cplx z = 0.0;
        for (int b = 0; b < Bp; ++b) {              /* p in I_P = {1, 3, ..., P} */
            int p = 2 * b + 1;
            cplx f = 0.0;
            for (int k = 0; k < L; ++k) f += h[b * L + k] * psi(sample(x, n, i - k), p);
            z += f;
        }
        for (int b = 0; b < Bq; ++b) {              /* q in I_Q = {1, 3, ..., Q} */
            int q = 2 * b + 1;
            cplx f = 0.0;
            for (int k = 0; k < L; ++k) f += h[(Bp + b) * L + k] * psibar(sample(x, n, i - k), q);
            z += f;
        }
        y[i] = z + c;
    }
    (void)nthreads;
    return OR_OK;
}

/*
 * One row of the basis matrix Psi (Eq. 2), columns in the stacking order of
 * Sec. 2.2: column (p,k) holds psi_p(x_{n-k}), column (q,k) holds
 * psibar_q(x_{n-k}), the last column is 1 (it multiplies c).
 */
static void basis_row(int P, int Q, int M, const cplx *x, int64_t n, int64_t i, cplx *row)
{
    const int L = M + 1, Bp = nbranch(P), Bq = nbranch(Q);
    for (int b = 0; b < Bp; ++b)
        for (int k = 0; k < L; ++k) row[b * L + k] = psi(sample(x, n, i - k), 2 * b + 1);
    for (int b = 0; b < Bq; ++b)
        for (int k = 0; k < L; ++k) row[(Bp + b) * L + k] = psibar(sample(x, n, i - k), 2 * b + 1);
    row[(Bp + Bq) * L] = 1.0;
}

static int nthreads_used(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * Gradient of a real loss through y = DPD(x) under the convention
 * grad = dL/dRe + j dL/dIm (PyTorch's), given gy = grad w.r.t. y.
 *
 *   gh_j = sum_n conj(Psi_{n,j}) gy_n                          (all K columns)
 *   gx_i = sum_{k} [ conj(dy_{i+k}/dx_i) gy_{i+k} + (dy_{i+k}/dconj(x_i)) conj(gy_{i+k}) ]
 *
 * With r = |x|^2 and m = (p-1)/2, psi_p = r^m x and psibar_q = r^m conj(x):
 *   d(r^m x)/dx = (m+1) r^m,            d(r^m x)/dconj(x) = m r^{m-1} x^2,
 *   d(r^m conj x)/dx = m r^{m-1} conj(x)^2,  d(r^m conj x)/dconj(x) = (m+1) r^m.
 * (m r^{m-1} is 0 for m = 0.)  gh or gx may be NULL.
 * Partial sums of gh are kept per thread and added in thread order.
 */
int oracle_grad(int P, int Q, int M, const double *h_, const double *x_, const double *gy_,
                int64_t n, double *gh_, double *gx_, int nthreads)
{
    if (!check_model(P, Q, M) || n < 0 || !h_) return OR_BAD_ARG;
    if (n > 0 && (!x_ || !gy_)) return OR_BAD_ARG;
    const cplx *h = (const cplx *)h_;
    const cplx *x = (const cplx *)x_;
    const cplx *gy = (const cplx *)gy_;
    const int L = M + 1, Bp = nbranch(P), Bq = nbranch(Q);
    const int K = (Bp + Bq) * L + 1;

    if (gh_) {
        int nt = nthreads_used(nthreads);
        cplx *part = (cplx *)calloc((size_t)nt * K, sizeof(cplx));
        if (!part) return OR_BAD_ARG;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
        {
            int t = 0, tn = 1;
#ifdef _OPENMP
            t = omp_get_thread_num();
            tn = omp_get_num_threads();
#endif
            cplx *acc = part + (size_t)t * K;
            cplx *row = (cplx *)malloc(sizeof(cplx) * K);
            int64_t lo = n * t / tn, hi = n * (t + 1) / tn;
            for (int64_t i = lo; i < hi; ++i) {
                basis_row(P, Q, M, x, n, i, row);
                for (int j = 0; j < K; ++j) acc[j] += conj(row[j]) * gy[i];
            }
            free(row);
        }
        cplx *gh = (cplx *)gh_;
        for (int j = 0; j < K; ++j) {
            cplx s = 0.0;
            for (int t = 0; t < nt; ++t) s += part[(size_t)t * K + j];
            gh[j] = s;
        }
        free(part);
    }

    if (gx_) {
        cplx *gx = (cplx *)gx_;
#ifdef _OPENMP
        if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < n; ++i) {
            cplx xi = x[i];
            double r = creal(xi) * creal(xi) + cimag(xi) * cimag(xi);
            cplx g = 0.0;
            for (int k = 0; k < L && i + k < n; ++k) {
                cplx dx = 0.0, dxc = 0.0;   /* dy_{i+k}/dx_i and dy_{i+k}/dconj(x_i) */
                for (int b = 0; b < Bp; ++b) {
                    cplx hk = h[b * L + k];
                    int m = b;
                    double rm = 1.0, rm1 = 1.0;
                    for (int e = 0; e < m; ++e) rm *= r;
                    for (int e = 0; e < m - 1; ++e) rm1 *= r;
                    dx += hk * (m + 1) * rm;
                    if (m > 0) dxc += hk * m * rm1 * xi * xi;
                }
                for (int b = 0; b < Bq; ++b) {
                    cplx gk = h[(Bp + b) * L + k];
                    int m = b;
                    double rm = 1.0, rm1 = 1.0;
                    for (int e = 0; e < m; ++e) rm *= r;
                    for (int e = 0; e < m - 1; ++e) rm1 *= r;
                    if (m > 0) dx += gk * m * rm1 * conj(xi) * conj(xi);
                    dxc += gk * (m + 1) * rm;
                }
                g += conj(dx) * gy[i + k] + dxc * conj(gy[i + k]);
            }
            gx[i] = g;
        }
    }
    return OR_OK;
}

/*
 * Normal equations of the least-squares estimate of Sec. 2.2:
 *   G = Psi^H Psi  (K x K, row-major),  b = Psi^H t.
 * Rows are taken one at a time; partial sums per thread, added in thread order.
 */
int oracle_gram(int P, int Q, int M, const double *u_, const double *t_, int64_t n,
                double *G_, double *b_, int nthreads)
{
    if (!check_model(P, Q, M) || n < 0 || !G_) return OR_BAD_ARG;
    if (n > 0 && !u_) return OR_BAD_ARG;
    const cplx *u = (const cplx *)u_;
    const cplx *t = (const cplx *)t_;
    const int L = M + 1, Bp = nbranch(P), Bq = nbranch(Q);
    const int K = (Bp + Bq) * L + 1;
    int nt = nthreads_used(nthreads);
    size_t per = (size_t)K * K + K;
    cplx *part = (cplx *)calloc((size_t)nt * per, sizeof(cplx));
    if (!part) return OR_BAD_ARG;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int th = 0, tn = 1;
#ifdef _OPENMP
        th = omp_get_thread_num();
        tn = omp_get_num_threads();
#endif
        cplx *accG = part + (size_t)th * per;
        cplx *accb = accG + (size_t)K * K;
        cplx *row = (cplx *)malloc(sizeof(cplx) * K);
        int64_t lo = n * th / tn, hi = n * (th + 1) / tn;
        for (int64_t i = lo; i < hi; ++i) {
            basis_row(P, Q, M, u, n, i, row);
            for (int a = 0; a < K; ++a) {
                cplx ca = conj(row[a]);
                for (int c2 = 0; c2 < K; ++c2) accG[(size_t)a * K + c2] += ca * row[c2];
                if (t) accb[a] += ca * t[i];
            }
        }
        free(row);
    }
    cplx *G = (cplx *)G_;
    cplx *b = (cplx *)b_;
    for (size_t j = 0; j < per; ++j) {
        cplx s = 0.0;
        for (int th = 0; th < nt; ++th) s += part[(size_t)th * per + j];
        if (j < (size_t)K * K) G[j] = s;
        else if (b) b[j - (size_t)K * K] = s;
    }
    free(part);
    return OR_OK;
}

/*
 * Solve G h = b for Hermitian positive definite G (K x K, row-major) by the
 * textbook Cholesky factorisation G = L L^H, then L w = b and L^H h = w.
 * Returns OR_NOT_SPD if a pivot is not positive.
 */
int oracle_chol_solve(int K, const double *G_, const double *b_, double *h_)
{
    if (K <= 0 || !G_ || !b_ || !h_) return OR_BAD_ARG;
    const cplx *G = (const cplx *)G_;
    const cplx *b = (const cplx *)b_;
    cplx *h = (cplx *)h_;
    cplx *Lm = (cplx *)calloc((size_t)K * K, sizeof(cplx));
    cplx *w = (cplx *)calloc((size_t)K, sizeof(cplx));
    if (!Lm || !w) { free(Lm); free(w); return OR_BAD_ARG; }
    for (int j = 0; j < K; ++j) {
        double d = creal(G[(size_t)j * K + j]);
        for (int k = 0; k < j; ++k) {
            cplx l = Lm[(size_t)j * K + k];
            d -= creal(l * conj(l));
        }
        if (!(d > 0.0)) { free(Lm); free(w); return OR_NOT_SPD; }
        double ljj = sqrt(d);
        Lm[(size_t)j * K + j] = ljj;
        for (int i = j + 1; i < K; ++i) {
            cplx s = G[(size_t)i * K + j];
            for (int k = 0; k < j; ++k) s -= Lm[(size_t)i * K + k] * conj(Lm[(size_t)j * K + k]);
            Lm[(size_t)i * K + j] = s / ljj;
        }
    }
    for (int i = 0; i < K; ++i) {
        cplx s = b[i];
        for (int k = 0; k < i; ++k) s -= Lm[(size_t)i * K + k] * w[k];
        w[i] = s / Lm[(size_t)i * K + i];
    }
    for (int i = K - 1; i >= 0; --i) {
        cplx s = w[i];
        for (int k = i + 1; k < K; ++k) s -= conj(Lm[(size_t)k * K + i]) * h[k];
        h[i] = s / creal(Lm[(size_t)i * K + i]);
    }
    free(Lm);
    free(w);
    return OR_OK;
}

/* Number of threads an OpenMP region would use for the given request. */
int oracle_threads(int nthreads) { return nthreads_used(nthreads); }
