/*
 * ORACLE for the signature-kernel schemes of "Numerical Schemes for Signature Kernels"
 * (Cass, Piatti, Pei).  TEST INFRASTRUCTURE ONLY: a plain, slow FP64 CPU restatement of the
 * paper's definitions, used by the test suite, the smoke check and the benchmark's CPU
 * baseline.  The product path never links, loads or calls it, and it shares no code, table or
 * helper with the CUDA library.
 *
 * Contents
 *   sko_scheme        one pair, any scheme: FD1 / FD2 (Definition "dyadic scheme" and eq.
 *                     (secondexplicitscheme), Section 2), polynomial approximation (Definition
 *                     "def:polyapproxscheme", Section 3.2), polynomial interpolation (Definition
 *                     "def:polyinterpscheme", Section 3.3), implicit FD (Remark "higherfd");
 *                     all with dyadic refinement.
 *   sko_pairs         many pairs over ragged concatenated paths, split over POSIX threads.
 *   sko_grad_entry    d k / d x[p][c] (or y) by the complex step on the same scheme code.
 *   sko_sig_trunc     the level-n truncated signature kernel sum_k <S_k(x), S_k(y)> by brute
 *                     force (Definition 1.1 with Chen's identity), the paper's accuracy benchmark
 *                     at level 21 (Section 4).
 *   sko_mmd2*         biased / unbiased MMD^2 from the three Gram blocks and its complex-step
 *                     derivative with respect to one input coordinate.
 *
 * Parity status: every function is pinned by tests in tests/test_oracle_*.py (closed forms,
 * brute-force signatures, library Bessel functions, convergence orders, invariants).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* Uniform partition 0 = s_0 < ... < s_l = 1.  The experiments never state the partition; every
 * scheme depends on it only through C_ij (s_{i+1} - s_i)(t_{j+1} - t_j) = <dx_i, dy_j>. */
static double* uniform_grid_(int64_t L) {
    double* s = (double*)malloc(sizeof(double) * (size_t)L);
    for (int64_t i = 0; i < L; ++i) s[i] = (L > 1) ? (double)i / (double)(L - 1) : 0.0;
    return s;
}

#define REAL double
#define FN(name) name##_r
#define MAG(v) fabs(v)
#include "oracle_schemes.h"
#undef REAL
#undef FN
#undef MAG

#define REAL double complex
#define FN(name) name##_c
#define MAG(v) cabs(v)
#include "oracle_schemes.h"
#undef REAL
#undef FN
#undef MAG

/* ----------------------------------------------------------------------------------------- */
/* One pair.  x: [Lx][d], y: [Ly][d] row-major points; s, t: optional partitions (NULL =       */
/* uniform on [0, 1]).  scheme: 0 FD1, 1 FD2, 2 approximation, 3 interpolation, 4 implicit FD. */
/* ----------------------------------------------------------------------------------------- */
double sko_scheme(int scheme, const double* x, int64_t Lx, const double* y, int64_t Ly, int d,
                  int N, int lam, const double* s, const double* t) {
    return scheme_r(scheme, x, Lx, y, Ly, d, N, lam, s, t);
}

/* ----------------------------------------------------------------------------------------- */
/* Many pairs.  X: concatenated points with xoff[nx+1] (row offsets), same for Y; the k-th     */
/* pair is (pa[k], pb[k]).  Pairs are split over nthreads POSIX threads (0 = all cores).       */
/* ----------------------------------------------------------------------------------------- */
typedef struct {
    int scheme, d, N, lam;
    const double *X, *Y;
    const int64_t *xoff, *yoff, *pa, *pb;
    int64_t npairs, first, stride;
    double* out;
} pairs_job_;

static void* pairs_worker_(void* arg) {
    pairs_job_* j = (pairs_job_*)arg;
    for (int64_t k = j->first; k < j->npairs; k += j->stride) {
        int64_t a = j->pa[k], b = j->pb[k];
        const double* x = j->X + j->xoff[a] * j->d;
        const double* y = j->Y + j->yoff[b] * j->d;
        j->out[k] = scheme_r(j->scheme, x, j->xoff[a + 1] - j->xoff[a], y, j->yoff[b + 1] - j->yoff[b],
                             j->d, j->N, j->lam, NULL, NULL);
    }
    return NULL;
}

int sko_pairs(int scheme, const double* X, const int64_t* xoff, const double* Y, const int64_t* yoff,
              int d, const int64_t* pa, const int64_t* pb, int64_t npairs, int N, int lam, int nthreads,
              double* out) {
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    pthread_t th[512];
    pairs_job_ jobs[512];
    for (int t = 0; t < nthreads; ++t) {
        pairs_job_ jb = {scheme, d, N, lam, X, Y, xoff, yoff, pa, pb, npairs, t, nthreads, out};
        jobs[t] = jb;
        pthread_create(&th[t], NULL, pairs_worker_, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return nthreads;
}

/* ----------------------------------------------------------------------------------------- */
/* Derivative of the scheme output with respect to one input coordinate, by the complex step: */
/* k(x + i h e_{p,c}) = k(x) + i h dk/dx_{p,c} + O(h^2), so Im(.)/h is exact to rounding for   */
/* h = 1e-30.  side 0 perturbs x[p][c], side 1 perturbs y[p][c].                                */
/* ----------------------------------------------------------------------------------------- */
static double complex* to_complex_(const double* v, int64_t n) {
    double complex* z = (double complex*)malloc(sizeof(double complex) * (size_t)n);
    for (int64_t k = 0; k < n; ++k) z[k] = v[k];
    return z;
}

double sko_grad_entry(int scheme, const double* x, int64_t Lx, const double* y, int64_t Ly, int d,
                      int N, int lam, int side, int64_t p, int c) {
    const double h = 1e-30;
    double complex* xc = to_complex_(x, Lx * d);
    double complex* yc = to_complex_(y, Ly * d);
    if (side == 0) xc[p * d + c] += I * h;
    else yc[p * d + c] += I * h;
    double complex k = scheme_c(scheme, xc, Lx, yc, Ly, d, N, lam, NULL, NULL);
    free(xc);
    free(yc);
    return cimag(k) / h;
}

/* Full gradients of one pair: gx[Lx][d] = dk/dx, gy[Ly][d] = dk/dy (either may be NULL); the
 * coordinates are split over nthreads POSIX threads (0 = all cores). */
typedef struct {
    int scheme, d, N, lam;
    const double *x, *y;
    int64_t Lx, Ly, first, stride;
    double *gx, *gy;
} grad_job_;

static void* grad_worker_(void* arg) {
    grad_job_* j = (grad_job_*)arg;
    int64_t nx = j->gx ? j->Lx * j->d : 0, ny = j->gy ? j->Ly * j->d : 0;
    for (int64_t q = j->first; q < nx + ny; q += j->stride) {
        if (q < nx)
            j->gx[q] = sko_grad_entry(j->scheme, j->x, j->Lx, j->y, j->Ly, j->d, j->N, j->lam, 0, q / j->d,
                                      (int)(q % j->d));
        else
            j->gy[q - nx] = sko_grad_entry(j->scheme, j->x, j->Lx, j->y, j->Ly, j->d, j->N, j->lam, 1,
                                           (q - nx) / j->d, (int)((q - nx) % j->d));
    }
    return NULL;
}

void sko_grad_pair(int scheme, const double* x, int64_t Lx, const double* y, int64_t Ly, int d, int N,
                   int lam, double* gx, double* gy, int nthreads) {
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    pthread_t th[512];
    grad_job_ jobs[512];
    for (int t = 0; t < nthreads; ++t) {
        grad_job_ jb = {scheme, d, N, lam, x, y, Lx, Ly, t, nthreads, gx, gy};
        jobs[t] = jb;
        pthread_create(&th[t], NULL, grad_worker_, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ----------------------------------------------------------------------------------------- */
/* Truncated signature kernel by brute force.  S(x) of a piecewise-linear path is the ordered   */
/* product of the segment exponentials exp(dx_i) = sum_k dx_i^{(x)k} / k! (Chen's identity for */
/* the signature of Definition 1.1); level n of S has d^n entries, index i_1 ... i_n in base d. */
/* Returns sum_{n=0..level} <S_n(x), S_n(y)> with the Hilbert-Schmidt inner product.           */
/* ----------------------------------------------------------------------------------------- */
static int64_t ipow_i64_(int64_t b, int e) {
    int64_t v = 1;
    for (int k = 0; k < e; ++k) v *= b;
    return v;
}

static double** signature_(const double* x, int64_t L, int d, int level) {
    double** S = (double**)malloc(sizeof(double*) * (size_t)(level + 1));
    double** E = (double**)malloc(sizeof(double*) * (size_t)(level + 1));
    for (int n = 0; n <= level; ++n) {
        S[n] = (double*)calloc((size_t)ipow_i64_(d, n), sizeof(double));
        E[n] = (double*)calloc((size_t)ipow_i64_(d, n), sizeof(double));
    }
    S[0][0] = 1.0;
    E[0][0] = 1.0;
    for (int64_t i = 0; i + 1 < L; ++i) {
        const double* a = x + i * d;
        const double* b = x + (i + 1) * d;
        /* E_k = dx^{(x)k} / k!, built as E_k = (E_{k-1} (x) dx) / k. */
        for (int k = 1; k <= level; ++k) {
            int64_t nprev = ipow_i64_(d, k - 1);
            for (int64_t u = 0; u < nprev; ++u)
                for (int c = 0; c < d; ++c) E[k][u * d + c] = E[k - 1][u] * (b[c] - a[c]) / (double)k;
        }
        /* S_n <- sum_{k=0..n} S_{n-k} (x) E_k, from the top level down so that every S_{n-k}
         * with k >= 1 read on the right is still the old value. */
        for (int n = level; n >= 1; --n) {
            for (int k = 1; k <= n; ++k) {
                int64_t nl = ipow_i64_(d, n - k), nr = ipow_i64_(d, k);
                for (int64_t u = 0; u < nl; ++u) {
                    double su = S[n - k][u];
                    if (su == 0.0) continue;
                    for (int64_t v = 0; v < nr; ++v) S[n][u * nr + v] += su * E[k][v];
                }
            }
        }
    }
    for (int n = 0; n <= level; ++n) free(E[n]);
    free(E);
    return S;
}

double sko_sig_trunc(const double* x, int64_t Lx, const double* y, int64_t Ly, int d, int level) {
    double** Sx = signature_(x, Lx, d, level);
    double** Sy = signature_(y, Ly, d, level);
    double k = 0.0;
    for (int n = 0; n <= level; ++n) {
        int64_t sz = ipow_i64_(d, n);
        double acc = 0.0;
        for (int64_t u = 0; u < sz; ++u) acc += Sx[n][u] * Sy[n][u];
        k += acc;
        free(Sx[n]);
        free(Sy[n]);
    }
    free(Sx);
    free(Sy);
    return k;
}

/* Level-n signature tensor of one path (for direct tests of the brute-force signature). */
void sko_signature_level(const double* x, int64_t L, int d, int level, double* out) {
    double** S = signature_(x, L, d, level);
    memcpy(out, S[level], sizeof(double) * (size_t)ipow_i64_(d, level));
    for (int n = 0; n <= level; ++n) free(S[n]);
    free(S);
}

/* ----------------------------------------------------------------------------------------- */
/* MMD^2 between path sets A (na paths) and B (nb paths), all of length L, d coordinates.      */
/* The paper names MMD (Sections 1 and 4) without a formula; this is the standard estimator:   */
/* biased:   mean(K_AA) + mean(K_BB) - 2 mean(K_AB)                                              */
/* unbiased: K_AA, K_BB means over off-diagonal entries only.                                   */
/* ----------------------------------------------------------------------------------------- */
static double complex mmd2_c_(int scheme, const double complex* A, int64_t na, const double complex* B,
                              int64_t nb, int64_t L, int d, int N, int lam, int unbiased) {
    double complex saa = 0.0, sbb = 0.0, sab = 0.0;
    for (int64_t a = 0; a < na; ++a)
        for (int64_t b = 0; b < na; ++b) {
            if (unbiased && a == b) continue;
            saa += scheme_c(scheme, A + a * L * d, L, A + b * L * d, L, d, N, lam, NULL, NULL);
        }
    for (int64_t a = 0; a < nb; ++a)
        for (int64_t b = 0; b < nb; ++b) {
            if (unbiased && a == b) continue;
            sbb += scheme_c(scheme, B + a * L * d, L, B + b * L * d, L, d, N, lam, NULL, NULL);
        }
    for (int64_t a = 0; a < na; ++a)
        for (int64_t b = 0; b < nb; ++b)
            sab += scheme_c(scheme, A + a * L * d, L, B + b * L * d, L, d, N, lam, NULL, NULL);
    double daa = unbiased ? (double)(na * (na - 1)) : (double)(na * na);
    double dbb = unbiased ? (double)(nb * (nb - 1)) : (double)(nb * nb);
    return saa / daa + sbb / dbb - 2.0 * sab / ((double)na * (double)nb);
}

double sko_mmd2(int scheme, const double* A, int64_t na, const double* B, int64_t nb, int64_t L, int d,
                int N, int lam, int unbiased) {
    double complex* Ac = to_complex_(A, na * L * d);
    double complex* Bc = to_complex_(B, nb * L * d);
    double v = creal(mmd2_c_(scheme, Ac, na, Bc, nb, L, d, N, lam, unbiased));
    free(Ac);
    free(Bc);
    return v;
}

/* d MMD^2 / d A[path][p][c] (side 0) or B[path][p][c] (side 1), by the complex step through    */
/* every Gram entry.                                                                             */
double sko_mmd2_grad_entry(int scheme, const double* A, int64_t na, const double* B, int64_t nb,
                           int64_t L, int d, int N, int lam, int unbiased, int side, int64_t path,
                           int64_t p, int c) {
    const double h = 1e-30;
    double complex* Ac = to_complex_(A, na * L * d);
    double complex* Bc = to_complex_(B, nb * L * d);
    if (side == 0) Ac[(path * L + p) * d + c] += I * h;
    else Bc[(path * L + p) * d + c] += I * h;
    double v = cimag(mmd2_c_(scheme, Ac, na, Bc, nb, L, d, N, lam, unbiased)) / h;
    free(Ac);
    free(Bc);
    return v;
}
