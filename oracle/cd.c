/*
 * Coordinate descent for the Elastic-Net family, part of the FP64 oracle.
 * TEST INFRASTRUCTURE ONLY: called from oracle/rac_oracle.py, never from the
 * product path.  It is an independent algorithm (not RAC-MBADMM) used to pin
 * converged solutions:
 *
 *   minimise 1/2 ||A x - b||^2 + c^T x + lam1 ||x||_1 + lam2/2 ||x||^2
 *
 * Each coordinate step minimises the objective exactly in x_j with the others
 * fixed.  With g_j = A_j^T r + c_j (r = A x - b) and a_j = ||A_j||^2 the
 * one-dimensional optimality condition gives
 *   x_j <- soft(a_j x_j - g_j, lam1) / (a_j + lam2),  soft(u, t) = sign(u) max(|u| - t, 0).
 * Full cycles alternate with cycles over the current nonzeros; the run stops
 * when the stationarity residual (recomputed from an exact r) is <= tol
 * relative to max(1, ||c - A^T b||_inf).  A is column-major with leading
 * dimension lda.  Returns the number of cycles, or -1 if max_passes is hit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double soft(double u, double t)
{
    if (u > t) return u - t;
    if (u < -t) return u + t;
    return 0.0;
}

static double dot(int64_t m, const double *a, const double *r)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += a[i] * r[i];
    return s;
}

static void exact_residual(int64_t m, int64_t n, const double *A, int64_t lda,
                           const double *b, const double *x, double *r)
{
    for (int64_t i = 0; i < m; ++i) r[i] = -b[i];
    for (int64_t j = 0; j < n; ++j) {
        if (x[j] == 0.0) continue;
        const double *aj = A + j * lda;
        for (int64_t i = 0; i < m; ++i) r[i] += aj[i] * x[j];
    }
}

static double stationarity(int64_t m, int64_t n, const double *A, int64_t lda,
                           const double *c, double lam1, double lam2,
                           const double *x, const double *r)
{
    double worst = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double v = dot(m, A + j * lda, r) + c[j];
        double s;
        if (x[j] != 0.0) {
            s = fabs(v + lam2 * x[j] + lam1 * (x[j] > 0 ? 1.0 : -1.0));
        } else {
            s = fabs(v) - lam1;
            if (s < 0.0) s = 0.0;
        }
        if (s > worst) worst = s;
    }
    return worst;
}

static double update(int64_t m, const double *aj, double ajj, double cj,
                     double lam1, double lam2, double *xj, double *r)
{
    if (ajj + lam2 <= 0.0) return 0.0;
    double g = dot(m, aj, r) + cj;
    double xn = soft(ajj * (*xj) - g, lam1) / (ajj + lam2);
    double dx = xn - *xj;
    if (dx != 0.0) {
        for (int64_t i = 0; i < m; ++i) r[i] += aj[i] * dx;
        *xj = xn;
    }
    return fabs(dx);
}

int64_t cd_enet(int64_t m, int64_t n, const double *A, int64_t lda, const double *b,
                const double *c, double lam1, double lam2, double *x, double tol,
                int64_t max_passes)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *ajj = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !ajj) { free(r); free(ajj); return -1; }
    double scale = 1.0;
    for (int64_t j = 0; j < n; ++j) {
        const double *aj = A + j * lda;
        ajj[j] = dot(m, aj, aj);
        double q = fabs(c[j] - dot(m, aj, b));
        if (q > scale) scale = q;
    }
    exact_residual(m, n, A, lda, b, x, r);
    int64_t passes = 0;
    while (passes < max_passes) {
        /* one full cycle */
        for (int64_t j = 0; j < n; ++j)
            update(m, A + j * lda, ajj[j], c[j], lam1, lam2, &x[j], r);
        ++passes;
        /* cycles over the nonzeros until they settle */
        for (int inner = 0; inner < 1000 && passes < max_passes; ++inner) {
            double big = 0.0, xmax = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (x[j] == 0.0) continue;
                double d = update(m, A + j * lda, ajj[j], c[j], lam1, lam2, &x[j], r);
                if (d > big) big = d;
                if (fabs(x[j]) > xmax) xmax = fabs(x[j]);
            }
            ++passes;
            if (big <= 1e-3 * tol * (xmax > 1.0 ? xmax : 1.0)) break;
        }
        exact_residual(m, n, A, lda, b, x, r);
        if (stationarity(m, n, A, lda, c, lam1, lam2, x, r) <= tol * scale) {
            free(r); free(ajj);
            return passes;
        }
    }
    free(r); free(ajj);
    return -1;
}
