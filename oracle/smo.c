/*
 * Sequential minimal optimisation for the soft-margin SVM dual, part of the
 * FP64 oracle.  TEST INFRASTRUCTURE ONLY: called from oracle/rac_oracle.py,
 * never from the product path.  It is an independent algorithm (not
 * RAC-MBADMM) that pins converged SVM duals (Sec. 3.2, eq. svm):
 *
 *   minimise 1/2 a^T Q a - e^T a   s.t.  y^T a = 0,  0 <= a <= C.
 *
 * Each step changes one pair (i, j) along the feasible direction
 * y_i d_i = -y_j d_j by the exact line minimum, clipped to the box, and
 * updates the gradient grad = Q a - e with the two rows of Q.  With
 * yg_k = -y_k grad_k, the up set holds k with (y_k > 0, a_k < C) or
 * (y_k < 0, a_k > 0), the low set k with (y_k > 0, a_k > 0) or
 * (y_k < 0, a_k < C); a is optimal when max_up yg <= min_low yg, and the run
 * stops when max_up yg - min_low yg <= tol.
 *
 * The pair is chosen with second-order information (Fan, Chen and Lin, "Working
 * set selection using second order information for training support vector
 * machines", JMLR 2005): i maximises yg over the up set; j, among low-set
 * indices with yg_j < yg_i, maximises the objective decrease of the
 * unclipped pair step, (yg_i - yg_j)^2 / q_ij with
 * q_ij = Q_ii + Q_jj - 2 y_i y_j Q_ij (a small constant where q_ij <= 0).
 * The numpy smo_svm of rac_oracle.py picks j as the plain minimum of yg (the
 * maximal violating pair); both reach the same optimum, this one in far fewer
 * steps, so that duals with N ~ 10^4 finish in seconds.
 * Q is N x N, symmetric, row-major.  Returns the steps taken, or -1 if
 * max_iter was reached.
 */
#include <stdint.h>
#include <stdlib.h>

int64_t smo_svm(int64_t N, const double *Q, const double *y, double C, double *a, double tol,
                int64_t max_iter)
{
    const double tau = 1e-12;
    int64_t it;
    /* grad = Q a - e; a starts at zero */
    double *grad = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!grad) return -1;
    for (int64_t k = 0; k < N; ++k) {
        a[k] = 0.0;
        grad[k] = -1.0;
    }
    for (it = 0; it < max_iter; ++it) {
        int64_t i = -1;
        double gi = 0.0, gmin = 0.0;
        int have_low = 0;
        for (int64_t k = 0; k < N; ++k) {
            const double yg = -y[k] * grad[k];
            const int up = (y[k] > 0 && a[k] < C) || (y[k] < 0 && a[k] > 0);
            const int low = (y[k] > 0 && a[k] > 0) || (y[k] < 0 && a[k] < C);
            if (up && (i < 0 || yg > gi)) { i = k; gi = yg; }
            if (low && (!have_low || yg < gmin)) { gmin = yg; have_low = 1; }
        }
        if (i < 0 || !have_low || gi - gmin <= tol) break;
        const double *Qi = Q + i * N;
        int64_t j = -1;
        double best = 0.0;
        for (int64_t k = 0; k < N; ++k) {
            const int low = (y[k] > 0 && a[k] > 0) || (y[k] < 0 && a[k] < C);
            if (!low) continue;
            const double yg = -y[k] * grad[k];
            const double bk = gi - yg;
            if (bk <= 0.0) continue;
            double qk = Qi[i] + Q[k * N + k] - 2.0 * y[i] * y[k] * Qi[k];
            if (qk <= 0.0) qk = tau;
            const double dec = bk * bk / qk;
            if (j < 0 || dec > best) { j = k; best = dec; }
        }
        if (j < 0) break;
        const double *Qj = Q + j * N;
        const double gj = -y[j] * grad[j];
        double quad = Qi[i] + Qj[j] - 2.0 * y[i] * y[j] * Qi[j];
        if (quad <= 0.0) quad = tau;
        double t = (gi - gj) / quad;
        const double ti = y[i] > 0 ? C - a[i] : a[i];
        const double tj = y[j] > 0 ? a[j] : C - a[j];
        if (ti < t) t = ti;
        if (tj < t) t = tj;
        const double di = y[i] * t, dj = -y[j] * t;
        a[i] += di;
        a[j] += dj;
        for (int64_t k = 0; k < N; ++k) grad[k] += Qi[k] * di + Qj[k] * dj;
    }
    free(grad);
    return it < max_iter ? it : -1;
}
