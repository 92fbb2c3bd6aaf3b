"""What the KKT residual of a soft-margin SVM dual point implies about its
objective and its primal w (Sec. 3.2, eq. svm: min f(a) = 1/2 a^T Q a - e^T a
with Q = Z Z^T, s.t. y^T a = 0, 0 <= a <= C).  The dual point a is not
unique, so tests compare the quantities these bounds control.

Let v = Q a - e - mu y and let r_i be the per-coordinate residual (|v_i| if
0 < a_i < C, max(-v_i, 0) at a_i = 0, max(v_i, 0) at a_i = C).  For a box-
feasible a and any optimal a* (y^T a* = 0), convexity gives

    f(a) - f*  <=  grad f(a)^T (a - a*)  =  v^T (a - a*) + mu y^T a
               <=  C sum_i r_i + |mu| |y^T a|,

since each v_i (a_i - a*_i) <= C r_i.  The exact KKT conditions at a* give
grad f(a*)^T (a - a*) >= mu* y^T a, so f(a) - f* >= -|mu*| |y^T a|, and,
because f is quadratic, f(a) - f* = grad f(a*)^T (a - a*) + 1/2 ||w - w*||^2
with w = Z^T a, hence

    1/2 ||w - w*||^2  <=  C sum_i r_i + (|mu| + |mu*|) |y^T a|.

mu* is estimated by the larger |mu| of the two points compared; the bounds
below use (|mu| + |mu*|) <= 2 max(|mu|, |mu_ref|) in both places.
"""
import numpy as np

from oracle import rac_oracle as O


def point(inst, a, C=1.0):
    """(objective, w, C sum_i r_i, |y^T a|, mu) of the dual point a; mu is the
    oracle KKT measure's minimising multiplier."""
    P = O.problem_from_instance(inst, dense_H=False)
    mu = O.kkt(P, a)["mu"]
    r = O._stationarity_vec(P, a, P.grad(a), mu)
    w = inst.A @ a
    obj = 0.5 * float(w @ w) - float(a.sum())
    return obj, w, C * float(r.sum()), abs(float(inst.E[0] @ a)), mu


def check(inst, a, a_ref, C=1.0):
    """Objective gap and w distance between a and a_ref against the sum of
    both points' bounds.  Returns (gap, gap_bound, wdist, w_bound)."""
    obj, w, rs, eps, mu = point(inst, a, C)
    obj_r, w_r, rs_r, eps_r, mu_r = point(inst, a_ref, C)
    ms = 2.0 * max(abs(mu), abs(mu_r))
    b1, b2 = rs + ms * eps, rs_r + ms * eps_r
    gap = abs(obj - obj_r)
    wdist = float(np.linalg.norm(w - w_r))
    # rounding of the two objective and w evaluations themselves
    fl = 1e-12 * max(1.0, abs(obj_r))
    return gap, b1 + b2 + fl, wdist, np.sqrt(2 * b1) + np.sqrt(2 * b2) + 1e-12 * max(
        1.0, float(np.linalg.norm(w_r)))


def check_q(Q, y, a, a_ref, C=1.0):
    """check() for a dual given by its matrix Q (a kernel SVM): the same
    bounds, with ||w - w*||^2 = (a - a*)^T Q (a - a*) in feature space.
    Returns (gap, gap_bound, wdist, w_bound)."""
    def pt(v):
        P = O.Problem(H=Q, q=-np.ones(len(v)), phi="box", lo=0.0, hi=C,
                      E=np.asarray(y, dtype=np.float64).reshape(1, -1), d=np.zeros(1))
        mu = O.kkt(P, v)["mu"]
        r = O._stationarity_vec(P, v, P.grad(v), mu)
        return 0.5 * float(v @ Q @ v) - float(v.sum()), C * float(r.sum()), abs(float(y @ v)), mu
    obj, rs, eps, mu = pt(a)
    obj_r, rs_r, eps_r, mu_r = pt(a_ref)
    ms = 2.0 * max(abs(mu), abs(mu_r))
    b1, b2 = rs + ms * eps, rs_r + ms * eps_r
    dlt = a - a_ref
    wdist = float(np.sqrt(max(0.0, float(dlt @ Q @ dlt))))
    fl = 1e-12 * max(1.0, abs(obj_r))
    return abs(obj - obj_r), b1 + b2 + fl, wdist, np.sqrt(2 * b1) + np.sqrt(2 * b2) + 1e-9
