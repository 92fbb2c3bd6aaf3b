"""FP64 CPU oracle for RAC-MBADMM (Zhu, Mihic, Ye, arXiv:1907.01995).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg call it.
It shares no code with the CUDA path (the two meet only in the seeded input
generators of the `synth` package, which hold none of the method's arithmetic).

What is here, each piece written from the paper's text:

* Philox4x64-10, the counter-based generator of Salmon, Moraes, Dror and Shaw
  ("Parallel random numbers: as easy as 1, 2, 3", SC'11), used to draw the
  random assembly.  Pinned to numpy's independent Philox bit generator.
* Random assembly of the n primal coordinates into p blocks (Sec. 1,
  eq. RAC-ADDM, "randomly (without replacement) assemble"; Sec. 2, sigma =
  [sigma_1, ..., sigma_p]), and the RP-MBADMM variant of Sec. 1 (a fixed
  partition visited in a random order).
* The block argmin of the augmented Lagrangian (Sec. 1, eq. lagrangian and
  eq. RAC-ADDM), literally with the box kept in the block (an exact
  bound-constrained QP per block, for phi = box), and in the split form the paper uses for the Elastic-Net
  (Sec. 3.1: x - z = 0 with penalty gamma and dual xi; x partitioned into RAC
  blocks, z solved as one block in closed form), with an optional single
  coupling row E x = d (penalty beta, dual mu) for the SVM dual (Sec. 3.2,
  eq. svm, y^T a = 0).
* The paper's un-split iteration for the linearly constrained QP (Sec. 2,
  eq. lcqp) and its exact linear-map view z^{k+1} = M_sigma z^k +
  Lbar_sigma^{-1} bbar (Sec. 2), plus Q = E_sigma[L_sigma^{-1}] (Lemma 2.3).
* KKT measures for the composite and box-constrained problems (the paper
  states none; the definitions below are this project's).
* Independent solvers that pin results without reference to the method:
  normal equations, coordinate descent (C helper, cd.c), brute-force
  active-set enumeration for LASSO/EN and for the SVM dual, and SMO for the
  SVM dual.

Parity status: every function is pinned by tests/test_oracle_*.py; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import dataclasses
import itertools
import math
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np
from scipy.linalg import cho_factor, cho_solve, solve_triangular

# ---------------------------------------------------------------------------
# Philox4x64-10 (Salmon et al., SC'11, Sec. 4: the Philox S-box, N=4, W=64,
# ten rounds).  Each round multiplies counter words 0 and 2 by fixed odd
# constants, takes the 128-bit products apart into high and low halves and
# mixes them with the other two words and the round key; the key is bumped by
# two Weyl constants between rounds.
# ---------------------------------------------------------------------------
PHILOX_M0 = np.uint64(0xD2E7470EE14C6C93)
PHILOX_M1 = np.uint64(0xCA5A826395121157)
PHILOX_W0 = np.uint64(0x9E3779B97F4A7C15)
PHILOX_W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo64(a: np.ndarray, b: np.uint64):
    """Full 64x64 -> 128-bit product of uint64 arrays, as (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.uint64(b)
    a_lo, a_hi = a & _LO32, a >> _S32
    b_lo, b_hi = b & _LO32, b >> _S32
    ll = a_lo * b_lo
    hl = a_hi * b_lo
    lh = a_lo * b_hi
    hh = a_hi * b_hi
    cross = (ll >> _S32) + (hl & _LO32) + (lh & _LO32)
    lo = (ll & _LO32) | (cross << _S32)
    hi = hh + (hl >> _S32) + (lh >> _S32) + (cross >> _S32)
    return hi, lo


def philox4x64_10(ctr: Sequence[np.ndarray], key: Sequence[int]):
    """Philox4x64 with 10 rounds on counter words (c0, c1, c2, c3) (uint64
    arrays, broadcast together) and key (k0, k1).  Returns four uint64 arrays."""
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in ctr)
        c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
        k0, k1 = np.uint64(key[0]), np.uint64(key[1])
        for rnd in range(10):
            if rnd > 0:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            hi0, lo0 = _mulhilo64(c0, PHILOX_M0)
            hi1, lo1 = _mulhilo64(c2, PHILOX_M1)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


# ---------------------------------------------------------------------------
# Random assembly (Sec. 1, eq. RAC-ADDM; Sec. 2).  This project's reading:
# sweep k draws, for every coordinate j, the 64-bit key word 0 of
# Philox4x64-10(counter = (j, k, 0, 0), key = (seed, 0)); sorting the keys in
# ascending order (ties by j) gives the permutation pi^k, and the blocks are
# consecutive slices of pi^k, the first (n mod p) of size ceil(n/p) and the
# rest of size floor(n/p) (the paper assumes p*s = n).
# ---------------------------------------------------------------------------
def assembly_keys(n: int, seed: int, sweep: int) -> np.ndarray:
    j = np.arange(n, dtype=np.uint64)
    w0, _, _, _ = philox4x64_10((j, np.uint64(sweep), np.uint64(0), np.uint64(0)),
                                (seed, 0))
    return w0


def random_permutation(n: int, seed: int, sweep: int) -> np.ndarray:
    keys = assembly_keys(n, seed, sweep)
    return np.argsort(keys, kind="stable").astype(np.int64)


def block_sizes(n: int, p: int) -> List[int]:
    if p < 1 or p > n:
        raise ValueError("need 1 <= p <= n")
    q, r = divmod(n, p)
    return [q + 1] * r + [q] * (p - r)


def blocks_from_permutation(perm: np.ndarray, p: int) -> List[np.ndarray]:
    out, o = [], 0
    for s in block_sizes(len(perm), p):
        out.append(np.asarray(perm[o:o + s], dtype=np.int64))
        o += s
    return out


def random_assembly(n: int, p: int, seed: int, sweep: int) -> List[np.ndarray]:
    return blocks_from_permutation(random_permutation(n, seed, sweep), p)


# RP-MBADMM (Sec. 1: blocks built by a predetermined rule and kept fixed, the
# block subproblems solved in a random order every iteration).  The rule here
# is the consecutive partition of 0..n-1 with the same block sizes as above;
# the order of sweep k is the Philox argsort of the p block indices.
def fixed_partition(n: int, p: int) -> List[np.ndarray]:
    return blocks_from_permutation(np.arange(n, dtype=np.int64), p)


def rp_order(p: int, seed: int, sweep: int) -> np.ndarray:
    return random_permutation(p, seed, sweep)


def rp_assembly(n: int, p: int, seed: int, sweep: int) -> List[np.ndarray]:
    blocks = fixed_partition(n, p)
    return [blocks[b] for b in rp_order(p, seed, sweep)]


# ---------------------------------------------------------------------------
# Problem: minimise 1/2 x^T H x + c^T x + sum_j phi(x_j)  s.t. E x = d
# (Sec. 1 eq. general_model with separable f = phi).  In data form H = A^T A
# and the linear term is c - A^T b (1/2 ||Ax - b||^2 + c^T x, constant dropped).
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    H: Optional[np.ndarray]       # n x n, symmetric PSD (None: data form without a dense H)
    q: np.ndarray                 # full linear term (c - A^T b in data form)
    phi: str = "none"             # none | l1l2 | box
    lam1: float = 0.0
    lam2: float = 0.0
    lo: float = 0.0
    hi: float = 0.0
    E: Optional[np.ndarray] = None
    d: Optional[np.ndarray] = None
    A: Optional[np.ndarray] = None
    b: Optional[np.ndarray] = None
    c: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return self.q.shape[0]

    def grad(self, x: np.ndarray) -> np.ndarray:
        """Gradient of the smooth part: H x + q, evaluated in data form as
        A^T (A x - b) + c when A is known (no explicit H product)."""
        if self.A is not None:
            return self.A.T @ (self.A @ x - self.b) + self.c
        return self.H @ x + self.q

    def objective(self, x: np.ndarray) -> float:
        if self.H is None:
            # data form: 1/2 x^T A^T A x + q^T x without the n x n product
            Ax = self.A @ x
            f = 0.5 * float(Ax @ Ax) + float(self.q @ x)
        else:
            f = 0.5 * float(x @ (self.H @ x)) + float(self.q @ x)
        if self.phi == "l1l2":
            f += self.lam1 * float(np.abs(x).sum()) + 0.5 * self.lam2 * float(x @ x)
        return f


def problem_from_data(A, b, phi="none", lam1=0.0, lam2=0.0, lo=0.0, hi=0.0,
                      c=None, E=None, d=None, dense_H=True) -> Problem:
    """dense_H=False leaves H = A^T A unformed (for n too large to hold an
    n x n matrix); the gradient, the objective and the KKT measure still work,
    the sweep and the linear-map functions need H."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[1]
    c = np.zeros(n) if c is None else np.asarray(c, dtype=np.float64)
    H = A.T @ A if dense_H else None
    q = c - A.T @ b
    return Problem(H=H, q=q, phi=phi, lam1=lam1, lam2=lam2, lo=lo, hi=hi,
                   E=None if E is None else np.asarray(E, dtype=np.float64).reshape(-1, n),
                   d=None if d is None else np.asarray(d, dtype=np.float64).reshape(-1),
                   A=A, b=b, c=c)


def problem_from_instance(inst, dense_H=True) -> Problem:
    """Read the attributes of a `synth` instance (duck-typed)."""
    return problem_from_data(inst.A, inst.b, inst.phi, inst.lam1, inst.lam2,
                             inst.lo, inst.hi, inst.c, inst.E, inst.d, dense_H=dense_H)


# ---------------------------------------------------------------------------
# z-block closed form (Sec. 3.1).  The paper writes
#   z*(i) = S(xi(i) - gamma x(i), lambda alpha) / ((1 - alpha) lambda + gamma)
# with S(a, b) = -(a - b) if b < |a|, a > 0;  -(a + b) if b < |a|, a <= 0;
# 0 if b >= |a|.  Here lambda alpha = lam1 and lambda (1 - alpha) = lam2.
# For the box the z-block is the projection of x - xi/gamma on [lo, hi]; with
# no penalty it is x - xi/gamma.
# ---------------------------------------------------------------------------
def paper_S(a, b):
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros_like(a)
    pos = (b < np.abs(a)) & (a > 0)
    neg = (b < np.abs(a)) & (a <= 0)
    out[pos] = -(a[pos] - b)
    out[neg] = -(a[neg] + b)
    return out


def z_block(P: Problem, x: np.ndarray, xi: np.ndarray, gamma: float) -> np.ndarray:
    if P.phi == "l1l2":
        return paper_S(xi - gamma * x, P.lam1) / (P.lam2 + gamma)
    if P.phi == "box":
        return np.clip(x - xi / gamma, P.lo, P.hi)
    return x - xi / gamma


# ---------------------------------------------------------------------------
# The split augmented Lagrangian (Sec. 3.1, eq. after eq. el_net, extended by
# the coupling row of eq. lagrangian):
#   L = 1/2 x^T H x + q^T x - xi^T (x - z) + gamma/2 ||x - z||^2 + phi(z)
#       - mu^T (E x - d) + beta/2 ||E x - d||^2
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class State:
    x: np.ndarray
    z: np.ndarray
    xi: np.ndarray
    mu: np.ndarray
    sweep: int = 0

    def copy(self) -> "State":
        return State(self.x.copy(), self.z.copy(), self.xi.copy(), self.mu.copy(),
                     self.sweep)


def initial_state(P: Problem, x0=None, xi0=None) -> State:
    n = P.n
    k = 0 if P.E is None else P.E.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    xi = np.zeros(n) if xi0 is None else np.array(xi0, dtype=np.float64)
    return State(x=x, z=x.copy(), xi=xi, mu=np.zeros(k))


def augmented_lagrangian(P: Problem, st: State, beta: float, gamma: float) -> float:
    """Value of the split augmented Lagrangian (phi(z) included)."""
    x, z = st.x, st.z
    val = 0.5 * float(x @ (P.H @ x)) + float(P.q @ x)
    val += -float(st.xi @ (x - z)) + 0.5 * gamma * float((x - z) @ (x - z))
    if P.phi == "l1l2":
        val += P.lam1 * float(np.abs(z).sum()) + 0.5 * P.lam2 * float(z @ z)
    if P.E is not None:
        res = P.E @ x - P.d
        val += -float(st.mu @ res) + 0.5 * beta * float(res @ res)
    return val


def block_argmin(P: Problem, st: State, S: np.ndarray, beta: float, gamma: float):
    """x_S <- argmin over x_S of the split augmented Lagrangian, all other
    variables fixed (one line of eq. RAC-ADDM).  The block problem is a
    strictly convex quadratic (Assumption 2.1 holds because of gamma I), so
    the minimiser solves K_S dx = -grad_S with
    K_S = H_SS + gamma I + beta E_S^T E_S."""
    x = st.x
    grad = P.H[S, :] @ x + P.q[S] - st.xi[S] + gamma * (x[S] - st.z[S])
    K = P.H[np.ix_(S, S)] + gamma * np.eye(len(S))
    if P.E is not None:
        ES = P.E[:, S]
        grad = grad + ES.T @ (beta * (P.E @ x - P.d) - st.mu)
        K = K + beta * ES.T @ ES
    cf = cho_factor(K, lower=True)
    x[S] = x[S] - cho_solve(cf, grad)


# ---------------------------------------------------------------------------
# The box kept inside the block.  Eq. RAC-ADDM restricts each block argmin to
# x_i in X_i; for the SVM dual (Sec. 3.2, eq. svm) X = [0, C]^n.  Read
# literally, a block step is then the bound-constrained quadratic
#   min { 1/2 d^T K d + r^T d : l <= d <= u },  d = x_S^new - x_S,
# with K = H_SS + beta E_S^T E_S (+ gamma I, an optional proximal term
# gamma/2 ||x_S - x_S^k||^2; gamma = 0 is the paper's step), r the gradient
# of the augmented Lagrangian at x restricted to S, l = lo - x_S <= 0 and
# u = hi - x_S >= 0.  There is no z-block and no xi in this reading.
# ---------------------------------------------------------------------------
def box_qp(K, r, l, u, tol=None, max_iter=None):
    """Exact minimiser of 1/2 d^T K d + r^T d over l <= d <= u (K symmetric
    positive definite, l <= 0 <= u) by the primal active-set method for convex
    QP (Nocedal and Wright, Numerical Optimization, Ch. 16, "active-set
    methods"), specialised to bounds: start at the feasible d = 0 with the
    bounds that hold there active; take the minimiser over the current face
    (a linear solve with the free rows and columns of K) as far as the first
    bound it would cross, which becomes active; at a face minimiser release
    the active bound whose multiplier (the gradient there) has the wrong sign
    by the most, or stop when none has.  Returns (d, state): state 0 free,
    1 at l, 2 at u; d equals l or u exactly where a bound is active."""
    K = np.asarray(K, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    s = r.shape[0]
    if tol is None:
        tol = 1e-13 * max(1.0, float(np.abs(r).max()) if s else 1.0)
    if max_iter is None:
        max_iter = 10 * s + 20
    d = np.zeros(s)
    state = np.zeros(s, dtype=np.int64)
    state[l == 0.0] = 1
    state[(u == 0.0) & (l < 0.0)] = 2
    for _ in range(max_iter):
        F = np.nonzero(state == 0)[0]
        g = K @ d + r
        step = np.zeros(s)
        if len(F):
            step[F] = np.linalg.solve(K[np.ix_(F, F)], -g[F])
        alpha, hit = 1.0, -1
        for j in F:
            if step[j] < 0.0 and d[j] + step[j] < l[j]:
                a = (l[j] - d[j]) / step[j]
            elif step[j] > 0.0 and d[j] + step[j] > u[j]:
                a = (u[j] - d[j]) / step[j]
            else:
                continue
            if a < alpha:
                alpha, hit = a, j
        d = d + alpha * step
        if hit >= 0:
            state[hit] = 1 if step[hit] < 0.0 else 2
            d[hit] = l[hit] if state[hit] == 1 else u[hit]
            continue
        g = K @ d + r
        viol = np.zeros(s)
        movable = u > l
        viol[(state == 1) & movable] = -g[(state == 1) & movable]
        viol[(state == 2) & movable] = g[(state == 2) & movable]
        j = int(np.argmax(viol)) if s else 0
        if s == 0 or viol[j] <= tol:
            d[state == 1] = l[state == 1]
            d[state == 2] = u[state == 2]
            return d, state
        state[j] = 0
    raise RuntimeError("box_qp: no convergence in %d iterations" % max_iter)


def block_argmin_box(P: Problem, st: State, S: np.ndarray, beta: float, gamma: float):
    """x_S <- argmin { L(x_S; others fixed) + gamma/2 ||x_S - x_S^k||^2 :
    lo <= x_S <= hi } (eq. RAC-ADDM with the box of eq. svm kept in the
    block); coordinates ending on a bound take its value exactly."""
    x = st.x
    grad = P.H[S, :] @ x + P.q[S]
    K = P.H[np.ix_(S, S)] + gamma * np.eye(len(S))
    if P.E is not None:
        ES = P.E[:, S]
        grad = grad + ES.T @ (beta * (P.E @ x - P.d) - st.mu)
        K = K + beta * ES.T @ ES
    d, state = box_qp(K, grad, P.lo - x[S], P.hi - x[S])
    xs = x[S] + d
    xs[state == 1] = P.lo
    xs[state == 2] = P.hi
    x[S] = xs


def sweep(P: Problem, st: State, p: int, seed: int, beta: float, gamma: float,
          blocks: Optional[List[np.ndarray]] = None, rp: bool = False,
          box_qp: bool = False) -> State:
    """One RAC-MBADMM iteration (eq. RAC-ADDM) in the split form of Sec. 3.1:
    random assembly, cyclic block argmins over the x-blocks, the z-block in
    closed form, then the multiplier ascent on both constraints.  rp=True is
    the RP-MBADMM iteration (Sec. 1): the fixed partition in a random order.
    box_qp=True (phi = box only) keeps the box in the block argmins instead
    of the split: gamma is then the proximal weight, z = x and xi stays 0."""
    if blocks is None:
        blocks = (rp_assembly if rp else random_assembly)(P.n, p, seed, st.sweep)
    if box_qp:
        if P.phi != "box":
            raise ValueError("box_qp needs phi = box")
        for S in blocks:
            block_argmin_box(P, st, S, beta, gamma)
        st.z = st.x.copy()
        if P.E is not None:
            st.mu = st.mu - beta * (P.E @ st.x - P.d)
        st.sweep += 1
        return st
    for S in blocks:
        block_argmin(P, st, S, beta, gamma)
    st.z = z_block(P, st.x, st.xi, gamma)
    st.xi = st.xi - gamma * (st.x - st.z)
    if P.E is not None:
        st.mu = st.mu - beta * (P.E @ st.x - P.d)
    st.sweep += 1
    return st


# ---------------------------------------------------------------------------
# KKT measures (the paper gives none; these are this project's definitions).
# v = H z + q - E^T mu.  Per coordinate:
#   none: |v_j|
#   l1l2: |v_j + lam2 z_j + lam1 sign z_j| if z_j != 0, else max(|v_j| - lam1, 0)
#   box : |v_j| strictly inside, max(-v_j, 0) at lo, max(v_j, 0) at hi
# stationarity = ||.||_inf / max(1, ||q||_inf)  (||q|| = ||grad at 0||)
# feasibility  = ||E z - d||_inf / max(1, ||z||_1)
# KKT = max(stationarity, feasibility).  With a coupling row and no mu given,
# mu minimises the stationarity term (a convex 1-D problem, ternary search).
# ---------------------------------------------------------------------------
def _stationarity_vec(P: Problem, z: np.ndarray, g: np.ndarray, mu) -> np.ndarray:
    v = g.copy()
    if P.E is not None:
        v = v - P.E.T @ np.atleast_1d(mu)
    if P.phi == "none":
        return np.abs(v)
    if P.phi == "l1l2":
        nz = z != 0.0
        r = np.maximum(np.abs(v) - P.lam1, 0.0)
        r[nz] = np.abs(v[nz] + P.lam2 * z[nz] + P.lam1 * np.sign(z[nz]))
        return r
    r = np.abs(v)
    at_lo = z <= P.lo
    at_hi = z >= P.hi
    r[at_lo] = np.maximum(-v[at_lo], 0.0)
    r[at_hi] = np.maximum(v[at_hi], 0.0)
    return r


def kkt(P: Problem, z: np.ndarray, mu=None) -> dict:
    g = P.grad(z)
    scale = max(1.0, float(np.abs(P.q).max()) if P.n else 1.0)
    feas = 0.0
    if P.E is not None:
        feas = float(np.abs(P.E @ z - P.d).max()) / max(1.0, float(np.abs(z).sum()))
        if mu is None:
            if P.E.shape[0] != 1:
                raise ValueError("mu minimisation implemented for one coupling row")
            f = lambda m: float(_stationarity_vec(P, z, g, m).max())
            lo_m, hi_m = -1.0, 1.0
            while f(lo_m) > f(0.5 * (lo_m + hi_m)) and lo_m > -1e12:
                lo_m *= 2.0
            while f(hi_m) > f(0.5 * (lo_m + hi_m)) and hi_m < 1e12:
                hi_m *= 2.0
            lo_m, hi_m = -max(abs(lo_m), abs(hi_m)), max(abs(lo_m), abs(hi_m))
            for _ in range(200):
                a = lo_m + (hi_m - lo_m) / 3.0
                bb = hi_m - (hi_m - lo_m) / 3.0
                if f(a) <= f(bb):
                    hi_m = bb
                else:
                    lo_m = a
            mu = 0.5 * (lo_m + hi_m)
    stat_vec = _stationarity_vec(P, z, g, mu if mu is not None else 0.0)
    stat = float(stat_vec.max()) / scale if P.n else 0.0
    return {"kkt": max(stat, feas), "stationarity": stat, "feasibility": feas,
            "mu": mu}


def solve(P: Problem, p: int, seed: int = 0, beta: float = 1.0, gamma: float = 1.0,
          tol: float = 1e-6, max_sweeps: int = 1000, check_every: int = 1,
          x0=None, xi0=None, record: bool = False, rp: bool = False,
          box_qp: bool = False):
    """Run sweeps from the initial state until KKT(z) <= tol or max_sweeps.
    Returns (state, info)."""
    st = initial_state(P, x0, xi0)
    hist = []
    k_val = kkt(P, st.z, st.mu if P.E is not None else None)["kkt"]
    while st.sweep < max_sweeps:
        sweep(P, st, p, seed, beta, gamma, rp=rp, box_qp=box_qp)
        if record:
            hist.append(st.copy())
        if st.sweep % check_every == 0 or st.sweep == max_sweeps:
            k_val = kkt(P, st.z, st.mu if P.E is not None else None)["kkt"]
            if k_val <= tol:
                break
    return st, {"sweeps": st.sweep, "kkt": k_val, "history": hist}


# ---------------------------------------------------------------------------
# The paper's un-split iteration for the linearly constrained QP (Sec. 2,
# eq. lcqp) with augmented Lagrangian eq. lagrangian (penalty beta), and its
# exact linear-map view (Sec. 2).
# ---------------------------------------------------------------------------
def sweep_lcqp(H, c, Aeq, beq, beta, x, y, blocks):
    """One iteration of eq. RAC-ADDM for eq. lcqp with the given assembly."""
    x = x.copy()
    for S in blocks:
        grad = H[S, :] @ x + c[S] - Aeq[:, S].T @ y + beta * Aeq[:, S].T @ (Aeq @ x - beq)
        K = H[np.ix_(S, S)] + beta * Aeq[:, S].T @ Aeq[:, S]
        x[S] = x[S] - np.linalg.solve(K, grad)
    y = y - beta * (Aeq @ x - beq)
    return x, y


def L_sigma(Sfull: np.ndarray, blocks: Sequence[np.ndarray]) -> np.ndarray:
    """(L_sigma)_{sigma_i, sigma_j} = (H + beta A^T A)_{sigma_i, sigma_j} for
    i >= j, zero otherwise (Sec. 2)."""
    L = np.zeros_like(Sfull)
    for i, Si in enumerate(blocks):
        for j in range(i + 1):
            Sj = blocks[j]
            L[np.ix_(Si, Sj)] = Sfull[np.ix_(Si, Sj)]
    return L


def linear_map(H, c, Aeq, beq, beta, blocks):
    """M_sigma = Lbar^{-1} Rbar and the offset Lbar^{-1} bbar (Sec. 2)."""
    n, mm = H.shape[0], Aeq.shape[0]
    Sfull = H + beta * Aeq.T @ Aeq
    L = L_sigma(Sfull, blocks)
    R = L - Sfull
    Lbar = np.block([[L, np.zeros((n, mm))], [beta * Aeq, np.eye(mm)]])
    Rbar = np.block([[R, Aeq.T], [np.zeros((mm, n)), np.eye(mm)]])
    bbar = np.concatenate([-c + beta * Aeq.T @ beq, beta * beq])
    M = np.linalg.solve(Lbar, Rbar)
    off = np.linalg.solve(Lbar, bbar)
    return M, off


def all_assemblies(n: int, p: int):
    """Every ordered partition sigma of {0..n-1} into p blocks of size n/p
    (the set Gamma(n, p) of Sec. 2), as lists of sorted index arrays."""
    s = n // p
    if s * p != n:
        raise ValueError("Gamma(n, p) is defined for p * s = n")
    seen = set()
    out = []
    for perm in itertools.permutations(range(n)):
        blocks = tuple(tuple(sorted(perm[i * s:(i + 1) * s])) for i in range(p))
        if blocks not in seen:
            seen.add(blocks)
            out.append([np.array(b_, dtype=np.int64) for b_ in blocks])
    return out


def expected_Q(H, Aeq, beta, n, p):
    """Q = E_sigma[L_sigma^{-1}] over the uniform assembly (Sec. 2)."""
    Sfull = H + beta * Aeq.T @ Aeq
    sig = all_assemblies(n, p)
    Q = np.zeros_like(Sfull)
    for blocks in sig:
        Q += np.linalg.inv(L_sigma(Sfull, blocks))
    return Q / len(sig), Sfull, len(sig)


# ---------------------------------------------------------------------------
# Independent solvers (no reference to RAC-MBADMM).
# ---------------------------------------------------------------------------
def normal_equations(A, b) -> np.ndarray:
    """Least squares by Cholesky of A^T A x = A^T b (full column rank)."""
    G = A.T @ A
    Lc = np.linalg.cholesky(G)
    y = solve_triangular(Lc, A.T @ b, lower=True)
    return solve_triangular(Lc.T, y, lower=False)


def enum_lasso(A, b, lam1, lam2=0.0, c=None) -> np.ndarray:
    """Brute-force active-set enumeration for min 1/2||Ax-b||^2 + c^T x +
    lam1 ||x||_1 + lam2/2 ||x||^2 (n <= 10): try every sign pattern in
    {-1, 0, +1}^n, solve the reduced stationarity system, keep the pattern
    whose solution is sign-consistent and satisfies |g_j| <= lam1 off it."""
    n = A.shape[1]
    c = np.zeros(n) if c is None else c
    G = A.T @ A
    r0 = A.T @ b - c
    found = []
    for signs in itertools.product((-1, 0, 1), repeat=n):
        s = np.array(signs, dtype=np.float64)
        F = np.nonzero(s)[0]
        x = np.zeros(n)
        if len(F):
            K = G[np.ix_(F, F)] + lam2 * np.eye(len(F))
            try:
                xf = np.linalg.solve(K, r0[F] - lam1 * s[F])
            except np.linalg.LinAlgError:
                continue
            if np.any(np.sign(xf) != s[F]) or np.any(xf == 0):
                continue
            x[F] = xf
        g = G @ x - r0
        off = np.setdiff1d(np.arange(n), F)
        if np.all(np.abs(g[off]) <= lam1 * (1 + 1e-12) + 1e-12):
            found.append(x)
    if not found:
        raise RuntimeError("no consistent sign pattern")
    return found[0]


def enum_svm(Q, y, C, e=None):
    """Brute force over {at 0, free, at C}^N for min 1/2 a^T Q a - e^T a
    s.t. y^T a = 0, 0 <= a <= C: solve the KKT system of the free set
    [[Q_FF, -y_F], [y_F^T, 0]] [a_F; mu] = [e_F - Q_FU C 1; -C y_U^T 1] and keep
    a feasible, sign-consistent pattern.  Returns (alpha, mu)."""
    N = Q.shape[0]
    e = np.ones(N) if e is None else e
    best = None
    for pat in itertools.product((0, 1, 2), repeat=N):
        pat = np.array(pat)
        F = np.nonzero(pat == 1)[0]
        U = np.nonzero(pat == 2)[0]
        Lw = np.nonzero(pat == 0)[0]
        a = np.zeros(N)
        a[U] = C
        nf = len(F)
        K = np.zeros((nf + 1, nf + 1))
        K[:nf, :nf] = Q[np.ix_(F, F)]
        K[:nf, nf] = -y[F]
        K[nf, :nf] = y[F]
        rhs = np.zeros(nf + 1)
        rhs[:nf] = e[F] - Q[np.ix_(F, U)] @ a[U]
        rhs[nf] = -float(y[U] @ a[U])
        try:
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            continue
        a[F] = sol[:nf]
        mu = sol[nf]
        tol = 1e-10
        if np.any(a[F] <= tol) or np.any(a[F] >= C - tol):
            continue
        v = Q @ a - e - mu * y
        if np.any(v[Lw] < -1e-9) or np.any(v[U] > 1e-9):
            continue
        if abs(float(y @ a)) > 1e-9:
            continue
        obj = 0.5 * float(a @ Q @ a) - float(e @ a)
        if best is None or obj < best[2] - 1e-12:
            best = (a, mu, obj)
    if best is None:
        raise RuntimeError("no KKT pattern found")
    return best[0], best[1]


def smo_svm(Q, y, C, tol=1e-10, max_iter=2_000_000):
    """Sequential minimal optimisation with the maximal-violating pair
    (Keerthi et al. 2001) for min 1/2 a^T Q a - e^T a, y^T a = 0, 0<=a<=C."""
    N = Q.shape[0]
    a = np.zeros(N)
    grad = -np.ones(N)                      # Q a - e
    for _ in range(max_iter):
        yg = -y * grad
        up = ((y > 0) & (a < C)) | ((y < 0) & (a > 0))
        lowm = ((y > 0) & (a > 0)) | ((y < 0) & (a < C))
        if not up.any() or not lowm.any():
            break
        i = np.flatnonzero(up)[np.argmax(yg[up])]
        j = np.flatnonzero(lowm)[np.argmin(yg[lowm])]
        if yg[i] - yg[j] <= tol:
            break
        # move along y_i d_i = -y_j d_j keeping y^T a = 0
        quad = Q[i, i] + Q[j, j] - 2.0 * y[i] * y[j] * Q[i, j]
        quad = max(quad, 1e-15)
        t = (yg[i] - yg[j]) / quad
        # bounds on t for a_i + y_i t and a_j - y_j t
        ti = (C - a[i]) if y[i] > 0 else a[i]
        tj = a[j] if y[j] > 0 else (C - a[j])
        t = min(t, ti, tj)
        di, dj = y[i] * t, -y[j] * t
        a[i] += di
        a[j] += dj
        grad += Q[:, i] * di + Q[:, j] * dj
    return a


# ---------------------------------------------------------------------------
# Coordinate descent (C helper, cd.c) for
#   min 1/2 ||A x - b||^2 + c^T x + lam1 ||x||_1 + lam2/2 ||x||^2,
# optionally with box bounds instead of the l1 term.  Cyclic exact coordinate
# minimisation, written from the one-dimensional optimality conditions.
# ---------------------------------------------------------------------------
_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_CD_LIB = None


def build_c_helpers() -> str:
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libracoracle.so")
    srcs = [os.path.join(_HERE, "cd.c"), os.path.join(_HERE, "smo.c")]
    if (not os.path.exists(out)) or any(os.path.getmtime(out) < os.path.getmtime(s)
                                        for s in srcs):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"])
        os.replace(tmp, out)
    return out


def _cd_lib():
    global _CD_LIB
    if _CD_LIB is None:
        lib = ctypes.CDLL(build_c_helpers())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.cd_enet.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, ctypes.c_int64, dp, dp,
                                ctypes.c_double, ctypes.c_double, dp,
                                ctypes.c_double, ctypes.c_int64]
        lib.cd_enet.restype = ctypes.c_int64
        lib.smo_svm.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, dp, ctypes.c_double,
                                ctypes.c_int64]
        lib.smo_svm.restype = ctypes.c_int64
        _CD_LIB = lib
    return _CD_LIB


def cd_enet(A, b, lam1, lam2=0.0, c=None, tol=1e-13, max_passes=100000, x0=None):
    """Coordinate descent to a relative stationarity residual <= tol (same
    scale as kkt()).  Returns x."""
    A = np.asfortranarray(A, dtype=np.float64)
    m, n = A.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.zeros(n) if c is None else np.ascontiguousarray(c, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    lib = _cd_lib()
    passes = lib.cd_enet(m, n, A.ctypes.data_as(dp), m, b.ctypes.data_as(dp),
                         c.ctypes.data_as(dp), float(lam1), float(lam2),
                         x.ctypes.data_as(dp), float(tol), int(max_passes))
    if passes < 0:
        raise RuntimeError("coordinate descent did not reach tol")
    return x


def smo_svm_c(Q, y, C, tol=1e-10, max_iter=50_000_000):
    """SMO compiled in oracle/smo.c with second-order working-set selection
    (Fan, Chen and Lin 2005), for duals too large for the numpy loop of
    smo_svm.  Same optimality test (max_up - min_low <= tol).  Returns alpha."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    N = Q.shape[0]
    a = np.zeros(N)
    dp = ctypes.POINTER(ctypes.c_double)
    it = _cd_lib().smo_svm(N, Q.ctypes.data_as(dp), y.ctypes.data_as(dp), float(C),
                           a.ctypes.data_as(dp), float(tol), int(max_iter))
    if it < 0:
        raise RuntimeError("SMO did not reach tol")
    return a


def svm_ipm(Z, y, C, tol=1e-11, max_iter=200, snap=1e-5):
    """Primal-dual interior-point method (Mehrotra's predictor-corrector) for
    the soft-margin SVM dual of Sec. 3.2 eq. svm,

        min 1/2 a^T Q a - e^T a  s.t.  y^T a = 0,  0 <= a <= C,  Q = Z Z^T,

    for duals whose N is too large for SMO but whose Q has low rank d (Z is
    N x d, row i = y_i x_i; linear kernel).  Multipliers lam >= 0 (a >= 0),
    nu >= 0 (a <= C) and b (y^T a = 0) make the KKT system

        Q a - e - b y - lam + nu = 0,  y^T a = 0,
        a_i lam_i = t,  (C - a_i) nu_i = t,  t -> 0.

    Each Newton step eliminates lam and nu, leaving (Q + D) da - y db = r1,
    y^T da = -y^T a with D = lam / a + nu / (C - a) diagonal, solved by the
    Sherman-Morrison-Woodbury identity with the d x d matrix I + Z^T D^{-1} Z
    (Cholesky), plus one step of iterative refinement.  Steps keep 0 < a < C
    and lam, nu > 0 (fraction 0.995 to the boundary).  It stops when the
    complementarity t and the scaled residuals are below tol; coordinates
    within snap * C of a bound whose multiplier marks them active are then put
    on it.  Returns alpha."""
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N, d = Z.shape
    e = np.ones(N)
    a = np.full(N, 0.5 * C)
    lam = np.ones(N)
    nu = np.ones(N)
    b = 0.0

    def qmul(v):
        return Z @ (Z.T @ v)

    def make_solver(Dg):
        Di = 1.0 / Dg
        S = np.eye(d) + Z.T @ (Z * Di[:, None])
        Lc = np.linalg.cholesky(S)

        def msolve(v):
            w = Di * v
            t = solve_triangular(Lc, Z.T @ w, lower=True)
            t = solve_triangular(Lc.T, t, lower=False)
            return w - Di * (Z @ t)

        def solve(v):                      # (D + Q) x = v, one refinement step
            x = msolve(v)
            return x + msolve(v - (Dg * x + qmul(x)))
        return solve

    def newton(solve, rd, rp, rc1, rc2):
        r1 = -rd + rc1 / a - rc2 / (C - a)
        u1 = solve(r1)
        u2 = solve(y)
        db = (-rp - y @ u1) / (y @ u2)
        da = u1 + db * u2
        dl = (rc1 - lam * da) / a
        dn = (rc2 + nu * da) / (C - a)
        return da, db, dl, dn

    def max_step(v, dv):
        neg = dv < 0
        return min(1.0, float(np.min(-v[neg] / dv[neg]))) if neg.any() else 1.0

    for _ in range(max_iter):
        Qa = qmul(a)
        rd = Qa - e - b * y - lam + nu
        rp = float(y @ a)
        t = (a @ lam + (C - a) @ nu) / (2 * N)
        # stop once complementarity is below tol and the residuals are at the
        # rounding level of Q a (they cannot be driven further in FP64)
        if (t <= tol and np.abs(rd).max() <= 1e-10 * max(1.0, float(np.abs(Qa).max()))
                and abs(rp) <= 1e-10 * max(1.0, float(a.sum()))):
            break
        Dg = lam / a + nu / (C - a)
        solve = make_solver(Dg)
        # predictor: the affine-scaling direction (t -> 0)
        da, db, dl, dn = newton(solve, rd, rp, -a * lam, -(C - a) * nu)
        sp = min(max_step(a, da), max_step(C - a, -da))
        sd = min(max_step(lam, dl), max_step(nu, dn))
        s = min(sp, sd)
        t_aff = ((a + s * da) @ (lam + s * dl) + (C - a - s * da) @ (nu + s * dn)) / (2 * N)
        sigma = (t_aff / t) ** 3
        # corrector: centring at sigma t plus the second-order terms
        rc1 = sigma * t - a * lam - da * dl
        rc2 = sigma * t - (C - a) * nu + da * dn
        da, db, dl, dn = newton(solve, rd, rp, rc1, rc2)
        sp = min(max_step(a, da), max_step(C - a, -da))
        sd = min(max_step(lam, dl), max_step(nu, dn))
        s = 0.995 * min(sp, sd)
        a_n, lam_n, nu_n = a + s * da, lam + s * dl, nu + s * dn
        if not (np.all(a_n > 0.0) and np.all(a_n < C) and np.all(lam_n > 0.0)
                and np.all(nu_n > 0.0) and np.isfinite(db)):
            # rounding put an iterate on the boundary: no further progress in FP64
            if t <= 1e-3 * tol ** 0.5:
                break
            raise RuntimeError("interior-point method stalled at complementarity %.2e" % t)
        a, b, lam, nu = a_n, b + s * db, lam_n, nu_n
    else:
        raise RuntimeError("interior-point method did not reach tol")
    # coordinates the multipliers mark as active (a_i < lam_i, or C - a_i <
    # nu_i) and within snap * C of their bound are put on it
    lo = (a < lam) & (a <= snap * C)
    hi = (C - a < nu) & (C - a <= snap * C)
    return np.where(lo, 0.0, np.where(hi, C, a))



def rbf_svm_matrix(X, y, sigma):
    """Q_ij = y_i y_j exp(-||x_i - x_j||^2 / (2 sigma^2)), the Gaussian-kernel
    C-SVC dual matrix (Sec. 3.2, eq. svm; the kernel of Table 8), in FP64
    from the plain definition: squared distances from coordinate
    differences."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    diff = X[:, None, :] - X[None, :, :]
    D = (diff * diff).sum(axis=2)
    return (y[:, None] * y[None, :]) * np.exp(-D / (2.0 * sigma * sigma))
