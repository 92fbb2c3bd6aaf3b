"""Seeded synthetic problem instances (inputs only, no solver arithmetic).

Every instance is the problem

    minimise  1/2 ||A x - b||^2 + c^T x + sum_j phi(x_j)   s.t.  E x = d

with A stored column-major (m x n, float64).  This is the paper's general model
(Sec. 1, eq. general_model) with H = A^T A, written in the data form that
Sec. 3.1 uses for regression (A = X / sqrt(n)) and Sec. 3.2 uses for the SVM
dual (Q = Z Z^T with Z = diag(y) X, so A = Z^T).

The recipes follow the workloads of the paper (Sec. 3.1 synthetic dense and
sparse designs, Sec. 3.2 C-SVC duals); the public LIBSVM/E2006 data sets the
paper uses are not available, so Gaussian designs of the same shape stand in.
All draws use numpy's PCG64 stream seeded by the instance seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Instance:
    """One problem instance plus the run parameters its workload fixes."""

    name: str
    A: np.ndarray                      # m x n, float64, Fortran order
    b: np.ndarray                      # m
    phi: str                           # "none" | "l1l2" | "box"
    lam1: float = 0.0
    lam2: float = 0.0
    lo: float = 0.0
    hi: float = 0.0
    c: Optional[np.ndarray] = None     # extra linear term (n) or None
    E: Optional[np.ndarray] = None     # 1 x n coupling row or None
    d: Optional[np.ndarray] = None     # 1
    num_blocks: int = 1
    beta: float = 1.0
    gamma: float = 1.0
    seed: int = 0
    x_true: Optional[np.ndarray] = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


def _unit_columns(A: np.ndarray) -> np.ndarray:
    nrm = np.sqrt((A * A).sum(axis=0))
    nrm[nrm == 0.0] = 1.0
    return np.asfortranarray(A / nrm)


def regression_instance(seed: int = 0, m: int = 500, n: int = 100,
                        num_blocks: int = 10) -> Instance:
    """Linear regression: A ~ N(0,1), x_true ~ N(0,1), b = A x_true + 0.01 N(0,1)."""
    rng = np.random.default_rng(seed)
    A = np.asfortranarray(rng.standard_normal((m, n)))
    x_true = rng.standard_normal(n)
    b = A @ x_true + 0.01 * rng.standard_normal(m)
    return Instance("regression", A, b, "none", num_blocks=num_blocks,
                    beta=1.0, gamma=1.0, seed=seed, x_true=x_true)


def lasso_instance(seed: int = 0, m: int = 10000, n: int = 2000,
                   num_blocks: int = 20, nnz_frac: float = 0.05,
                   lam_frac: float = 0.1) -> Instance:
    """LASSO: unit-norm N(0,1) columns, x_true 5% nonzero +-U[1,3], noise 0.01,
    lambda1 = 0.1 ||A^T b||_inf."""
    rng = np.random.default_rng(seed)
    A = _unit_columns(rng.standard_normal((m, n)))
    k = max(1, int(round(nnz_frac * n)))
    support = rng.choice(n, size=k, replace=False)
    x_true = np.zeros(n)
    x_true[support] = rng.choice([-1.0, 1.0], size=k) * rng.uniform(1.0, 3.0, size=k)
    b = A @ x_true + 0.01 * rng.standard_normal(m)
    lam1 = lam_frac * float(np.abs(A.T @ b).max())
    return Instance("lasso", A, b, "l1l2", lam1=lam1, lam2=0.0,
                    num_blocks=num_blocks, beta=1.0, gamma=1.0, seed=seed,
                    x_true=x_true)


def elastic_net_instance(seed: int = 0, m: int = 2000, n: int = 50000,
                         num_blocks: int = 100, group: int = 10, rho: float = 0.7,
                         nnz_frac: float = 0.01, noise: float = 0.05,
                         lam_frac: float = 0.05, lam2: float = 0.1) -> Instance:
    """Elastic-Net, n >> m: groups of `group` columns a_j = sqrt(rho) u_g +
    sqrt(1-rho) e_j (pairwise correlation rho), unit-normalised; x_true 1%
    nonzero N(0,1); noise 0.05; lambda1 = 0.05 lambda_max, lambda2 = 0.1."""
    rng = np.random.default_rng(seed)
    ngroups = (n + group - 1) // group
    U = rng.standard_normal((m, ngroups))
    A = np.empty((m, n), order="F")
    sr, sn = math.sqrt(rho), math.sqrt(1.0 - rho)
    for g in range(ngroups):
        j0, j1 = g * group, min(n, (g + 1) * group)
        A[:, j0:j1] = sr * U[:, g:g + 1] + sn * rng.standard_normal((m, j1 - j0))
    A = _unit_columns(A)
    k = max(1, int(round(nnz_frac * n)))
    support = rng.choice(n, size=k, replace=False)
    x_true = np.zeros(n)
    x_true[support] = rng.standard_normal(k)
    b = A @ x_true + noise * rng.standard_normal(m)
    lam_max = float(np.abs(A.T @ b).max())
    return Instance("elastic_net", A, b, "l1l2", lam1=lam_frac * lam_max,
                    lam2=lam2, num_blocks=num_blocks, beta=1.0, gamma=1.0,
                    seed=seed, x_true=x_true, meta={"lambda_max": lam_max})


def svm_instance(seed: int, N: int, d: int, C: float = 1.0, mu_norm: float = 1.5,
                 flip: float = 0.05, block: int = 64) -> Instance:
    """Soft-margin linear C-SVC dual (Sec. 3.2, eq. svm) on two Gaussian classes.

    Samples x_i ~ N(y_i mu, I_d) with ||mu|| = 1.5, 5% of labels flipped.
    With Z = diag(y) X the dual is min 1/2 a^T Z Z^T a - e^T a s.t. y^T a = 0,
    0 <= a <= C, i.e. A = Z^T (d x N), b = 0, c = -e, E = y^T, box [0, C].
    Blocks hold at most `block` dual variables; beta = 0.1 p (Sec. 3.2) for
    the coupling row, and the split penalty gamma = 0.3 mean_j ||A_j||^2 (the
    split x - z = 0 has no counterpart in the paper's SVM runs).
    """
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(d)
    mu = mu_norm * u / np.linalg.norm(u)
    y = rng.choice([-1.0, 1.0], size=N)
    X = y[:, None] * mu[None, :] + rng.standard_normal((N, d))
    flips = rng.random(N) < flip
    y = np.where(flips, -y, y)
    Z = y[:, None] * X                          # N x d
    A = np.asfortranarray(Z.T)                  # d x N, column i = y_i x_i
    p = (N + block - 1) // block
    pen = 0.1 * p
    gam = 0.3 * float((A * A).sum()) / N
    return Instance("svm", A, np.zeros(d), "box", lo=0.0, hi=C,
                    c=-np.ones(N), E=y.reshape(1, N).copy(), d=np.zeros(1),
                    num_blocks=p, beta=pen, gamma=gam, seed=seed,
                    meta={"X": X, "y": y, "C": C, "block": block})


def svm_batch(seed: int = 0, count: int = 256, N_range=(500, 20000),
              d_range=(20, 1000), C: float = 1.0, block: int = 64):
    """`count` uneven SVM dual instances; instance i is drawn with seed + 1 + i,
    its sizes N ~ U{N_range}, d ~ U{d_range} from the master seed."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(N_range[0], N_range[1] + 1, size=count)
    ds = rng.integers(d_range[0], d_range[1] + 1, size=count)
    return [svm_instance(seed + 1 + i, int(Ns[i]), int(ds[i]), C=C, block=block)
            for i in range(count)]


def _ar1_design(rng, m: int, n: int, rho: float) -> np.ndarray:
    A = np.empty((m, n), order="F")
    prev = rng.standard_normal(m)
    A[:, 0] = prev
    s = math.sqrt(max(0.0, 1.0 - rho * rho))
    for j in range(1, n):
        prev = rho * prev + s * rng.standard_normal(m)
        A[:, j] = prev
    return _unit_columns(A)


def warmstart_instance(seed: int, m: int, n: int, rho: float, nnz_frac: float,
                       lam1_frac: float, lam2: float, num_blocks: Optional[int] = None,
                       block: int = 100, noise: float = 0.01) -> Instance:
    """LASSO/Elastic-Net instance with AR(1)-correlated unit-norm columns
    (a_j = rho a_{j-1} + sqrt(1-rho^2) e_j), x_true N(0,1) on a random support,
    lambda1 = lam1_frac * lambda_max."""
    rng = np.random.default_rng(seed)
    A = _ar1_design(rng, m, n, rho)
    k = max(1, int(round(nnz_frac * n)))
    support = rng.choice(n, size=k, replace=False)
    x_true = np.zeros(n)
    x_true[support] = rng.standard_normal(k)
    b = A @ x_true + noise * rng.standard_normal(m)
    lam_max = float(np.abs(A.T @ b).max())
    p = num_blocks if num_blocks is not None else max(1, (n + block - 1) // block)
    return Instance("warmstart", A, b, "l1l2", lam1=lam1_frac * lam_max, lam2=lam2,
                    num_blocks=p, beta=1.0, gamma=1.0, seed=seed, x_true=x_true,
                    meta={"lambda_max": lam_max, "rho": rho})


def warmstart_family(seed: int = 0, count: int = 4096, m_range=(1000, 8000),
                     n_range=(500, 4000), scale: float = 1.0):
    """Parameters of the learned-warm-start family: m, n, rho ~ U[0, 0.8],
    1-10% sparsity, lambda1 ~ U[0.01, 0.5] lambda_max, lambda2 in {0, 0.1}.
    Returns lazily-built (seed_i, kwargs) pairs; `scale` shrinks m and n."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1) * scale)
        n = int(rng.integers(n_range[0], n_range[1] + 1) * scale)
        kw = dict(m=max(8, m), n=max(8, n), rho=float(rng.uniform(0.0, 0.8)),
                  nnz_frac=float(rng.uniform(0.01, 0.10)),
                  lam1_frac=float(rng.uniform(0.01, 0.5)),
                  lam2=float(rng.choice([0.0, 0.1])))
        out.append((seed + 1 + i, kw))
    return out


def path_instance(seed: int = 0, m: int = 20000, n: int = 5000, nlambda: int = 64,
                  rho: float = 0.5, nnz_frac: float = 0.05, lam2: float = 0.0,
                  block: int = 100):
    """Regularisation-path workload: one AR(1) design and `nlambda` values of
    lambda1 geometric from lambda_max down to 0.01 lambda_max."""
    inst = warmstart_instance(seed, m, n, rho, nnz_frac, 0.5, lam2, block=block)
    lam_max = inst.meta["lambda_max"]
    lams = lam_max * np.geomspace(1.0, 0.01, nlambda)
    return inst, lams


def small_instance(seed: int, m: int, n: int, num_blocks: int, phi: str = "l1l2",
                   lam_frac: float = 0.2, lam2: float = 0.0, coupling: bool = False,
                   box=(0.0, 1.0), beta: float = 1.0, gamma: float = 1.0,
                   unit_columns: bool = True) -> Instance:
    """Small generic instance for parity tests (ragged sizes allowed)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    A = _unit_columns(A) if unit_columns else np.asfortranarray(A)
    x_true = np.where(rng.random(n) < 0.3, rng.standard_normal(n), 0.0)
    b = A @ x_true + 0.05 * rng.standard_normal(m)
    lam_max = float(np.abs(A.T @ b).max())
    E = d = c = None
    lo = hi = 0.0
    if phi == "box":
        lo, hi = box
        c = -np.abs(rng.standard_normal(n))
    if coupling:
        E = rng.choice([-1.0, 1.0], size=(1, n))
        d = np.zeros(1)
    return Instance("small", A, b, phi, lam1=lam_frac * lam_max if phi == "l1l2" else 0.0,
                    lam2=lam2, lo=lo, hi=hi, c=c, E=E, d=d, num_blocks=num_blocks,
                    beta=beta, gamma=gamma, seed=seed, x_true=x_true)


def sparse_en_instance(seed: int = 0, m: int = 2000, n: int = 20000, density: float = 0.01,
                       nnz_frac: float = 0.01, noise: float = 0.01, lam_frac: float = 0.1,
                       lam2: float = 0.0, block: int = 100,
                       num_blocks: Optional[int] = None) -> Instance:
    """Sparse LASSO / Elastic-Net design (Sec. 3.1, Table 3: X 40000 x 4M at
    99.8% sparsity, here scaled): every column holds about density * m N(0,1)
    entries at uniformly random rows (coinciding rows summed), scaled to unit
    norm; x_true nnz_frac nonzero N(0,1); b = A x_true + noise; lambda1 =
    lam_frac ||A^T b||_inf.  A is a scipy.sparse CSC matrix."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    per = max(1, int(round(density * m)))
    rows = rng.integers(0, m, size=(n, per), dtype=np.int64).ravel()
    cols = np.repeat(np.arange(n, dtype=np.int64), per)
    vals = rng.standard_normal(n * per)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(m, n))
    A.sum_duplicates()
    A.sort_indices()
    nrm = np.sqrt(np.asarray(A.multiply(A).sum(axis=0)).ravel())
    nrm[nrm == 0.0] = 1.0
    A = sp.csc_matrix(A @ sp.diags(1.0 / nrm))
    A.sort_indices()
    k = max(1, int(round(nnz_frac * n)))
    support = rng.choice(n, size=k, replace=False)
    x_true = np.zeros(n)
    x_true[support] = rng.standard_normal(k)
    b = A @ x_true + noise * rng.standard_normal(m)
    lam_max = float(np.abs(A.T @ b).max())
    p = num_blocks if num_blocks is not None else max(1, (n + block - 1) // block)
    return Instance("sparse_en", A, b, "l1l2", lam1=lam_frac * lam_max, lam2=lam2,
                    num_blocks=p, beta=1.0, gamma=1.0, seed=seed, x_true=x_true,
                    meta={"lambda_max": lam_max, "density": density})


def rbf_svm_data(seed: int = 0, N: int = 20000, d: int = 8, noise: float = 0.5):
    """Features and labels for a Gaussian-kernel C-SVC (Sec. 3.2, Table 8's
    non-linear SVMs): x_i ~ N(0, I_d), y_i = sign(||x_i||^2 - d + noise * eps_i),
    a spherical class boundary that a linear kernel cannot separate.  Stands
    in for the LIBSVM data sets of Table 8, which are not available here.
    Returns (X, y), X of shape (N, d)."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, d))
    y = np.where((X ** 2).sum(1) + noise * rng.normal(size=N) > d, 1.0, -1.0)
    return X, y
