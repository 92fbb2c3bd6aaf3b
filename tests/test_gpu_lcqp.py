"""The paper's linearly constrained QP (Sec. 2, eq. lcqp: min 1/2 x^T H x + c^T x
s.t. E x = d) with k > 1 constraint rows, through the C-ABI: the rows are
folded into the Gram form (beta E^T E in the Gram matrix, the multipliers in
the linear term), so the iterates must still equal the oracle's explicit
split sweep, and the converged point the solution of the KKT system
[[H, E^T], [E, 0]] [x; -mu] = [-c; d]."""
import numpy as np
import pytest

from oracle import rac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01995_gb300 import api  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / max(1.0, float(np.abs(b).max()))


def _lcqp(seed, n, k, m=None):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(m or n + 10, n)) / np.sqrt(n)
    H = B.T @ B
    c = rng.normal(size=n)
    E = rng.normal(size=(k, n))
    d = rng.normal(size=k)
    return B, H, c, E, d


def _kkt_solution(H, c, E, d):
    n, k = H.shape[0], E.shape[0]
    K = np.zeros((n + k, n + k))
    K[:n, :n] = H
    K[:n, n:] = E.T
    K[n:, :n] = E
    sol = np.linalg.solve(K, np.concatenate([-c, d]))
    return sol[:n], -sol[n:]          # x*, mu* (stationarity H x + c - E^T mu = 0)


@pytest.mark.parametrize("chain", ["auto", "grid"])
@pytest.mark.parametrize("k", [2, 5])
def test_lcqp_fp64_iterates_match_oracle(k, chain):
    _, H, c, E, d = _lcqp(3, 41, k)
    P = O.Problem(H=H, q=c, phi="none", E=E, d=d)
    ost = O.initial_state(P)
    with api.Handle(H=H, c=c, E=E, d=d, phi="none", num_blocks=5, beta=0.7, gamma=0.9,
                    tol=0.0, max_sweeps=1, refresh_every=1, seed=4, chain=chain) as h:
        for it in range(30):
            O.sweep(P, ost, 5, 4, 0.7, 0.9)
            _, info = h.solve()
            st = h.state()
            for key in ("x", "z", "xi"):
                assert rel(st[key], getattr(ost, key)) <= 1e-10, (it, key)
            assert rel(st["mu"], ost.mu) <= 1e-10, it


@pytest.mark.parametrize("storage,bound", [("fp64", 1e-8), ("fp32", 1e-5), ("bf16", 1e-3)])
def test_lcqp_converged_matches_kkt_system(storage, bound):
    """Data form (H = B^T B through the tensor-core Gram for FP32/BF16) with
    four constraint rows, every storage, to KKT 1e-9."""
    B, H, c, E, d = _lcqp(5, 96, 4, m=140)
    x_ref, mu_ref = _kkt_solution(H, c, E, d)
    with api.Handle(B, np.zeros(B.shape[0]), c=c, E=E, d=d, phi="none", num_blocks=6, beta=1.0,
                    gamma=1.0, tol=1e-9, max_sweeps=20000, refresh_every=10,
                    storage=storage) as h:
        z, info = h.solve()
        st = h.state()
    assert info["status"] == 0, info
    assert info["form"].startswith("gram/" + storage), info["form"]
    assert rel(z, x_ref) <= bound, rel(z, x_ref)
    assert rel(st["mu"], mu_ref) <= bound * 10, rel(st["mu"], mu_ref)
    P = O.problem_from_data(B, np.zeros(B.shape[0]), "none", c=c, E=E, d=d)
    assert O.kkt(P, z, mu=st["mu"])["kkt"] <= 1e-9 * 1.01
