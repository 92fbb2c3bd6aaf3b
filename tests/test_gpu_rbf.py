"""The Gaussian-kernel C-SVC dual (Sec. 3.2, eq. svm, with the kernel of
Table 8): the GPU kernel matrix against the oracle's definition, and the dual
solved by the H form against SMO within the bounds both KKT residuals imply."""
import numpy as np
import pytest

import synth
from oracle import rac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01995_gb300 import api  # noqa: E402

import svm_gap  # noqa: E402


@pytest.mark.parametrize("N,d,sigma", [(1, 1, 1.0), (130, 7, 0.8), (300, 33, 2.5)])
def test_rbf_matrix_matches_oracle(N, d, sigma):
    rng = np.random.default_rng(N + d)
    X = rng.normal(size=(N, d))
    y = rng.choice([-1.0, 1.0], size=N)
    Q = api.rbf_svm_matrix(X, y, sigma).cpu().numpy()
    ref = O.rbf_svm_matrix(X, y, sigma)
    assert np.abs(Q - ref).max() <= 1e-14
    assert np.array_equal(Q, Q.T)


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16"])
def test_rbf_svm_converged_matches_smo(storage):
    inst = synth.svm_instance(12, 320, 5, block=64)
    X, y = inst.meta["X"], inst.meta["y"]
    sigma = 1.5
    Q = api.rbf_svm_matrix(X, y, sigma)
    p = (320 + 63) // 64
    tol = 1e-7 if storage != "bf16" else 1e-6
    with api.Handle(H=Q, c=-np.ones(320), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=1.0,
                    num_blocks=p, beta=0.1 * p, gamma=-0.3, tol=tol, max_sweeps=60000,
                    refresh_every=20, storage=storage) as h:
        a, info = h.solve()
    assert info["status"] == 0, info
    Qh = Q.cpu().numpy()
    a_smo = O.smo_svm_c(Qh, y, 1.0, tol=1e-11)
    P = O.Problem(H=Qh, q=-np.ones(320), phi="box", lo=0.0, hi=1.0, E=y.reshape(1, -1),
                  d=np.zeros(1))
    assert O.kkt(P, a)["kkt"] <= tol * 1.01
    gap, gap_bound, wdist, w_bound = svm_gap.check_q(Qh, y, a, a_smo)
    assert gap <= gap_bound, (gap, gap_bound)
    assert wdist <= w_bound, (wdist, w_bound)
