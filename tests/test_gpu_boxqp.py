"""The box kept inside the block argmins (eq. RAC-ADDM with x_i in X_i; the
SVM dual of Sec. 3.2, eq. svm, with the Gaussian kernel of Table 8) through
the C-ABI: FP64 iterates equal to the oracle's literal box sweep, converged
points equal to SMO (within the bounds both KKT residuals imply) and to the
split form, and the error paths."""
import numpy as np
import pytest

import synth
from oracle import rac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01995_gb300 import _lib  # noqa: E402
from paper_1907_01995_gb300 import api  # noqa: E402

import svm_gap  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / max(1.0, float(np.abs(b).max()))


def _rbf_svm(seed, N, d, sigma, C=1.0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, d))
    w = rng.normal(size=d)
    y = np.where(X @ w + 0.5 * rng.normal(size=N) > 0, 1.0, -1.0)
    Q = O.rbf_svm_matrix(X, y, sigma)
    P = O.Problem(H=Q, q=-np.ones(N), phi="box", lo=0.0, hi=C, E=y[None, :], d=np.zeros(1))
    return X, y, Q, P


# (N, p): blocks of 12 (ragged: 61 = 12 + 4 x 12 + 1), 64 and 128
SVM_CASES = [(60, 5), (61, 5), (256, 4), (256, 2)]


@pytest.mark.parametrize("prox", [0.0, 0.4])
@pytest.mark.parametrize("N,p", SVM_CASES)
def test_boxqp_svm_fp64_iterates_match_oracle(N, p, prox):
    _, y, Q, P = _rbf_svm(N + p, N, 3, 1.2)
    beta = 0.1 * p
    ost = O.initial_state(P)
    with api.Handle(H=Q, c=-np.ones(N), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=1.0,
                    num_blocks=p, beta=beta, box_qp=True, box_prox=prox, tol=0.0,
                    max_sweeps=1, refresh_every=1, seed=6) as h:
        for k in range(25):
            O.sweep(P, ost, p, 6, beta, prox, box_qp=True)
            _, info = h.solve()
            assert info["status"] == _lib.RAC_ERR_NOT_CONVERGED, info   # tol = 0
            assert info["form"].endswith("/boxqp"), info["form"]
            assert info["box_capped"] == 0 and info["box_iters"] >= p
            st = h.state()
            assert rel(st["x"], ost.x) <= 1e-10, k
            assert np.array_equal(st["z"], st["x"]) and not np.any(st["xi"])
            assert np.all(st["x"] >= 0.0) and np.all(st["x"] <= 1.0)
            mu = float(np.atleast_1d(st["mu"])[0])
            assert abs(mu - ost.mu[0]) <= 1e-10 * max(1.0, abs(ost.mu[0])), k


def test_boxqp_data_form_fp64_iterates_match_oracle():
    """A box-constrained least squares (no coupling row) in the data form:
    H = A^T A through the Gram build, two-sided box, blocks of 40."""
    rng = np.random.default_rng(8)
    A = rng.normal(size=(300, 200)) / np.sqrt(300)
    b = rng.normal(size=300)
    P = O.problem_from_data(A, b, "box", lo=-0.3, hi=0.5)
    ost = O.initial_state(P)
    with api.Handle(A, b, phi="box", lo=-0.3, hi=0.5, num_blocks=5, box_qp=True, tol=0.0,
                    max_sweeps=1, refresh_every=1, seed=2) as h:
        for k in range(25):
            O.sweep(P, ost, 5, 2, 1.0, 0.0, box_qp=True)
            _, info = h.solve()
            assert info["form"] == "gram/fp64/boxqp"
            assert rel(h.state()["x"], ost.x) <= 1e-10, k


@pytest.mark.parametrize("storage,tol,bound", [("fp64", 1e-9, 1e-6), ("fp32", 1e-8, 1e-4),
                                               ("bf16", 1e-7, 1e-3)])
def test_boxqp_rbf_svm_converged_matches_smo_and_split(storage, tol, bound):
    """Gaussian-kernel C-SVC dual, N = 400: Q formed on the GPU, the literal
    box-block iteration run to KKT tol in every storage; the result is within
    the bounds the KKT residuals imply of SMO's, and equal (to the same
    accuracy) to the split form's."""
    inst = synth.svm_instance(21, 400, 5, block=64)
    X, y = inst.meta["X"], inst.meta["y"]
    Q = api.rbf_svm_matrix(X, y, 1.5)
    p = (400 + 63) // 64
    with api.Handle(H=Q, c=-np.ones(400), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=1.0,
                    num_blocks=p, beta=0.1 * p, box_qp=True, box_prox=0.0, tol=tol,
                    max_sweeps=20000, refresh_every=10, storage=storage) as h:
        a, info = h.solve()
    assert info["status"] == 0, info
    assert info["box_capped"] == 0
    Qh = Q.cpu().numpy()
    P = O.Problem(H=Qh, q=-np.ones(400), phi="box", lo=0.0, hi=1.0, E=y.reshape(1, -1),
                  d=np.zeros(1))
    assert O.kkt(P, a)["kkt"] <= tol * 1.01
    a_smo = O.smo_svm_c(Qh, y, 1.0, tol=1e-11)
    gap, gap_bound, wdist, w_bound = svm_gap.check_q(Qh, y, a, a_smo)
    assert gap <= gap_bound, (gap, gap_bound)
    assert wdist <= w_bound, (wdist, w_bound)
    with api.Handle(H=Q, c=-np.ones(400), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=1.0,
                    num_blocks=p, beta=0.1 * p, gamma=-0.3, tol=tol, max_sweeps=60000,
                    refresh_every=20, storage=storage) as h:
        a_split, info_s = h.solve()
    assert info_s["status"] == 0, info_s
    assert abs(info["obj"] - info_s["obj"]) <= bound * max(1.0, abs(info_s["obj"]))


def test_boxqp_warm_start_projected_and_reset():
    _, y, Q, P = _rbf_svm(3, 50, 2, 1.0)
    x0 = np.linspace(-1.0, 2.0, 50)
    with api.Handle(H=Q, c=-np.ones(50), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=1.0,
                    num_blocks=4, beta=0.4, box_qp=True, tol=0.0, max_sweeps=1,
                    x0=x0, xi0=np.ones(50)) as h:
        st = h.state()
        assert np.array_equal(st["x"], np.clip(x0, 0.0, 1.0))
        assert np.array_equal(st["z"], st["x"]) and not np.any(st["xi"])
        ost = O.initial_state(P, x0=np.clip(x0, 0.0, 1.0))
        for k in range(5):
            O.sweep(P, ost, 4, 0, 0.4, 0.0, box_qp=True)
            h.solve()
            assert rel(h.state()["x"], ost.x) <= 1e-10


def test_boxqp_singular_block_reports_not_pd():
    """The literal block argmin (box_prox = 0) of a linear objective (H = 0, no
    coupling row) has no unique minimiser: the sweep of a free pivot meets a
    zero and the solve returns RAC_ERR_NOT_PD; a proximal weight cures it."""
    rng = np.random.default_rng(1)
    H = np.zeros((40, 40))
    q = rng.normal(size=40)
    x0 = np.full(40, 0.5)             # all coordinates free
    with api.Handle(H=H, c=q, phi="box", lo=0.0, hi=1.0, num_blocks=2, box_qp=True,
                    tol=0.0, max_sweeps=2, x0=x0) as h:
        with pytest.raises(_lib.RacError) as ei:
            h.solve()
    assert ei.value.status == _lib.RAC_ERR_NOT_PD
    with api.Handle(H=H, c=q, phi="box", lo=0.0, hi=1.0, num_blocks=2, box_qp=True,
                    box_prox=0.5, tol=1e-10, max_sweeps=20000, x0=x0) as h:
        z, info = h.solve()
    assert info["status"] == 0, info
    P = O.Problem(H=H, q=q, phi="box", lo=0.0, hi=1.0)
    assert O.kkt(P, z)["kkt"] <= 1e-10 * 1.01


def test_boxqp_data_form_box_excluding_zero_converges_on_the_oracle_kkt():
    """A box that excludes 0 (bounded least squares on [2, 3]): the cold
    start is projected into the box, while the KKT measure keeps its scale
    max(1, ||grad f(0)||_inf) from the gradient at zero; converged to tol, the
    point meets the oracle's KKT measure to the same tol."""
    rng = np.random.default_rng(12)
    A = rng.normal(size=(240, 150)) / np.sqrt(240)
    b = 3.0 * rng.normal(size=240)
    tol = 1e-9
    with api.Handle(A, b, phi="box", lo=2.0, hi=3.0, num_blocks=5, box_qp=True, tol=tol,
                    max_sweeps=20000, refresh_every=10) as h:
        z, info = h.solve()
    assert info["status"] == 0, info
    assert np.all(z >= 2.0) and np.all(z <= 3.0)
    P = O.problem_from_data(A, b, "box", lo=2.0, hi=3.0)
    k = O.kkt(P, z)["kkt"]
    assert k <= tol * 1.01
    # the reported measure is the oracle's (same scale), both ways within 1%
    assert k <= info["kkt"] * 1.01 + 1e-15 and info["kkt"] <= k * 1.01 + 1e-15, (k, info["kkt"])
