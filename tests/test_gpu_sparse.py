"""GPU parity of the sparse residual form (compressed columns; the large
sparse Elastic-Net designs of Sec. 3.1, Table 3) through the C-ABI, against
the FP64 oracle on the densified matrix."""
import numpy as np
import pytest

import synth
from oracle import rac_oracle as O

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

from paper_1907_01995_gb300 import _lib  # noqa: E402
from paper_1907_01995_gb300 import api  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / max(1.0, float(np.abs(b).max()))


CASES = {
    # blocks of 60 and of 150 (both through the blocked inverse), ragged p
    "lasso_s60": dict(m=120, n=300, density=0.05, p=5, lam2=0.0),
    "en_s150_ragged": dict(m=90, n=301, density=0.08, p=2, lam2=0.1),
    "en_many_blocks": dict(m=200, n=640, density=0.03, p=32, lam2=0.05),
}


def _inst(c, seed=2):
    return synth.sparse_en_instance(seed, m=c["m"], n=c["n"], density=c["density"],
                                    nnz_frac=0.1, lam_frac=0.2, lam2=c["lam2"],
                                    num_blocks=c["p"])


@pytest.mark.parametrize("assembly", ["rac", "rp"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_sparse_fp64_iterates_match_oracle(name, assembly):
    c = CASES[name]
    if assembly == "rp" and c["n"] % c["p"]:
        pytest.skip("RP on a handle needs equal blocks")
    inst = _inst(c)
    P = O.problem_from_data(inst.A.toarray(), inst.b, "l1l2", inst.lam1, inst.lam2)
    ost = O.initial_state(P)
    with api.Handle(inst.A, inst.b, phi="l1l2", lambda1=inst.lam1, lambda2=inst.lam2,
                    num_blocks=c["p"], tol=0.0, max_sweeps=1, refresh_every=1, seed=5,
                    assembly=assembly) as h:
        for k in range(30):
            O.sweep(P, ost, c["p"], 5, 1.0, 1.0, rp=assembly == "rp")
            _, info = h.solve()
            assert info["form"].startswith("sparse/fp64"), info["form"]
            st = h.state()
            for key in ("x", "z", "xi"):
                assert rel(st[key], getattr(ost, key)) <= 1e-10, (k, key)


@pytest.mark.parametrize("chain", ["auto", "grid"])
@pytest.mark.parametrize("storage,tol,bound", [("fp64", 1e-10, 1e-8), ("fp32", 1e-9, 1e-5),
                                               ("bf16", 1e-7, 1e-3)])
def test_sparse_converged_matches_coordinate_descent(storage, tol, bound, chain):
    """FP64 storage runs the one-CTA chain; FP32 / BF16 run the one-cluster
    chain (auto) or the one-CTA chain (grid)."""
    inst = synth.sparse_en_instance(7, m=600, n=3000, density=0.02, nnz_frac=0.02,
                                    lam_frac=0.1, lam2=0.05, block=100)
    Ad = inst.A.toarray()
    ref = O.cd_enet(Ad, inst.b, inst.lam1, inst.lam2, tol=1e-13)
    with api.Handle(inst.A, inst.b, phi="l1l2", lambda1=inst.lam1, lambda2=inst.lam2,
                    num_blocks=inst.num_blocks, tol=tol, max_sweeps=20000, refresh_every=10,
                    storage=storage, chain=chain) as h:
        z, info = h.solve()
    assert info["status"] == 0, info
    assert info["form"].startswith("sparse/" + storage)
    assert ("/cluster" in info["form"]) == (chain == "auto" and storage != "fp64"), info["form"]
    assert rel(z, ref) <= bound, rel(z, ref)
    assert np.array_equal(z != 0, ref != 0)
    P = O.problem_from_data(Ad, inst.b, "l1l2", inst.lam1, inst.lam2)
    assert O.kkt(P, z)["kkt"] <= tol * 1.01 + 1e-15


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_sparse_cluster_chain_with_coupling_row_and_ragged_blocks(storage):
    """A box QP with one coupling row on a sparse design, blocks of 61 and 60
    (ragged), m not a multiple of the cluster's row split: the one-cluster
    chain converges to a point the oracle's KKT measure certifies."""
    rng = np.random.default_rng(4)
    m, n = 1003, 2441
    A = sp.random(m, n, density=0.03, random_state=5, format="csc")
    A.data = rng.normal(size=A.nnz)
    b = rng.normal(size=m)
    e = rng.choice([-1.0, 1.0], size=n)
    tol = 1e-9 if storage == "fp32" else 1e-7
    with api.Handle(A, b, E=e, d=np.zeros(1), phi="box", lo=0.0, hi=0.5, num_blocks=40,
                    beta=1.0, gamma=1.0, tol=tol, max_sweeps=40000, refresh_every=10,
                    storage=storage) as h:
        z, info = h.solve()
        mu = float(np.atleast_1d(h.state()["mu"])[0])
    assert info["status"] == 0, info
    assert "/cluster" in info["form"], info["form"]
    P = O.problem_from_data(A.toarray(), b, "box", lo=0.0, hi=0.5, E=e, d=np.zeros(1))
    assert np.all(z >= 0.0) and np.all(z <= 0.5)
    assert O.kkt(P, z, mu=mu)["kkt"] <= tol * 1.01


def test_sparse_matches_dense_form():
    """The same problem given densely (residual form) and sparsely reaches
    the same solution."""
    inst = synth.sparse_en_instance(9, m=150, n=400, density=0.1, nnz_frac=0.05,
                                    lam_frac=0.2, lam2=0.1, num_blocks=4)
    kw = dict(phi="l1l2", lambda1=inst.lam1, lambda2=0.1, num_blocks=4, tol=1e-10,
              max_sweeps=20000)
    with api.Handle(inst.A, inst.b, **kw) as h:
        zs, _ = h.solve()
    with api.Handle(inst.A.toarray(), inst.b, form="residual", **kw) as h:
        zd, _ = h.solve()
    assert rel(zs, zd) <= 1e-8


def test_sparse_invalid_indices_rejected():
    inst = synth.sparse_en_instance(3, m=50, n=80, density=0.1, num_blocks=4)
    bad = inst.A.copy()
    bad.indices[3] = 50                       # row out of range
    with pytest.raises(_lib.RacError) as ei:
        api.Handle(_Raw(bad), inst.b, phi="l1l2", lambda1=inst.lam1, num_blocks=4)
    assert ei.value.status == _lib.RAC_ERR_ARG


class _Raw:
    """A CSC matrix passed as is (no sorting or duplicate summing by the binding)."""

    def __init__(self, A):
        self.A = A
        self.shape = A.shape

    def tocsc(self, copy=True):
        return _Frozen(self.A)


class _Frozen:
    def __init__(self, A):
        self.indptr, self.indices, self.data, self.shape = A.indptr, A.indices, A.data, A.shape

    def sum_duplicates(self):
        pass

    def sort_indices(self):
        pass
