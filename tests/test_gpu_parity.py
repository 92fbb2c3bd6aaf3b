"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Integer work (the random assembly) must be bit-exact.  FP64 iterates must
match the oracle to 1e-10 relative over the first 50 sweeps; converged
solutions must match the independent oracle solvers within the tolerance of
their storage precision (FP64 1e-8, FP32 1e-5, BF16 1e-3 plus the support).
"""
import numpy as np
import pytest

import synth
from oracle import rac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_01995_gb300 import api  # noqa: E402
from paper_1907_01995_gb300 import _lib  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / max(1.0, float(np.abs(b).max()))


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("n,p,seed,sweep0,ns", [
    (1, 1, 0, 0, 1), (7, 3, 3, 2, 4), (100, 10, 0, 0, 3), (2000, 20, 0, 5, 10),
    (4097, 13, 9, 1000, 3), (50000, 100, 0, 0, 2), (20000, 313, 77, 3, 2)])
def test_assembly_bit_exact(n, p, seed, sweep0, ns):
    perm, blk = api.assembly(n, p, seed, sweep0, ns)
    perm, blk = perm.cpu().numpy(), blk.cpu().numpy()
    for s in range(ns):
        ref = O.random_permutation(n, seed, sweep0 + s)
        assert np.array_equal(perm[s], ref)
        bref = np.empty(n, dtype=np.int64)
        for bi, S in enumerate(O.blocks_from_permutation(ref, p)):
            bref[S] = bi
        assert np.array_equal(blk[s], bref)


# ------------------------------------------------------- FP64 iterate parity
CASES = {
    "lasso_gram": dict(m=57, n=43, p=5, phi="l1l2", form="gram"),
    "lasso_residual": dict(m=57, n=43, p=5, phi="l1l2", form="residual"),
    "en_wide_residual": dict(m=31, n=97, p=9, phi="l1l2", lam2=0.1, form="residual"),
    "en_wide_gram": dict(m=31, n=97, p=9, phi="l1l2", lam2=0.1, form="gram"),
    "regression_gram": dict(m=80, n=33, p=4, phi="none", form="gram"),
    "svm_box_residual": dict(m=23, n=71, p=6, phi="box", coupling=True, form="residual",
                             beta=0.6, gamma=0.6),
    "svm_box_gram": dict(m=23, n=71, p=6, phi="box", coupling=True, form="gram",
                         beta=0.6, gamma=0.6),
    "coupled_l1_gamma_ne_beta": dict(m=40, n=29, p=3, phi="l1l2", coupling=True,
                                     form="residual", beta=0.5, gamma=1.5),
    "one_block": dict(m=30, n=12, p=1, phi="l1l2", form="gram"),
    "singleton_blocks": dict(m=30, n=12, p=12, phi="l1l2", form="residual"),
    # blocks of more than 128 coordinates: gathered Gram + blocked inverse +
    # distributed-solve chain (ragged: 602 = 201 + 201 + 200)
    "big_blocks_residual": dict(m=150, n=602, p=3, phi="l1l2", lam2=0.1, form="residual"),
    "big_blocks_coupled": dict(m=90, n=451, p=2, phi="box", coupling=True, form="residual",
                               beta=0.7, gamma=0.9),
    # long columns: the FP64 refresh's A^T r streams whole columns per CTA in
    # 2048-row chunks (4100 = 2 x 2048 + 4: a ragged last chunk; 300 columns
    # split unevenly over the CTAs)
    "long_columns_gram": dict(m=4100, n=300, p=6, phi="l1l2", form="gram"),
    "long_columns_residual": dict(m=4100, n=300, p=6, phi="l1l2", lam2=0.05, form="residual"),
}


def _instance(c, seed=3):
    return synth.small_instance(seed, c["m"], c["n"], c["p"], phi=c["phi"],
                                lam2=c.get("lam2", 0.0), coupling=c.get("coupling", False),
                                beta=c.get("beta", 1.0), gamma=c.get("gamma", 1.0))


def _handle(inst, form, storage="fp64", **kw):
    return api.Handle(inst.A, inst.b, c=inst.c, E=None if inst.E is None else inst.E[0],
                      d=inst.d, phi=inst.phi, lambda1=inst.lam1, lambda2=inst.lam2,
                      lo=inst.lo, hi=inst.hi, num_blocks=inst.num_blocks, beta=inst.beta,
                      gamma=inst.gamma, storage=storage, form=form, **kw)


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_iterates_first_50_sweeps(name):
    c = CASES[name]
    inst = _instance(c)
    P = O.problem_from_instance(inst)
    ost = O.initial_state(P)
    with _handle(inst, c["form"], tol=0.0, max_sweeps=1, refresh_every=1, seed=11) as h:
        for k in range(50):
            O.sweep(P, ost, inst.num_blocks, 11, inst.beta, inst.gamma)
            _, info = h.solve()
            assert info["sweeps"] == 1
            st = h.state()
            for key in ("x", "z", "xi"):
                assert rel(st[key], getattr(ost, key)) <= 1e-10, (k, key)
            if inst.E is not None:
                assert abs(st["mu"] - ost.mu[0]) <= 1e-10 * max(1.0, abs(ost.mu[0]))


@pytest.mark.parametrize("name", ["lasso_gram", "svm_box_residual", "en_wide_residual"])
def test_fp64_periods_match_single_sweeps(name):
    """50 sweeps in periods of 10 (one CUDA graph per period) equal the oracle."""
    c = CASES[name]
    inst = _instance(c, seed=5)
    P = O.problem_from_instance(inst)
    ost = O.initial_state(P)
    for _ in range(50):
        O.sweep(P, ost, inst.num_blocks, 2, inst.beta, inst.gamma)
    with _handle(inst, c["form"], tol=0.0, max_sweeps=50, refresh_every=10, seed=2) as h:
        _, info = h.solve()
        st = h.state()
    assert info["sweeps"] == 50
    for key in ("x", "z", "xi"):
        assert rel(st[key], getattr(ost, key)) <= 1e-10


def test_h_form_matches_oracle():
    rng = np.random.default_rng(0)
    B = rng.normal(size=(40, 25))
    H = B.T @ B
    cvec = rng.normal(size=25)
    P = O.Problem(H=H, q=cvec, phi="l1l2", lam1=0.5)
    ost = O.initial_state(P)
    for _ in range(30):
        O.sweep(P, ost, 4, 0, 1.0, 1.0)
    with api.Handle(H=H, c=cvec, phi="l1l2", lambda1=0.5, num_blocks=4, tol=0.0,
                    max_sweeps=30, refresh_every=7) as h:
        h.solve()
        st = h.state()
    assert rel(st["z"], ost.z) <= 1e-10


# ------------------------------------------------------ converged solutions
def test_regression_config_normal_equations():
    """Linear regression 500 x 100, p = 10, beta = 1, KKT <= 1e-10 within 300
    sweeps, equal to the normal-equation solution."""
    inst = synth.regression_instance(0)
    ref = O.normal_equations(inst.A, inst.b)
    with api.Handle(inst.A, inst.b, phi="none", num_blocks=10, beta=1.0, tol=1e-10,
                    max_sweeps=300, seed=0) as h:
        z, info = h.solve()
    assert info["status"] == 0 and info["kkt"] <= 1e-10
    assert rel(z, ref) <= 1e-8
    P = O.problem_from_instance(inst)
    assert O.kkt(P, z)["kkt"] <= 2e-10


@pytest.fixture(scope="module")
def lasso_ref():
    inst = synth.lasso_instance(0)
    x = O.cd_enet(inst.A, inst.b, inst.lam1, 0.0, tol=1e-13)
    return inst, x


@pytest.mark.parametrize("chain", ["auto", "grid"])
@pytest.mark.parametrize("assembly", ["rac", "rp"])
@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_big_blocks_converged(storage, assembly, chain):
    """Elastic-Net with n > m and 3 blocks of 300 coordinates in FP32 / BF16
    storage reaches the coordinate-descent solution with the same support, on
    the one-cluster residual chain (auto) and on the grid-barrier chain, under
    RAC and RP assembly."""
    inst = synth.small_instance(21, 200, 900, 3, lam2=0.1, lam_frac=0.1)
    ref = O.cd_enet(inst.A, inst.b, inst.lam1, 0.1, tol=1e-13)
    with api.Handle(inst.A, inst.b, phi="l1l2", lambda1=inst.lam1, lambda2=0.1, num_blocks=3,
                    tol=1e-9, max_sweeps=20000, storage=storage, form="residual",
                    assembly=assembly, chain=chain) as h:
        z, info = h.solve()
    assert info["status"] == 0, info
    assert ("/cluster" in info["form"]) == (chain == "auto"), info["form"]
    assert rel(z, ref) <= (1e-5 if storage == "fp32" else 1e-3)
    assert np.array_equal(z != 0, ref != 0)


@pytest.mark.parametrize("storage,tol", [("fp32", 1e-9), ("bf16", 1e-7)])
def test_big_blocks_coupled_box_converged_on_cluster_chain(storage, tol):
    """Box QP with one coupling row (the SVM-dual structure of eq. svm) and
    blocks of 226 in the residual form on the one-cluster chain.  H = A^T A has
    rank 90 < n, so the minimiser need not be unique: the returned point is
    certified by the oracle's KKT measure (with the solver's multiplier) and
    the box."""
    inst = _instance(CASES["big_blocks_coupled"], seed=3)
    P = O.problem_from_instance(inst)
    with _handle(inst, "residual", storage=storage, tol=tol, max_sweeps=40000,
                 refresh_every=10) as h:
        z, info = h.solve()
        mu = float(np.atleast_1d(h.state()["mu"])[0])
    assert info["status"] == 0, info
    assert "/cluster" in info["form"], info["form"]
    assert np.all(z >= inst.lo) and np.all(z <= inst.hi)
    assert O.kkt(P, z, mu=mu)["kkt"] <= tol * 1.01


@pytest.mark.parametrize("storage,form,tol,bound", [
    ("fp64", "gram", 1e-10, 1e-8), ("fp32", "gram", 1e-9, 1e-5),
    ("fp64", "residual", 1e-10, 1e-8), ("fp32", "residual", 1e-9, 1e-5),
    ("bf16", "residual", 1e-7, 1e-3), ("bf16", "gram", 1e-7, 1e-3)])
def test_lasso_config_converged(lasso_ref, storage, form, tol, bound):
    """LASSO 10000 x 2000 (lambda1 = 0.1 ||A^T b||_inf, p = 20): every storage
    precision reaches the FP64 oracle's solution (coordinate descent to
    1e-13) within its tolerance, with the same support."""
    inst, ref = lasso_ref
    with api.Handle(inst.A, inst.b, phi="l1l2", lambda1=inst.lam1, num_blocks=20, beta=1.0,
                    tol=tol, max_sweeps=3000, refresh_every=10, storage=storage,
                    form=form) as h:
        z, info = h.solve()
    assert info["status"] == 0, info
    assert rel(z, ref) <= bound, (rel(z, ref), info)
    assert np.array_equal(z != 0, ref != 0)
    P = O.problem_from_instance(inst)
    assert O.kkt(P, z)["kkt"] <= tol * 1.01 + 1e-15
    # rac_info.obj: 1/2 ||A z - b||^2 + lambda1 ||z||_1 (the oracle drops the constant 1/2 ||b||^2)
    ref_obj = P.objective(z) + 0.5 * float(inst.b @ inst.b)
    assert abs(info["obj"] - ref_obj) <= 1e-12 * abs(ref_obj)


def test_svm_small_converged_matches_smo():
    inst = synth.svm_instance(4, 300, 12, block=64)
    Q = inst.A.T @ inst.A
    y = inst.E[0]
    a_smo = O.smo_svm(Q, y, 1.0, tol=1e-11)
    with api.Handle(inst.A, inst.b, c=inst.c, E=y, d=inst.d, phi="box", lo=0.0, hi=1.0,
                    num_blocks=inst.num_blocks, beta=inst.beta, gamma=-0.3, tol=1e-8,
                    max_sweeps=40000, refresh_every=20) as h:
        a, info = h.solve()
    assert info["status"] == 0, info
    obj = lambda v: 0.5 * v @ Q @ v - v.sum()
    assert abs(obj(a) - obj(a_smo)) <= 1e-6 * max(1.0, abs(obj(a_smo)))
    assert rel(inst.A @ a, inst.A @ a_smo) <= 1e-4
    P = O.problem_from_instance(inst)
    assert O.kkt(P, a)["kkt"] <= 1e-8 * 1.01


# ------------------------------------------------------- state and errors
def test_checkpoint_restore_bitwise():
    inst = _instance(CASES["svm_box_residual"], seed=8)
    with _handle(inst, "residual", tol=0.0, max_sweeps=100, refresh_every=10, seed=4) as h:
        h.solve()
        full = h.state()
    with _handle(inst, "residual", tol=0.0, max_sweeps=50, refresh_every=10, seed=4) as h:
        h.solve()
        blob = h.checkpoint()
    with _handle(inst, "residual", tol=0.0, max_sweeps=50, refresh_every=10, seed=4) as h2:
        h2.restore(blob)
        h2.solve()
        resumed = h2.state()
    for key in ("x", "z", "xi"):
        assert np.array_equal(full[key], resumed[key])
    assert full["mu"] == resumed["mu"]


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_not_positive_definite_is_reported(storage):
    H = -np.eye(6)
    with api.Handle(H=H, c=np.ones(6), phi="none", num_blocks=2, beta=0.5, tol=0.0,
                    max_sweeps=2, storage=storage) as h:
        with pytest.raises(_lib.RacError) as ei:
            h.solve()
    assert ei.value.status == _lib.RAC_ERR_NOT_PD


def test_device_inputs_and_outputs():
    """torch CUDA tensors in and out give the same result as host arrays."""
    inst = _instance(CASES["lasso_gram"], seed=1)
    A = torch.tensor(inst.A, device="cuda")
    b = torch.tensor(inst.b, device="cuda")
    out = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    kw = dict(phi="l1l2", lambda1=inst.lam1, num_blocks=inst.num_blocks, tol=0.0,
              max_sweeps=20)
    with api.Handle(A, b, **kw) as h:
        h.solve(out)
    with api.Handle(inst.A, inst.b, **kw) as h:
        z, _ = h.solve()
    assert np.array_equal(out.cpu().numpy(), z)


@pytest.mark.parametrize("where", ["cuda", "pinned"])
@pytest.mark.parametrize("m,ldpad", [(600, 0), (601, 0), (600, 2), (600, 3)])
def test_bf16_gram_device_A_copy_and_conversion_in_one_pass(m, ldpad, where):
    """A device-resident (or pinned host) A in the BF16 Gram form is copied to
    FP64 and rounded for the tensor-core Gram build in one pass (paired rows
    for even m and lda, single rows otherwise); a pageable host A is copied
    first and converted after.  Both handles' iterates, KKT and objective are
    bit-identical."""
    rng = np.random.default_rng(m + ldpad)
    n = 260
    A = rng.normal(size=(m, n)) / np.sqrt(m)
    b = rng.normal(size=m)
    if where == "cuda":
        big = torch.zeros((n, m + ldpad), dtype=torch.float64, device="cuda")
    else:
        big = torch.zeros((n, m + ldpad), dtype=torch.float64).pin_memory()
    big[:, :m] = torch.tensor(A.T).to(big.device)
    Ad = big.t()[:m]                       # column-major, ld = m + ldpad
    assert Ad.stride() == (1, m + ldpad)
    kw = dict(phi="l1l2", lambda1=0.05, num_blocks=5, tol=0.0, max_sweeps=25,
              storage="bf16", form="gram", refresh_every=5)
    with api.Handle(Ad, torch.tensor(b).to(big.device), **kw) as h:
        zd, infod = h.solve()
        std = h.state()
    with api.Handle(A, b, **kw) as h:
        zh, infoh = h.solve()
        sth = h.state()
    assert infod["form"] == infoh["form"] and infod["form"].startswith("gram/bf16")
    assert np.array_equal(zd, zh)
    for k in ("x", "xi"):
        assert np.array_equal(std[k], sth[k]), k
    assert infod["kkt"] == infoh["kkt"] and infod["obj"] == infoh["obj"]


@pytest.mark.parametrize("storage,m,n", [("fp64", 333, 301), ("fp32", 333, 301),
                                         ("bf16", 333, 301), ("bf16", 1000, 520)])
def test_gram_build_matches_fp64(storage, m, n):
    """G~ = A~^T A~ (rac_gram) on ragged sizes against the FP64 Gram matrix of
    the storage-rounded A: FP64 to 1e-12; FP32 (three-term TF32 split, FP32
    tensor-core accumulation, whose additions are not round-to-nearest) within
    the worst-case bound of a length-m FP32 reduction, m 2^-23 max|G|; BF16
    (stored as BF16) to one BF16 rounding of each entry."""
    rng = np.random.default_rng(7)
    A = np.asfortranarray(rng.normal(size=(m, n)))
    At = torch.tensor(A, device="cuda").t().contiguous().t()
    dt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[storage]
    G = torch.empty((n, n), dtype=dt, device="cuda")
    code = _lib.STORAGE[storage]
    assert _lib.load().rac_gram(m, n, At.data_ptr(), m, code, G.data_ptr(),
                                torch.cuda.current_stream().cuda_stream) == 0
    Ar = torch.tensor(A).to(dt).double().numpy()
    ref = Ar.T @ Ar
    got = G.double().cpu().numpy()
    scale = np.abs(ref).max()
    if storage == "bf16":
        assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * scale)
    else:
        tol = 1e-12 if storage == "fp64" else m * 2.0 ** -23
        assert np.abs(got - ref).max() <= tol * scale
    assert np.array_equal(got, got.T)


@pytest.mark.parametrize("storage,form", [("fp64", "gram"), ("bf16", "gram"), ("fp32", "residual")])
def test_pooled_handles_repeat_bitwise(storage, form):
    """Handles draw memory, streams and events from per-device caches: a
    handle set up on reused (not re-zeroed) memory, or after the cache was
    trimmed, gives bit-identical iterates."""
    inst = _instance(CASES["lasso_gram"], seed=2)
    runs = []
    for rep in range(3):
        if rep == 2:
            api.trim_pool()
        with _handle(inst, form, storage=storage, tol=0.0, max_sweeps=25, refresh_every=5) as h:
            h.solve()
            runs.append(h.state())
    for r in runs[1:]:
        for key in ("x", "z", "xi"):
            assert np.array_equal(runs[0][key], r[key])


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", [
    dict(m=70, n=96, p=7, phi="l1l2"),                          # few owning CTAs, ragged blocks
    dict(m=90, n=104, p=8, phi="box", coupling=True),           # coupling row (t, mu terms)
    dict(m=400, n=2048, p=17, phi="l1l2", lam2=0.05),            # s = 121 / 120
])
def test_cluster_chain_matches_grid_chain(storage, shape):
    """The Gram-form chain on one thread-block cluster and the grid-barrier
    chain compute the same iterates up to FP32 summation order."""
    inst = synth.small_instance(5, shape["m"], shape["n"], shape["p"], phi=shape["phi"],
                                lam2=shape.get("lam2", 0.0), coupling=shape.get("coupling", False))
    out = {}
    for chain in ("grid", "cluster"):
        with _handle(inst, "gram", storage=storage, tol=0.0, max_sweeps=20, refresh_every=5,
                     chain=chain) as h:
            _, info = h.solve()
            out[chain] = (h.state(), info)
    assert "cluster" in out["cluster"][1]["form"], out["cluster"][1]["form"]
    assert "cluster" not in out["grid"][1]["form"]
    for key in ("x", "z", "xi"):
        a, b = out["grid"][0][key], out["cluster"][0][key]
        assert np.linalg.norm(a - b) <= 1e-4 * max(1.0, np.linalg.norm(a)), key


def test_cluster_chain_svm_converged():
    """Soft-margin SVM dual (box + equality row) in FP32 Gram storage on the
    cluster chain reaches the SMO solution."""
    inst = synth.svm_instance(4, 300, 12, block=64)
    Q = inst.A.T @ inst.A
    y = inst.E[0]
    a_smo = O.smo_svm(Q, y, 1.0, tol=1e-11)
    with api.Handle(inst.A, inst.b, c=inst.c, E=y, d=inst.d, phi="box", lo=0.0, hi=1.0,
                    num_blocks=inst.num_blocks, beta=inst.beta, gamma=-0.3, tol=1e-8,
                    max_sweeps=40000, refresh_every=20, storage="fp32", form="gram",
                    chain="cluster") as h:
        a, info = h.solve()
    assert "cluster" in info["form"], info["form"]
    assert info["status"] == 0, info
    obj = lambda v: 0.5 * v @ Q @ v - v.sum()
    assert abs(obj(a) - obj(a_smo)) <= 1e-6 * max(1.0, abs(obj(a_smo)))
    P = O.problem_from_instance(inst)
    assert O.kkt(P, a)["kkt"] <= 1e-8 * 1.01


# ------------------------------------------------------- RP-MBADMM, one problem
RP_CASES = {
    "lasso_gram": dict(m=57, n=45, p=5, phi="l1l2", form="gram"),
    "en_wide_residual": dict(m=31, n=96, p=8, phi="l1l2", lam2=0.1, form="residual"),
    "svm_box_gram": dict(m=23, n=72, p=6, phi="box", coupling=True, form="gram",
                         beta=0.6, gamma=0.6),
    "big_blocks_residual": dict(m=150, n=600, p=3, phi="l1l2", lam2=0.1, form="residual"),
}


@pytest.mark.parametrize("name", sorted(RP_CASES))
def test_rp_handle_fp64_iterates_match_oracle(name):
    """RP-MBADMM on the single-problem handle (fixed consecutive blocks in a
    random order per sweep, inverses computed once) follows the oracle's RP
    iterates sweep by sweep, in both forms and with blocks above 128."""
    c = RP_CASES[name]
    inst = _instance(c, seed=4)
    P = O.problem_from_instance(inst)
    ost = O.initial_state(P)
    with _handle(inst, c["form"], tol=0.0, max_sweeps=1, refresh_every=1, seed=6,
                 assembly="rp") as h:
        for k in range(30):
            O.sweep(P, ost, inst.num_blocks, 6, inst.beta, inst.gamma, rp=True)
            _, info = h.solve()
            assert info["form"].endswith("/rp"), info["form"]
            st = h.state()
            for key in ("x", "z", "xi"):
                assert rel(st[key], getattr(ost, key)) <= 1e-10, (k, key)


@pytest.mark.parametrize("storage,form,bound", [("bf16", "gram", 1e-3), ("fp32", "residual", 1e-5)])
def test_rp_handle_lasso_config_converged(lasso_ref, storage, form, bound):
    """LASSO 10000 x 2000, p = 20 blocks of 100 under RP-MBADMM reaches the
    coordinate-descent solution with the same support."""
    inst, ref = lasso_ref
    with api.Handle(inst.A, inst.b, phi="l1l2", lambda1=inst.lam1, num_blocks=20, beta=1.0,
                    tol=1e-8, max_sweeps=5000, refresh_every=10, storage=storage, form=form,
                    assembly="rp") as h:
        z, info = h.solve()
    assert info["status"] == 0, info
    assert info["form"].endswith("/rp")
    assert rel(z, ref) <= bound
    assert np.array_equal(z != 0, ref != 0)
