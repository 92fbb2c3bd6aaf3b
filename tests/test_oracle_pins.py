"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: an
independent library routine (numpy's Philox, lstsq, scipy's scalar
minimiser), a closed form, the paper's own linear-map view of one sweep
(Sec. 2), brute-force enumeration, or a textbook algorithm written out
separately in this file.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import synth
from oracle import rac_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# --------------------------------------------------------------------------- Philox
@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((5, 7, 9, 11), (123, 456)),
    ((0xFFFFFFFF, 1, 2, 3), (0xDEADBEEF, 0x12345678)),
    ((2**40 + 17, 0, 2**63, 99), (2**64 - 5, 1)),
])
def test_philox_matches_numpy(ctr, key):
    """numpy's Philox bit generator returns Philox4x64-10(counter + 1, key)
    as its first four raw words; our restatement must agree bit for bit."""
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(4).astype(np.uint64)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    got = O.philox4x64_10(tuple(np.uint64(v) for v in c), key)
    assert [int(v) for v in got] == [int(v) for v in ref]


def test_philox_vectorised_matches_scalar():
    j = np.arange(50, dtype=np.uint64)
    vec = O.philox4x64_10((j, np.uint64(3), np.uint64(0), np.uint64(0)), (7, 0))
    for i in (0, 1, 17, 49):
        bg = np.random.Philox(counter=np.array([i - 1 if i else 2**64 - 1, 3 if i else 2, 0, 0],
                                                dtype=np.uint64),
                              key=np.array([7, 0], dtype=np.uint64))
        ref = bg.random_raw(4)
        assert [int(v[i]) for v in vec] == [int(v) for v in ref]


# --------------------------------------------------------------- random assembly
def test_permutation_is_sorted_keys():
    for n, seed, k in [(1, 0, 0), (7, 3, 2), (1000, 11, 5)]:
        perm = O.random_permutation(n, seed, k)
        assert sorted(perm.tolist()) == list(range(n))
        keys = O.assembly_keys(n, seed, k)
        assert np.all(np.diff(keys[perm].astype(np.float64)) >= 0)


def test_block_sizes_rule():
    for n, p in [(10, 10), (100, 10), (203, 7), (5, 1), (50000, 100), (20000, 313)]:
        sz = O.block_sizes(n, p)
        assert sum(sz) == n and len(sz) == p
        assert max(sz) - min(sz) <= 1
        assert sz == sorted(sz, reverse=True)
    with pytest.raises(ValueError):
        O.block_sizes(3, 4)


@pytest.mark.parametrize("row", _rows("counting.txt"))
def test_assembly_counts(row):
    """|Gamma| and |Upsilon| of Sec. 2, by enumeration of all permutations
    through the oracle's permutation -> blocks map; every ordered block
    sequence is reached by exactly (s!)^p permutations (uniform assembly)."""
    n, p, gam, ups = (int(v) for v in row)
    s = n // p
    counts = {}
    for perm in itertools.permutations(range(n)):
        blocks = O.blocks_from_permutation(np.array(perm), p)
        key = tuple(tuple(sorted(b.tolist())) for b in blocks)
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == gam
    assert set(counts.values()) == {math.factorial(s) ** p}
    unordered = {frozenset(k) for k in counts}
    assert len(unordered) == ups
    assert len(O.all_assemblies(n, p)) == gam


def test_assembly_empirically_uniform():
    """Over many sweeps each ordered partition of 4 into 2 blocks appears
    with frequency close to 1/6 (Philox keys are uniform)."""
    counts = {}
    T = 6000
    for k in range(T):
        blocks = O.random_assembly(4, 2, seed=5, sweep=k)
        key = tuple(tuple(sorted(b.tolist())) for b in blocks)
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 6
    for v in counts.values():
        assert abs(v / T - 1 / 6) < 0.025


# --------------------------------------------------------------------- z-block
@pytest.mark.parametrize("row", _rows("soft_threshold.txt"))
def test_paper_soft_threshold_cases(row):
    a, b, s = (float(v) for v in row)
    assert O.paper_S(np.array([a]), b)[0] == s


def test_z_block_minimises_subproblem():
    """The closed form of Sec. 3.1 must minimise, per coordinate,
    (xi - gamma x) z + gamma/2 z^2 + lam2/2 z^2 + lam1 |z| (l1l2), and the box
    form must minimise -xi z + gamma/2 (x - z)^2 on [lo, hi]."""
    rng = np.random.default_rng(0)
    for _ in range(60):
        x, xi = rng.normal(size=2) * 2
        gamma = rng.uniform(0.1, 3)
        lam1, lam2 = rng.uniform(0, 2), rng.choice([0.0, rng.uniform(0, 1)])
        P = O.Problem(H=np.eye(1), q=np.zeros(1), phi="l1l2", lam1=lam1, lam2=lam2)
        z = O.z_block(P, np.array([x]), np.array([xi]), gamma)[0]
        f = lambda t: (xi - gamma * x) * t + 0.5 * (gamma + lam2) * t * t + lam1 * abs(t)
        ref = minimize_scalar(f, bounds=(-20, 20), method="bounded",
                              options={"xatol": 1e-12}).x
        assert abs(z - ref) < 1e-7
        lo, hi = sorted(rng.uniform(-1, 2, size=2))
        P = O.Problem(H=np.eye(1), q=np.zeros(1), phi="box", lo=lo, hi=hi)
        z = O.z_block(P, np.array([x]), np.array([xi]), gamma)[0]
        # the z-part of the split Lagrangian is +xi z + gamma/2 (x - z)^2
        ref = minimize_scalar(lambda t: xi * t + 0.5 * gamma * (x - t) ** 2,
                              bounds=(lo, hi), method="bounded",
                              options={"xatol": 1e-12}).x
        assert abs(z - ref) < 1e-6


# ------------------------------------------------------------------ block argmin
def test_block_argmin_zero_block_gradient_and_descent():
    """After a block update the finite-difference gradient of the split
    augmented Lagrangian in the block's coordinates vanishes, and no block
    update increases it."""
    inst = synth.small_instance(3, 30, 11, 3, phi="box", coupling=True, beta=0.7, gamma=1.3)
    P = O.problem_from_instance(inst)
    rng = np.random.default_rng(1)
    st = O.State(x=rng.normal(size=11), z=np.clip(rng.normal(size=11), 0, 1),
                 xi=rng.normal(size=11), mu=rng.normal(size=1))
    beta, gamma = inst.beta, inst.gamma
    blocks = O.random_assembly(11, 3, seed=0, sweep=0)
    before = O.augmented_lagrangian(P, st, beta, gamma)
    for S in blocks:
        O.block_argmin(P, st, S, beta, gamma)
        after = O.augmented_lagrangian(P, st, beta, gamma)
        assert after <= before + 1e-12
        before = after
        h = 1e-6
        for j in S:
            sp, sm = st.copy(), st.copy()
            sp.x[j] += h
            sm.x[j] -= h
            fd = (O.augmented_lagrangian(P, sp, beta, gamma)
                  - O.augmented_lagrangian(P, sm, beta, gamma)) / (2 * h)
            assert abs(fd) < 1e-6


# ---------------------------------------------------- the linear-map view (Sec. 2)
def _lifted(P, beta):
    """Split problem with lam1 = 0 as an eq. lcqp in w = (x, z): H_w =
    blkdiag(H, lam2 I), c_w = (q, 0), constraints [I -I; E 0] w = [0; d]."""
    n = P.n
    Hw = np.zeros((2 * n, 2 * n))
    Hw[:n, :n] = P.H
    Hw[n:, n:] = P.lam2 * np.eye(n)
    cw = np.concatenate([P.q, np.zeros(n)])
    rows = [np.hstack([np.eye(n), -np.eye(n)])]
    rhs = [np.zeros(n)]
    if P.E is not None:
        rows.append(np.hstack([P.E, np.zeros_like(P.E)]))
        rhs.append(P.d)
    return Hw, cw, np.vstack(rows), np.concatenate(rhs)


@pytest.mark.parametrize("coupling", [False, True])
def test_split_sweep_equals_paper_linear_map(coupling):
    """With lam1 = 0 and gamma = beta the split sweep is the paper's iteration
    on the lifted eq. lcqp with assembly sigma = (S_1 .. S_p, z-block), so one
    oracle sweep must equal z^{k+1} = M_sigma z^k + Lbar^{-1} bbar (Sec. 2)."""
    inst = synth.small_instance(7, 25, 13, 4, phi="l1l2", coupling=coupling,
                                beta=0.8, gamma=0.8, lam2=0.3)
    inst.lam1 = 0.0
    P = O.problem_from_instance(inst)
    beta = 0.8
    rng = np.random.default_rng(2)
    st = O.State(x=rng.normal(size=13), z=rng.normal(size=13), xi=rng.normal(size=13),
                 mu=rng.normal(size=1) if coupling else np.zeros(0))
    blocks = O.random_assembly(13, 4, seed=9, sweep=0)
    Hw, cw, Aw, bw = _lifted(P, beta)
    sigma = [np.asarray(S) for S in blocks] + [np.arange(13, 26)]
    M, off = O.linear_map(Hw, cw, Aw, bw, beta, sigma)
    y = np.concatenate([st.xi, st.mu])
    zk = np.concatenate([st.x, st.z, y])
    expect = M @ zk + off
    O.sweep(P, st, 4, 9, beta, beta, blocks=blocks)
    got = np.concatenate([st.x, st.z, st.xi, st.mu])
    assert np.allclose(got, expect, rtol=1e-11, atol=1e-11)


def test_split_sweep_with_three_coupling_rows_equals_paper_linear_map():
    """The split sweep with k = 3 coupling rows (the general eq. lcqp
    constraint block) equals the paper's linear map of the lifted problem
    (Sec. 2), as the one-row case above."""
    inst = synth.small_instance(8, 25, 13, 4, phi="l1l2", beta=0.8, gamma=0.8, lam2=0.3)
    inst.lam1 = 0.0
    rng = np.random.default_rng(5)
    inst.E = rng.normal(size=(3, 13))
    inst.d = rng.normal(size=3)
    P = O.problem_from_instance(inst)
    beta = 0.8
    st = O.State(x=rng.normal(size=13), z=rng.normal(size=13), xi=rng.normal(size=13),
                 mu=rng.normal(size=3))
    blocks = O.random_assembly(13, 4, seed=3, sweep=2)
    Hw, cw, Aw, bw = _lifted(P, beta)
    sigma = [np.asarray(S) for S in blocks] + [np.arange(13, 26)]
    M, off = O.linear_map(Hw, cw, Aw, bw, beta, sigma)
    zk = np.concatenate([st.x, st.z, st.xi, st.mu])
    expect = M @ zk + off
    O.sweep(P, st, 4, 3, beta, beta, blocks=blocks)
    got = np.concatenate([st.x, st.z, st.xi, st.mu])
    assert np.allclose(got, expect, rtol=1e-11, atol=1e-11)


def test_lcqp_sweep_equals_paper_linear_map():
    rng = np.random.default_rng(4)
    n, mm = 9, 3
    B = rng.normal(size=(12, n))
    H = B.T @ B
    c = rng.normal(size=n)
    Aeq = rng.normal(size=(mm, n))
    beq = rng.normal(size=mm)
    beta = 1.7
    blocks = O.random_assembly(n, 3, seed=1, sweep=4)
    x, y = rng.normal(size=n), rng.normal(size=mm)
    M, off = O.linear_map(H, c, Aeq, beq, beta, blocks)
    x1, y1 = O.sweep_lcqp(H, c, Aeq, beq, beta, x, y, blocks)
    assert np.allclose(np.concatenate([x1, y1]), M @ np.concatenate([x, y]) + off,
                       rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("n,p", [(4, 2), (6, 2), (6, 3)])
def test_lemma_eig_QS(n, p):
    """Lemma 2.3: eig(QS) lies in [0, 4/3) with Q = E_sigma[L_sigma^{-1}] and
    S = H + beta A^T A; and the expected map M has spectral radius <= 1."""
    rng = np.random.default_rng(n * 10 + p)
    B = rng.normal(size=(n + 2, n))
    H = B.T @ B * 0.3
    Aeq = rng.normal(size=(2, n))
    beta = 1.0
    Q, S, count = O.expected_Q(H, Aeq, beta, n, p)
    assert count == math.factorial(n) // math.factorial(n // p) ** p
    ev = np.linalg.eigvals(Q @ S)
    assert np.all(ev.real > -1e-10) and np.all(ev.real < 4 / 3)
    assert np.max(np.abs(ev.imag)) < 1e-8
    # expected M from the paper's block formula equals the average of M_sigma
    mm = Aeq.shape[0]
    Mexp = np.block([[np.eye(n) - Q @ S, Q @ Aeq.T],
                     [-beta * Aeq + beta * Aeq @ Q @ S, np.eye(mm) - beta * Aeq @ Q @ Aeq.T]])
    Mavg = np.zeros_like(Mexp)
    sig = O.all_assemblies(n, p)
    for blocks in sig:
        Mavg += O.linear_map(H, np.zeros(n), Aeq, np.zeros(mm), beta, blocks)[0]
    Mavg /= len(sig)
    assert np.allclose(Mavg, Mexp, atol=1e-10)
    assert np.max(np.abs(np.linalg.eigvals(Mexp))) <= 1 + 1e-9


# ------------------------------------------------------------ special cases
def test_one_block_is_textbook_admm_lasso():
    """p = 1: the split iteration is the textbook scaled two-block
    ADMM for the LASSO, x = (A^T A + g I)^{-1}(A^T b + g (z - u)),
    z = soft(x + u, lam/g), u = u + x - z, with u = -xi / g."""
    inst = synth.small_instance(5, 40, 15, 1)
    P = O.problem_from_instance(inst)
    g = 0.9
    st = O.initial_state(P)
    A, b, lam = inst.A, inst.b, inst.lam1
    x = np.zeros(15)
    z = np.zeros(15)
    u = np.zeros(15)
    Kinv = np.linalg.inv(A.T @ A + g * np.eye(15))
    for k in range(25):
        O.sweep(P, st, 1, 0, 1.0, g)
        x = Kinv @ (A.T @ b + g * (z - u))
        v = x + u
        z = np.sign(v) * np.maximum(np.abs(v) - lam / g, 0)
        u = u + x - z
        assert np.allclose(st.x, x, atol=1e-12)
        assert np.allclose(st.z, z, atol=1e-12)
        assert np.allclose(-st.xi / g, u, atol=1e-12)


def test_regression_matches_normal_equations():
    """Regression workload (500 x 100, p = 10): converged iterates equal the
    normal-equation solution and numpy's lstsq (Sec. 3.1 with lambda = 0)."""
    inst = synth.regression_instance(0)
    P = O.problem_from_instance(inst)
    st, info = O.solve(P, inst.num_blocks, seed=0, beta=1.0, gamma=1.0, tol=1e-10,
                       max_sweeps=300)
    assert info["kkt"] <= 1e-10
    ne = O.normal_equations(inst.A, inst.b)
    ls = np.linalg.lstsq(inst.A, inst.b, rcond=None)[0]
    assert np.abs(ne - ls).max() < 1e-10
    assert np.abs(st.z - ne).max() < 1e-8 * max(1, np.abs(ne).max())


def test_orthogonal_design_closed_form():
    """A^T A = I: the Elastic-Net solution is soft(A_j^T b, lam1)/(1 + lam2)."""
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.normal(size=(60, 20)))
    A = np.asfortranarray(Qm)
    b = rng.normal(size=60)
    for lam1, lam2 in [(0.3, 0.0), (0.5, 0.4)]:
        ref = np.sign(A.T @ b) * np.maximum(np.abs(A.T @ b) - lam1, 0) / (1 + lam2)
        P = O.problem_from_data(A, b, "l1l2", lam1, lam2)
        st, info = O.solve(P, 4, seed=1, tol=1e-12, max_sweeps=2000)
        assert np.abs(st.z - ref).max() < 1e-10
        x = O.cd_enet(A, b, lam1, lam2)
        assert np.abs(x - ref).max() < 1e-12


@pytest.mark.parametrize("seed,lam2", [(0, 0.0), (1, 0.2), (2, 0.0)])
def test_lasso_matches_enumeration_and_cd(seed, lam2):
    inst = synth.small_instance(seed, 30, 8, 3, lam2=lam2)
    P = O.problem_from_instance(inst)
    ref = O.enum_lasso(inst.A, inst.b, inst.lam1, lam2)
    st, info = O.solve(P, 3, seed=seed, tol=1e-12, max_sweeps=5000)
    assert info["kkt"] <= 1e-12
    assert np.abs(st.z - ref).max() < 1e-9
    assert np.array_equal(st.z != 0, ref != 0)
    x = O.cd_enet(inst.A, inst.b, inst.lam1, lam2)
    assert np.abs(x - ref).max() < 1e-11


def _svm_tiny(seed, N=7, d=3):
    inst = synth.svm_instance(seed, N, d, C=1.0, block=3)
    return inst


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_svm_matches_enumeration_and_smo(seed):
    """Dual C-SVC (eq. svm): the converged split iteration, SMO and
    brute-force enumeration agree on w = Z^T a and the objective; the KKT
    measure is ~0 at the enumerated optimum."""
    inst = _svm_tiny(seed)
    P = O.problem_from_instance(inst)
    Q = inst.A.T @ inst.A
    y = inst.E[0]
    a_enum, mu_enum = O.enum_svm(Q, y, 1.0)
    a_smo = O.smo_svm(Q, y, 1.0)
    st, info = O.solve(P, inst.num_blocks, seed=seed, beta=inst.beta, gamma=inst.gamma,
                       tol=1e-9, max_sweeps=20000)
    assert info["kkt"] <= 1e-9
    obj = lambda a: 0.5 * a @ Q @ a - a.sum()
    for a in (a_smo, st.z):
        assert abs(obj(a) - obj(a_enum)) < 1e-7
        assert np.abs(inst.A @ a - inst.A @ a_enum).max() < 1e-5
    assert O.kkt(P, a_enum)["kkt"] < 1e-9


def test_kkt_detects_planted_errors():
    """The KKT measure is ~0 at a known optimum and grows under a small
    perturbation of any coordinate, a wrong sign, or a broken bound."""
    inst = synth.small_instance(0, 30, 8, 3)
    P = O.problem_from_instance(inst)
    ref = O.enum_lasso(inst.A, inst.b, inst.lam1)
    assert O.kkt(P, ref)["kkt"] < 1e-12
    for j in range(8):
        bad = ref.copy()
        bad[j] += 1e-3
        assert O.kkt(P, bad)["kkt"] > 1e-5
    nz = np.flatnonzero(ref)
    bad = ref.copy()
    bad[nz[0]] = -bad[nz[0]]
    assert O.kkt(P, bad)["kkt"] > 1e-3
    inst = _svm_tiny(1)
    P = O.problem_from_instance(inst)
    a, mu = O.enum_svm(inst.A.T @ inst.A, inst.E[0], 1.0)
    r = O.kkt(P, a)
    assert r["kkt"] < 1e-9
    bad = a.copy()
    bad[0] = bad[0] + 0.01 if bad[0] < 1 else bad[0] - 0.01
    assert O.kkt(P, bad)["kkt"] > 1e-4


def test_cd_matches_rac_medium():
    """Coordinate descent and the RAC iteration agree on a medium
    Elastic-Net instance with a ragged block split."""
    inst = synth.small_instance(11, 120, 61, 7, lam2=0.1)
    P = O.problem_from_instance(inst)
    x = O.cd_enet(inst.A, inst.b, inst.lam1, 0.1)
    st, info = O.solve(P, 7, seed=3, tol=1e-11, max_sweeps=5000)
    assert np.abs(st.z - x).max() < 1e-9
    assert np.array_equal(st.z != 0, x != 0)


# ---------------------------------------------------------------------------
# RP-MBADMM (Sec. 1): a fixed partition whose blocks are solved in a random
# order every iteration.
# ---------------------------------------------------------------------------
def test_rp_fixed_partition_and_random_order():
    """Every RP sweep visits the blocks of one fixed partition exactly once,
    the orders are permutations of 0..p-1, and all p! orders occur about
    equally often."""
    n, p = 23, 4
    fixed = O.fixed_partition(n, p)
    assert [len(b) for b in fixed] == O.block_sizes(n, p)
    assert np.array_equal(np.concatenate(fixed), np.arange(n))
    counts = {}
    for k in range(2400):
        order = O.rp_order(p, 5, k)
        assert sorted(order.tolist()) == list(range(p))
        blocks = O.rp_assembly(n, p, 5, k)
        for b, S in zip(order, blocks):
            assert np.array_equal(S, fixed[b])
        counts[tuple(order)] = counts.get(tuple(order), 0) + 1
    assert len(counts) == 24
    assert min(counts.values()) > 100 * 0.6 and max(counts.values()) < 100 * 1.4


def test_rp_one_block_equals_rac_one_block():
    """With p = 1 there is no order to draw: RP and RAC run the same
    iteration (the single block argmin is the whole x-minimisation)."""
    inst = synth.small_instance(2, 40, 12, 3, lam2=0.1)
    P = O.problem_from_instance(inst)
    a, b = O.initial_state(P), O.initial_state(P)
    for _ in range(15):
        O.sweep(P, a, 1, 3, 1.0, 1.0)
        O.sweep(P, b, 1, 3, 1.0, 1.0, rp=True)
    assert np.abs(a.z - b.z).max() < 1e-12
    assert np.abs(a.xi - b.xi).max() < 1e-12


@pytest.mark.parametrize("seed,lam2", [(0, 0.0), (1, 0.2)])
def test_rp_lasso_matches_enumeration(seed, lam2):
    """The RP fixed point is the LASSO / Elastic-Net solution (brute-force
    active-set enumeration and coordinate descent)."""
    inst = synth.small_instance(seed, 30, 8, 3, lam2=lam2)
    P = O.problem_from_instance(inst)
    ref = O.enum_lasso(inst.A, inst.b, inst.lam1, lam2)
    st, info = O.solve(P, 3, seed=seed, tol=1e-12, max_sweeps=8000, rp=True)
    assert info["kkt"] <= 1e-12
    assert np.abs(st.z - ref).max() < 1e-9
    assert np.array_equal(st.z != 0, ref != 0)


def test_rp_svm_matches_enumeration():
    """The RP fixed point of the SVM dual is the enumerated optimum."""
    inst = _svm_tiny(1)
    P = O.problem_from_instance(inst)
    Q = inst.A.T @ inst.A
    a_enum, _ = O.enum_svm(Q, inst.E[0], 1.0)
    st, info = O.solve(P, inst.num_blocks, seed=4, beta=inst.beta, gamma=inst.gamma,
                       tol=1e-9, max_sweeps=30000, rp=True)
    assert info["kkt"] <= 1e-9
    obj = lambda a: 0.5 * a @ Q @ a - a.sum()
    assert abs(obj(st.z) - obj(a_enum)) < 1e-7


def obj_m(Q, a):
    return 0.5 * a @ Q @ a - a.sum()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_compiled_smo_matches_enumeration_and_numpy_smo(seed):
    """The compiled SMO (oracle/smo.c, second-order pair selection) reaches the
    enumerated optimum of tiny duals and the numpy SMO's optimum (maximal
    violating pair) on medium ones: same objective and w (alpha need not be
    unique)."""
    inst = _svm_tiny(seed)
    Q = inst.A.T @ inst.A
    y = inst.E[0]
    a_enum, _ = O.enum_svm(Q, y, 1.0)
    a_c = O.smo_svm_c(Q, y, 1.0)
    obj = lambda a: 0.5 * a @ Q @ a - a.sum()
    assert abs(obj(a_c) - obj(a_enum)) < 1e-9
    assert np.abs(inst.A @ a_c - inst.A @ a_enum).max() < 1e-6
    assert abs(float(y @ a_c)) < 1e-12
    med = synth.svm_instance(40 + seed, 240, 9)
    Qm = med.A.T @ med.A
    a_py = O.smo_svm(Qm, med.E[0], 1.0, tol=1e-11)
    a_cm = O.smo_svm_c(Qm, med.E[0], 1.0, tol=1e-11)
    assert abs(obj_m(Qm, a_py) - obj_m(Qm, a_cm)) < 1e-8 * max(1.0, abs(obj_m(Qm, a_py)))
    assert np.abs(med.A @ a_py - med.A @ a_cm).max() < 1e-5
    assert abs(float(med.E[0] @ a_cm)) < 1e-10


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_svm_gap_bounds_hold_for_any_feasible_point(seed):
    """The objective and w bounds that tests/svm_gap.py derives from a dual
    point's KKT residual hold for arbitrary box-feasible points (feasible or
    not for y^T a = 0) against the enumerated optimum, and are ~0 at it."""
    import svm_gap
    inst = _svm_tiny(seed)
    Q = inst.A.T @ inst.A
    y = inst.E[0]
    a_star, _ = O.enum_svm(Q, y, 1.0)
    f = lambda a: 0.5 * a @ Q @ a - a.sum()
    rng = np.random.default_rng(seed)
    obj0, w0, rs0, eps0, mu0 = svm_gap.point(inst, a_star)
    assert rs0 < 1e-9 and eps0 < 1e-12
    for trial in range(40):
        a = np.clip(a_star + rng.normal(scale=10.0 ** rng.uniform(-6, -1), size=a_star.size),
                    0.0, 1.0)
        if trial % 2:                       # project onto y^T a = 0 (then clip again)
            a = np.clip(a - y * (y @ a) / (y @ y), 0.0, 1.0)
        obj, w, rs, eps, mu = svm_gap.point(inst, a)
        mstar = 2.0 * max(abs(mu), abs(mu0))
        gap = f(a) - f(a_star)
        assert gap <= rs + mstar * eps + 1e-12
        assert gap >= -mstar * eps - 1e-12
        assert 0.5 * np.sum((w - w0) ** 2) <= rs + mstar * eps + 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_interior_point_svm_matches_enumeration_and_smo(seed):
    """The interior-point SVM dual solver reaches the enumerated optimum of
    tiny duals, and on medium duals the SMO optimum within the bounds both
    points' KKT residuals imply (objective and w = Z^T a)."""
    import svm_gap
    inst = _svm_tiny(seed)
    Q = inst.A.T @ inst.A
    y = inst.E[0]
    a_enum, _ = O.enum_svm(Q, y, 1.0)
    a_ipm = O.svm_ipm(inst.A.T, y, 1.0)
    obj = lambda a: 0.5 * a @ Q @ a - a.sum()
    assert abs(obj(a_ipm) - obj(a_enum)) < 1e-9
    assert np.abs(inst.A @ a_ipm - inst.A @ a_enum).max() < 1e-6
    med = synth.svm_instance(60 + seed, 500 + 200 * seed, 15 + 10 * seed)
    a_smo = O.smo_svm_c(med.A.T @ med.A, med.E[0], 1.0, tol=1e-11)
    a_ipm = O.svm_ipm(med.A.T, med.E[0], 1.0)
    P = O.problem_from_instance(med, dense_H=False)
    assert O.kkt(P, a_ipm)["kkt"] < 1e-6
    gap, gap_bound, wdist, w_bound = svm_gap.check(med, a_ipm, a_smo)
    assert gap <= gap_bound and wdist <= w_bound
    assert gap_bound < 1e-5


def test_rbf_matrix_definition():
    """The Gaussian-kernel dual matrix against a plain double loop; unit
    diagonal, symmetric, positive semidefinite, and y y^T as sigma grows."""
    import math
    rng = np.random.default_rng(11)
    X = rng.normal(size=(9, 3))
    y = rng.choice([-1.0, 1.0], size=9)
    Q = O.rbf_svm_matrix(X, y, 0.7)
    for i in range(9):
        for j in range(9):
            d2 = sum((X[i, k] - X[j, k]) ** 2 for k in range(3))
            assert abs(Q[i, j] - y[i] * y[j] * math.exp(-d2 / (2 * 0.49))) < 1e-15
    assert np.allclose(np.diag(Q), 1.0) and np.array_equal(Q, Q.T)
    assert np.linalg.eigvalsh(Q).min() > -1e-12
    assert np.abs(O.rbf_svm_matrix(X, y, 1e6) - np.outer(y, y)).max() < 1e-10


# --------------------------------------------------------------------------
# The box kept inside the block (eq. RAC-ADDM with x_i in X_i; eq. svm)
# --------------------------------------------------------------------------
def _box_enum(K, r, l, u):
    """Every pattern in {free, at l, at u}^s: the free rows solve K_FF d_F =
    -(r + K_FW d_W)_F; keep the feasible pattern whose bound multipliers have
    the right signs (the unique KKT point of a strictly convex box QP)."""
    s = len(r)
    found = []
    for pat in itertools.product((0, 1, 2), repeat=s):
        pat = np.array(pat)
        if np.any((pat == 1) & ~np.isfinite(l)) or np.any((pat == 2) & ~np.isfinite(u)):
            continue
        d = np.zeros(s)
        d[pat == 1] = l[pat == 1]
        d[pat == 2] = u[pat == 2]
        F = np.nonzero(pat == 0)[0]
        if len(F):
            W = np.nonzero(pat != 0)[0]
            rhs = -(r[F] + K[np.ix_(F, W)] @ d[W])
            d[F] = np.linalg.solve(K[np.ix_(F, F)], rhs)
        sc = 1e-9 * max(1.0, np.abs(r).max())
        if np.any(d < l - sc) or np.any(d > u + sc):
            continue
        g = K @ d + r
        if np.any(g[pat == 1] < -sc) or np.any(g[pat == 2] > sc):
            continue
        found.append(d)
    assert found, "no KKT pattern"
    for d in found[1:]:
        assert np.abs(d - found[0]).max() < 1e-8
    return found[0]


def _box_case(rng, s, cond):
    Qm, _ = np.linalg.qr(rng.normal(size=(s, s)))
    ev = np.geomspace(1.0, cond, s)
    K = (Qm * ev) @ Qm.T
    r = rng.normal(size=s) * 3.0
    l = -rng.uniform(0.0, 1.5, s)
    u = rng.uniform(0.0, 1.5, s)
    l[rng.random(s) < 0.25] = 0.0          # starts on a lower bound
    u[rng.random(s) < 0.15] = 0.0          # starts on an upper bound
    u[rng.random(s) < 0.15] = np.inf       # one-sided
    if s > 2:
        l[1] = u[1] = 0.0                  # a fixed coordinate
    return K, r, l, u


@pytest.mark.parametrize("seed", range(12))
def test_box_qp_matches_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    s = 1 + seed % 6
    K, r, l, u = _box_case(rng, s, 10.0 ** (seed % 4 + 1))
    d, state = O.box_qp(K, r, l, u)
    ref = _box_enum(K, r, l, u)
    assert np.abs(d - ref).max() <= 1e-10 * max(1.0, np.abs(ref[np.isfinite(ref)]).max())
    assert np.array_equal(d[state == 1], l[state == 1])
    assert np.array_equal(d[state == 2], u[state == 2])


def test_box_qp_diagonal_is_clipped_newton_step():
    rng = np.random.default_rng(5)
    k = rng.uniform(0.5, 4.0, 30)
    r = rng.normal(size=30)
    l, u = -rng.uniform(0, 1, 30), rng.uniform(0, 1, 30)
    d, _ = O.box_qp(np.diag(k), r, l, u)
    assert np.abs(d - np.clip(-r / k, l, u)).max() < 1e-15


def test_box_qp_kkt_at_size_and_clipping_is_not_enough():
    """s = 80, condition 1e4: the optimality conditions of a box QP hold to
    rounding; the clipped unconstrained minimiser (a plausible shortcut)
    violates them on the same instance."""
    rng = np.random.default_rng(9)
    K, r, l, u = _box_case(rng, 80, 1e4)
    d, state = O.box_qp(K, r, l, u)
    g = K @ d + r
    sc = 1e-10 * max(1.0, np.abs(r).max())
    assert np.all(d >= l) and np.all(d <= u)
    assert np.abs(g[state == 0]).max() <= sc
    movable = u > l
    assert np.all(g[(state == 1) & movable] >= -sc)
    assert np.all(g[(state == 2) & movable] <= sc)
    dc = np.clip(np.linalg.solve(K, -r), l, u)
    gc = K @ dc + r
    inside = (dc > l) & (dc < u)
    assert np.abs(gc[inside]).max() > 1e-3


def test_box_sweep_with_unit_blocks_is_projected_coordinate_descent():
    """Blocks of one coordinate: the literal box step is the clipped exact
    line minimisation along that coordinate, taken in the assembled order."""
    rng = np.random.default_rng(3)
    n = 12
    B = rng.normal(size=(20, n))
    H = B.T @ B
    q = rng.normal(size=n)
    e = rng.choice([-1.0, 1.0], size=(1, n))
    P = O.Problem(H=H, q=q, phi="box", lo=0.0, hi=0.8, E=e, d=np.zeros(1))
    st = O.initial_state(P)
    x, mu = np.zeros(n), np.zeros(1)
    beta, gamma = 0.7, 0.3
    for k in range(6):
        order = np.concatenate(O.random_assembly(n, n, 4, k))
        O.sweep(P, st, n, 4, beta, gamma, box_qp=True)
        for j in order:
            g = H[j] @ x + q[j] + e[0, j] * (beta * (e[0] @ x) - mu[0])
            x[j] = min(max(x[j] - g / (H[j, j] + beta + gamma), 0.0), 0.8)
        mu = mu - beta * (e[0] @ x)
        assert np.abs(st.x - x).max() < 1e-13
        assert np.array_equal(st.z, st.x) and not st.xi.any()
        assert abs(st.mu[0] - mu[0]) < 1e-13


@pytest.mark.parametrize("gamma", [0.0, 0.5])
@pytest.mark.parametrize("seed", [0, 1])
def test_box_sweep_svm_converges_to_enumeration(seed, gamma):
    """Gaussian-kernel C-SVC dual (eq. svm, Sec. 3.2): the literal box-block
    iteration converges to the enumerated optimum; every iterate is in the box."""
    rng = np.random.default_rng(40 + seed)
    X = rng.normal(size=(7, 2))
    y = np.where(X[:, 0] + 0.3 * rng.normal(size=7) > 0, 1.0, -1.0)
    C = 1.0
    Q = O.rbf_svm_matrix(X, y, 1.0)
    P = O.Problem(H=Q, q=-np.ones(7), phi="box", lo=0.0, hi=C, E=y[None, :], d=np.zeros(1))
    a_enum, _ = O.enum_svm(Q, y, C)
    st = O.initial_state(P)
    for _ in range(3000):
        O.sweep(P, st, 3, seed, 0.3, gamma, box_qp=True)
        assert np.all(st.x >= 0.0) and np.all(st.x <= C)
    assert np.abs(st.x - a_enum).max() < 1e-8
    assert O.kkt(P, st.x, mu=st.mu)["kkt"] < 1e-9
