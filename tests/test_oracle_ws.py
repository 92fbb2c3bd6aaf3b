"""Pins of the FP64 warm-start network reference (CPU)."""
import numpy as np

from oracle import ws_mlp as W


def _params(seed=0):
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in W.SHAPES:
        d[name] = rng.normal(size=shp) * (0.4 if name.startswith("W") else 0.1)
    return W.pack(d)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(9, W.F))
    T = np.stack([rng.normal(size=9), (rng.random(9) < 0.5).astype(float)], axis=1)
    p = _params(2)
    _, g = W.loss_grad(X, T, p)
    idx = rng.choice(p.size, size=60, replace=False)
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (W.loss(X, T, pp) - W.loss(X, T, pm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))


def test_forward_closed_form_linear_region():
    """With all pre-activations positive the network is the product of its
    affine maps."""
    p = _params(3)
    w = W.unpack(p)
    w["b1"][:] = 100.0
    w["b2"][:] = 1000.0
    w["W2"] = np.abs(w["W2"])
    p = W.pack(w)
    X = np.random.default_rng(4).normal(size=(5, W.F)) * 0.1
    out, _ = W.forward(X, p)
    lin = ((X @ w["W1"].T + w["b1"]) @ w["W2"].T + w["b2"]) @ w["W3"].T + w["b3"]
    assert np.allclose(out, lin)


def test_adam_first_step_is_sign_step():
    g = np.array([0.3, -2.0, 1e-3])
    p = np.zeros(3)
    p1, _, _ = W.adam_step(p, g, np.zeros(3), np.zeros(3), 1, 0.01, 0.9, 0.999, 1e-12)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-6)


def test_features_orthogonal_design():
    """On an orthonormal design the features read off A^T b directly and the
    targets of the closed-form solution soft(A^T b, lam1) / (1 + lam2)."""
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(40, 12)))
    b = rng.normal(size=40)
    lam1, lam2 = 0.3, 0.1
    x = np.sign(Q.T @ b) * np.maximum(np.abs(Q.T @ b) - lam1, 0) / (1 + lam2)
    Fx, T, lmax = W.features_targets(Q, b, lam1, lam2, x)
    assert np.isclose(lmax, np.abs(Q.T @ b).max())
    assert np.allclose(Fx[:, 1], 1.0)
    assert np.allclose(Fx[:, 0] * lmax, Q.T @ b)
    assert np.array_equal(T[:, 1] == 1, Fx[:, 4] > 1.0)
