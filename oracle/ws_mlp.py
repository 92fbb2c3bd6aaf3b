"""FP64 reference of the learned warm-start network (test infrastructure only).

The per-coordinate MLP 6 -> 128 -> 128 -> 2 with ReLU, its loss
(u - t0)^2 + BCE-with-logits(logit, t1) averaged over the samples, the
gradient by the chain rule, one Adam step, and the feature / target map.
The learned part has no counterpart in the paper; these functions are the
plain definitions and are pinned by finite differences and closed forms in
tests/test_oracle_ws.py.
"""
from __future__ import annotations

import numpy as np

F, H, O = 6, 128, 2
SHAPES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)),
          ("b3", (O,))]


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = p[o:o + k].reshape(shp)
        o += k
    assert o == p.size
    return out


def pack(d):
    return np.concatenate([d[name].reshape(-1) for name, _ in SHAPES])


def forward(X, p):
    w = unpack(p)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ w["W3"].T + w["b3"]
    return out, (X, a1, h1, a2, h2)


def loss(X, T, p):
    out, _ = forward(X, p)
    o0, o1 = out[:, 0], out[:, 1]
    sp = np.logaddexp(0.0, o1)
    return float(np.mean((o0 - T[:, 0]) ** 2 + sp - T[:, 1] * o1))


def loss_grad(X, T, p):
    w = unpack(p)
    out, (X, a1, h1, a2, h2) = forward(X, p)
    N = X.shape[0]
    o0, o1 = out[:, 0], out[:, 1]
    d = np.stack([2.0 * (o0 - T[:, 0]), 1.0 / (1.0 + np.exp(-o1)) - T[:, 1]], axis=1) / N
    g = {"W3": d.T @ h2, "b3": d.sum(0)}
    dh2 = (d @ w["W3"]) * (a2 > 0)
    g["W2"], g["b2"] = dh2.T @ h1, dh2.sum(0)
    dh1 = (dh2 @ w["W2"]) * (a1 > 0)
    g["W1"], g["b1"] = dh1.T @ X, dh1.sum(0)
    return loss(X, T, p), pack(g)


def adam_step(p, g, m1, m2, step, lr, b1, b2, eps):
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2


def features_targets(A, b, lam1, lam2, xstar=None):
    """Features [A_j^T b / (||A_j|| lmax), ||A_j||, lam1/lmax, lam2, |A_j^T b|/lam1,
    log(n/m)] and targets [x*_j ||A_j|| / lmax, x*_j != 0]."""
    m, n = A.shape
    nrm = np.sqrt((A * A).sum(0))
    atb = A.T @ b
    lmax = np.abs(atb).max()
    Fx = np.stack([atb / (nrm * lmax), nrm, np.full(n, lam1 / lmax), np.full(n, lam2),
                   np.minimum(np.abs(atb) / lam1, 1e6), np.full(n, np.log(n / m))], axis=1)
    T = None
    if xstar is not None:
        T = np.stack([xstar * nrm / lmax, (xstar != 0).astype(np.float64)], axis=1)
    return Fx, T, lmax
