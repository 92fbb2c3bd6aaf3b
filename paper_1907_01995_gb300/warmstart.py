"""Learned warm start (form (4)): per-coordinate MLP trained on the solver's
own solutions.  Argument marshalling only; features, the network's forward
and backward passes, Adam and the decode run in the CUDA library."""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib as L
from .api import _stream_handle

F, H, O = 6, 128, 2


def num_params() -> int:
    return int(L.load().rac_ws_num_params())


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-uniform initial weights, zero biases (layout W1 b1 W2 b2 W3 b3)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for fan_in, fan_out in ((F, H), (H, H), (H, O)):
        bound = math.sqrt(6.0 / fan_in)
        parts.append((torch.rand((fan_out, fan_in), generator=g) * 2 - 1) * bound)
        parts.append(torch.zeros(fan_out))
    p = torch.cat([t.reshape(-1) for t in parts]).to(torch.float32)
    assert p.numel() == num_params()
    return p.to(device)


def _colmajor(A):
    if A.stride(0) != 1:
        A = A.t().contiguous().t()
    return A


def features(A: torch.Tensor, b: torch.Tensor, lam1: float, lam2: float, xstar=None):
    """(F (n x 6), T (n x 2) or None, lambda_max) for a device problem."""
    A = _colmajor(A.to(torch.float64))
    m, n = A.shape
    Fx = torch.empty((n, F), dtype=torch.float32, device=A.device)
    T = None
    lmax = ctypes.c_double(0.0)
    st = _stream_handle(None)
    if xstar is None:
        L.check(L.load().rac_ws_features(m, n, A.data_ptr(), A.stride(1), b.data_ptr(),
                                         float(lam1), float(lam2), Fx.data_ptr(),
                                         ctypes.byref(lmax), st), "rac_ws_features")
    else:
        xs = xstar.to(torch.float64).contiguous()
        T = torch.empty((n, 2), dtype=torch.float32, device=A.device)
        L.check(L.load().rac_ws_features_targets(m, n, A.data_ptr(), A.stride(1), b.data_ptr(),
                                                 float(lam1), float(lam2), Fx.data_ptr(),
                                                 xs.data_ptr(), T.data_ptr(), ctypes.byref(lmax),
                                                 st), "rac_ws_features_targets")
    return Fx, T, lmax.value


def forward(Fx: torch.Tensor, params: torch.Tensor) -> torch.Tensor:
    out = torch.empty((Fx.shape[0], O), dtype=torch.float32, device=Fx.device)
    L.check(L.load().rac_ws_forward(Fx.shape[0], Fx.data_ptr(), params.data_ptr(),
                                    out.data_ptr(), _stream_handle(None)), "rac_ws_forward")
    return out


def loss_grad(Fx, T, params):
    grad = torch.empty_like(params)
    loss = ctypes.c_float(0.0)
    L.check(L.load().rac_ws_loss_grad(Fx.shape[0], Fx.data_ptr(), T.data_ptr(),
                                      params.data_ptr(), grad.data_ptr(), ctypes.byref(loss),
                                      _stream_handle(None)), "rac_ws_loss_grad")
    return loss.value, grad


class Trainer:
    """Adam on the device (rac_ws_train_step); minibatches are row subsets."""

    def __init__(self, params: torch.Tensor, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        self.p = params
        self.g = torch.zeros_like(params)
        self.m1 = torch.zeros_like(params)
        self.m2 = torch.zeros_like(params)
        self.lr, self.b1, self.b2, self.eps = lr, betas[0], betas[1], eps
        self.step = 0

    def train_step(self, Fx, T) -> float:
        self.step += 1
        loss = ctypes.c_float(0.0)
        L.check(L.load().rac_ws_train_step(Fx.shape[0], Fx.data_ptr(), T.data_ptr(),
                                           self.p.data_ptr(), self.g.data_ptr(),
                                           self.m1.data_ptr(), self.m2.data_ptr(), self.step,
                                           self.lr, self.b1, self.b2, self.eps,
                                           ctypes.byref(loss), _stream_handle(None)),
                "rac_ws_train_step")
        return loss.value

    def fit(self, Fx, T, epochs=20, batch=4096, seed=0):
        g = torch.Generator(device=Fx.device).manual_seed(seed)
        N = Fx.shape[0]
        hist = []
        for _ in range(epochs):
            order = torch.randperm(N, generator=g, device=Fx.device)
            tot = 0.0
            for s in range(0, N, batch):
                idx = order[s:s + batch]
                tot += self.train_step(Fx[idx].contiguous(), T[idx].contiguous()) * idx.numel()
            hist.append(tot / N)
        return hist


def predict(A: torch.Tensor, b: torch.Tensor, lam1: float, lam2: float,
            params: torch.Tensor) -> torch.Tensor:
    """Decoded warm start x0 (device, float64)."""
    A = _colmajor(A.to(torch.float64))
    m, n = A.shape
    x0 = torch.empty(n, dtype=torch.float64, device=A.device)
    L.check(L.load().rac_ws_predict(m, n, A.data_ptr(), A.stride(1), b.data_ptr(), float(lam1),
                                    float(lam2), params.data_ptr(), x0.data_ptr(),
                                    _stream_handle(None)), "rac_ws_predict")
    return x0
