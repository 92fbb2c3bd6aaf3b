"""Python front end of the RAC-MBADMM CUDA library (argument marshalling only).

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); the
library reads them through plain pointers and copies them into its own device
buffers.  A scipy.sparse data matrix is passed as compressed columns.  torch
is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _lib as L

try:  # torch is optional for callers that pass numpy arrays
    import torch
except Exception:  # pragma: no cover
    torch = None


def _is_tensor(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


class _Keep:
    """Holds converted arrays alive while the C call reads them."""

    def __init__(self):
        self.items = []

    def vec(self, a, n: Optional[int] = None):
        if a is None:
            return None
        if _is_tensor(a):
            if a.dtype == torch.float64 and a.is_contiguous():
                t = a   # read in place (a contiguous tensor is one flat buffer)
            else:
                t = a.detach().to(torch.float64).contiguous().reshape(-1)
            if n is not None and t.numel() != n:
                raise ValueError("vector length %d, expected %d" % (t.numel(), n))
            self.items.append(t)
            return t.data_ptr()
        v = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
        if n is not None and v.size != n:
            raise ValueError("vector length %d, expected %d" % (v.size, n))
        self.items.append(v)
        return v.ctypes.data

    def colmajor(self, a):
        """(pointer, rows, cols, ld) of a 2-D array in column-major float64."""
        if _is_tensor(a):
            t = a if a.dtype == torch.float64 else a.detach().to(torch.float64)
            if not (t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0])):
                t = t.detach().t().contiguous().t()
            self.items.append(t)
            return t.data_ptr(), t.shape[0], t.shape[1], max(1, t.stride(1))
        m = np.asfortranarray(np.asarray(a, dtype=np.float64))
        self.items.append(m)
        return m.ctypes.data, m.shape[0], m.shape[1], max(1, m.shape[0])


_CUDA = None   # torch.cuda.is_available(), asked once per process


def _stream_handle(stream) -> int:
    global _CUDA
    if stream is None:
        if _CUDA is None:
            _CUDA = torch is not None and torch.cuda.is_available()
        if _CUDA:
            return torch.cuda.current_stream().cuda_stream
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_problem(keep: _Keep, A=None, b=None, *, H=None, c=None, E=None, d=None, phi="none",
                 lambda1=0.0, lambda2=0.0, lo=0.0, hi=0.0) -> L.RacProblem:
    pr = L.RacProblem()
    if A is not None and hasattr(A, "tocsc") and not _is_tensor(A):
        # scipy.sparse matrix: compressed columns (sorted, duplicates summed)
        Ac = A.tocsc(copy=True)
        Ac.sum_duplicates()
        Ac.sort_indices()
        pr.m, pr.n = int(Ac.shape[0]), int(Ac.shape[1])
        colptr = np.ascontiguousarray(Ac.indptr, dtype=np.int64)
        rowidx = np.ascontiguousarray(Ac.indices, dtype=np.int32)
        vals = np.ascontiguousarray(Ac.data, dtype=np.float64)
        keep.items.extend([colptr, rowidx, vals])
        pr.nnz = int(vals.size)
        pr.colptr, pr.rowidx = colptr.ctypes.data, rowidx.ctypes.data
        if not vals.size:          # an all-zero matrix still passes a values pointer
            vals = np.zeros(1)
            keep.items.append(vals)
        pr.vals = vals.ctypes.data
        pr.b = keep.vec(b, pr.m)
    elif A is not None:
        pr.A, pr.m, pr.n, pr.lda = keep.colmajor(A)
        pr.b = keep.vec(b, pr.m)
    elif H is not None:
        pr.H, n1, n2, ld = keep.colmajor(H)
        if n1 != n2 or ld != n1:
            raise ValueError("H must be square")
        pr.m, pr.n, pr.lda = 0, n1, 0
    else:
        raise ValueError("need A or H")
    pr.c = keep.vec(c, pr.n)
    if E is not None:
        Ek = E if _is_tensor(E) else np.asarray(E, dtype=np.float64)
        k = 1 if Ek.ndim == 1 else int(Ek.shape[0])
        pr.E = keep.vec(Ek, k * pr.n)        # k x n row-major
        pr.d = keep.vec(np.zeros(k) if d is None else d, k)
        pr.k = k
    pr.phi = L.PHI[phi]
    pr.lambda1, pr.lambda2, pr.lo, pr.hi = float(lambda1), float(lambda2), float(lo), float(hi)
    return pr


def make_options(keep: _Keep, n: int, *, num_blocks=1, beta=1.0, gamma=0.0, tol=1e-6,
                 max_sweeps=1000, refresh_every=10, seed=0, storage="fp64", form="auto",
                 grid=0, x0=None, xi0=None, stream=None, profile=False, xi0_from_grad=False,
                 ws_fallback=False, chain="auto", assembly="rac",
                 debug_exit_cta=0, path="auto", box_qp=False, box_prox=0.0) -> L.RacOptions:
    o = L.RacOptions()
    L.load().rac_options_default(ctypes.byref(o))
    o.num_blocks = int(num_blocks)
    o.beta, o.gamma, o.tol = float(beta), float(gamma), float(tol)
    o.max_sweeps, o.refresh_every = int(max_sweeps), int(refresh_every)
    o.seed = int(seed)
    o.storage = L.STORAGE[storage]
    o.form = L.FORM[form]
    o.grid = int(grid)
    o.x0 = keep.vec(x0, n)
    o.xi0 = keep.vec(xi0, n)
    o.stream = _stream_handle(stream)
    o.profile = 1 if profile else 0
    o.xi0_from_grad = int(xi0_from_grad)
    o.ws_fallback = 1 if ws_fallback else 0
    o.chain = L.CHAIN[chain]
    o.assembly = L.ASSEMBLY[assembly]
    o.debug_exit_cta = int(debug_exit_cta)
    o.path = L.PATH[path]
    o.box_qp = 1 if box_qp else 0
    o.box_prox = float(box_prox)
    return o


def _info_dict(info: L.RacInfo) -> dict:
    return {"sweeps": info.sweeps, "block_updates": info.block_updates, "kkt": info.kkt,
            "primal_res": info.primal_res, "mu": info.mu, "seconds": info.seconds,
            "status": info.status, "form": info.form.decode(),
            "kernel_launches": info.kernel_launches, "setup_launches": info.setup_launches,
            "t_assembly_ms": info.t_assembly_ms, "t_factor_ms": info.t_factor_ms,
            "t_chain_ms": info.t_chain_ms, "t_prox_ms": info.t_prox_ms,
            "t_refresh_ms": info.t_refresh_ms, "chain_launches": info.chain_launches,
            "warm_start_rejected": info.warm_start_rejected, "t_loop_ms": info.t_loop_ms,
            "obj": info.obj, "box_iters": info.box_iters, "box_capped": info.box_capped}


class Handle:
    """A set-up problem on the GPU (rac_admm_setup ... rac_admm_destroy)."""

    def __init__(self, A=None, b=None, *, H=None, c=None, E=None, d=None, phi="none",
                 lambda1=0.0, lambda2=0.0, lo=0.0, hi=0.0, **opts):
        self._lib = L.load()
        keep = _Keep()
        self.problem = make_problem(keep, A, b, H=H, c=c, E=E, d=d, phi=phi, lambda1=lambda1,
                                    lambda2=lambda2, lo=lo, hi=hi)
        self.n = int(self.problem.n)
        self.options = make_options(keep, self.n, **opts)
        self.num_blocks = int(self.options.num_blocks)
        h = ctypes.c_void_p()
        L.check(self._lib.rac_admm_setup(ctypes.byref(self.problem), ctypes.byref(self.options),
                                         ctypes.byref(h)), "rac_admm_setup")
        self._h = h
        self._stream = self.options.stream
        del keep

    def _out(self, out, n):
        if out is None:
            return np.empty(n, dtype=np.float64), None
        if _is_tensor(out):
            if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != n:
                raise ValueError("out must be a contiguous float64 tensor of %d entries" % n)
            return out, out.data_ptr()
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != n:
            raise ValueError("out must be a contiguous float64 array of %d entries" % n)
        return out, out.ctypes.data

    def solve(self, out=None, *, raise_not_converged: bool = False):
        out, ptr = self._out(out, self.n)
        if ptr is None:
            ptr = out.ctypes.data
        info = L.RacInfo()
        st = self._lib.rac_admm_solve(self._h, ptr, ctypes.byref(info))
        allow = (L.RAC_OK,) if raise_not_converged else (L.RAC_OK, L.RAC_ERR_NOT_CONVERGED)
        L.check(st, "rac_admm_solve", allow)
        return out, _info_dict(info)

    def reset(self, x0=None, xi0=None):
        keep = _Keep()
        L.check(self._lib.rac_admm_reset(self._h, keep.vec(x0, self.n), keep.vec(xi0, self.n)),
                "rac_admm_reset")

    def state(self):
        """Current iterates; "mu" is the multiplier (k = 1) or the array of k."""
        x, z, xi = (np.empty(self.n) for _ in range(3))
        k = max(1, int(self.problem.k))
        mu = np.zeros(k)
        L.check(self._lib.rac_admm_get_state(self._h, x.ctypes.data, z.ctypes.data,
                                             xi.ctypes.data, mu.ctypes.data),
                "rac_admm_get_state")
        return {"x": x, "z": z, "xi": xi, "mu": mu[0] if k == 1 else mu}

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t(0)
        L.check(self._lib.rac_admm_checkpoint(self._h, None, ctypes.byref(n)), "checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        L.check(self._lib.rac_admm_checkpoint(self._h, buf, ctypes.byref(n)), "checkpoint")
        return buf.raw[:n.value]

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        L.check(self._lib.rac_admm_restore(self._h, buf, len(blob)), "restore")

    def path(self, lambda1: Sequence[float], lambda2: Optional[Sequence[float]] = None):
        """Regularisation path (rac_admm_path): lambda2 None keeps the handle's
        lambda2 for every point.  Returns (X with column l = point l's z, infos)."""
        lam1 = np.ascontiguousarray(np.asarray(lambda1, dtype=np.float64))
        nl = lam1.size
        lam2 = None if lambda2 is None else np.ascontiguousarray(
            np.asarray(lambda2, dtype=np.float64))
        if lam2 is not None and lam2.size != nl:
            raise ValueError("lambda2 needs %d entries" % nl)
        X = np.empty((nl, self.n), dtype=np.float64)   # row l = column l of n x nl col-major
        infos = (L.RacInfo * nl)()
        st = self._lib.rac_admm_path(self._h, nl, lam1.ctypes.data,
                                     None if lam2 is None else lam2.ctypes.data,
                                     X.ctypes.data, infos)
        L.check(st, "rac_admm_path", (L.RAC_OK, L.RAC_ERR_NOT_CONVERGED))
        return X.T.copy(), [_info_dict(i) for i in infos]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rac_admm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve(A=None, b=None, **kw):
    """One-shot setup + solve + destroy.  Returns (z, info)."""
    with Handle(A, b, **kw) as h:
        return h.solve()


def batch(problems, *, out=None, allow=(L.RAC_OK, L.RAC_ERR_NOT_CONVERGED), **opts):
    """Solve independent data-form problems (dicts of make_problem arguments)
    together, one graph of batched kernels per refresh period
    (rac_admm_batch).  Returns (list of z, infos);
    raises unless the call's status is in `allow` (per-problem statuses are
    in infos[i]["status"])."""
    lib = L.load()
    keep = _Keep()
    cnt = len(problems)
    probs = (L.RacProblem * cnt)()
    for i, p in enumerate(problems):
        probs[i] = make_problem(keep, **p)
    o = make_options(keep, 1, **opts)
    outs = [np.empty(int(probs[i].n)) for i in range(cnt)] if out is None else out
    ptrs = (ctypes.c_void_p * cnt)(*[
        (o_.data_ptr() if _is_tensor(o_) else o_.ctypes.data) for o_ in outs])
    infos = (L.RacInfo * cnt)()
    st = lib.rac_admm_batch(cnt, probs, ctypes.byref(o), ptrs, infos)
    L.check(st, "rac_admm_batch", allow)
    return outs, [_info_dict(i) for i in infos]


def assembly(n: int, num_blocks: int, seed: int, sweep0: int, nsweeps: int, stream=None):
    """Random assembly of sweeps sweep0.. (device int32 tensors perm, blk)."""
    lib = L.load()
    perm = torch.empty((nsweeps, n), dtype=torch.int32, device="cuda")
    blk = torch.empty((nsweeps, n), dtype=torch.int32, device="cuda")
    L.check(lib.rac_assembly(n, num_blocks, seed, sweep0, nsweeps, perm.data_ptr(),
                             blk.data_ptr(), _stream_handle(stream)), "rac_assembly")
    return perm, blk


def trim_pool():
    """Return the cached, unused device memory of closed handles to the driver."""
    L.check(L.load().rac_trim_pool(), "rac_trim_pool")


def rbf_svm_matrix(X, y, sigma: float, stream=None):
    """Q = diag(y) K diag(y) with the Gaussian kernel K_ij = exp(-||x_i -
    x_j||^2 / (2 sigma^2)) on the GPU (rac_rbf_gram).  X: N x d samples (host
    or device), y: N labels.  Returns Q as an N x N float64 CUDA tensor, the
    H of the C-SVC dual (with c = -1, E = y, box [0, C])."""
    Xt = torch.as_tensor(X, dtype=torch.float64, device="cuda").contiguous()  # N x d row-major
    yt = torch.as_tensor(y, dtype=torch.float64, device="cuda").contiguous()
    N, d = int(Xt.shape[0]), int(Xt.shape[1])
    Q = torch.empty((N, N), dtype=torch.float64, device="cuda")
    # row-major N x d is column-major d x N with leading dimension d
    L.check(L.load().rac_rbf_gram(N, d, Xt.data_ptr(), d, yt.data_ptr(), float(sigma),
                                  Q.data_ptr(), _stream_handle(stream)), "rac_rbf_gram")
    return Q
