"""ctypes declarations of the C-ABI in include/rac_admm.h.

Argument marshalling only: every step of the method runs in the CUDA library.
If the library has not been built the import of the binding fails loudly;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librac_admm.so")

c_int32, c_int64, c_uint64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
c_double, c_void_p, c_size_t = ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
c_float = ctypes.c_float

RAC_OK, RAC_ERR_ARG, RAC_ERR_CUDA, RAC_ERR_OOM = 0, 1, 2, 3
RAC_ERR_NOT_PD, RAC_ERR_NUMERIC, RAC_ERR_TIMEOUT = 4, 5, 6
RAC_ERR_NOT_CONVERGED, RAC_ERR_STATE = 7, 8
PHI = {"none": 0, "l1l2": 1, "box": 2}
STORAGE = {"fp64": 0, "fp32": 1, "bf16": 2}
CHAIN = {"auto": 0, "grid": 1, "cluster": 2}
ASSEMBLY = {"rac": 0, "rp": 1}
FORM = {"auto": 0, "gram": 1, "residual": 2}
PATH = {"auto": 0, "sequential": 1, "batched": 2}


class RacProblem(ctypes.Structure):
    _fields_ = [("m", c_int64), ("n", c_int64), ("A", c_void_p), ("lda", c_int64),
                ("b", c_void_p), ("H", c_void_p), ("c", c_void_p), ("E", c_void_p),
                ("d", c_void_p), ("k", c_int32), ("phi", c_int32), ("lambda1", c_double),
                ("lambda2", c_double), ("lo", c_double), ("hi", c_double),
                ("nnz", c_int64), ("colptr", c_void_p), ("rowidx", c_void_p), ("vals", c_void_p)]


class RacOptions(ctypes.Structure):
    _fields_ = [("num_blocks", c_int32), ("beta", c_double), ("gamma", c_double),
                ("tol", c_double), ("max_sweeps", c_int32), ("refresh_every", c_int32),
                ("seed", c_uint64), ("storage", c_int32), ("form", c_int32), ("grid", c_int32),
                ("x0", c_void_p), ("xi0", c_void_p), ("stream", c_void_p), ("profile", c_int32),
                ("xi0_from_grad", c_int32), ("ws_fallback", c_int32), ("chain", c_int32),
                ("assembly", c_int32), ("debug_exit_cta", c_int32), ("path", c_int32),
                ("box_qp", c_int32), ("box_prox", c_double)]


class RacInfo(ctypes.Structure):
    _fields_ = [("sweeps", c_int32), ("block_updates", c_int64), ("kkt", c_double),
                ("primal_res", c_double), ("mu", c_double), ("seconds", c_double),
                ("status", c_int32), ("form", ctypes.c_char * 32),
                ("kernel_launches", c_int64), ("setup_launches", c_int64),
                ("t_assembly_ms", c_double), ("t_factor_ms", c_double), ("t_chain_ms", c_double),
                ("t_prox_ms", c_double), ("t_refresh_ms", c_double), ("chain_launches", c_int64),
                ("warm_start_rejected", c_int32), ("t_loop_ms", c_double), ("obj", c_double),
                ("box_iters", c_int64), ("box_capped", c_int64)]


P = ctypes.POINTER
# (name, restype, argtypes) of every exported function
SIGNATURES = [
    ("rac_status_string", ctypes.c_char_p, [c_int32]),
    ("rac_last_error", ctypes.c_char_p, []),
    ("rac_trim_pool", c_int32, []),
    ("rac_options_default", c_int32, [P(RacOptions)]),
    ("rac_admm_setup", c_int32, [P(RacProblem), P(RacOptions), P(c_void_p)]),
    ("rac_admm_solve", c_int32, [c_void_p, c_void_p, P(RacInfo)]),
    ("rac_admm_reset", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("rac_admm_get_state", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rac_admm_batch", c_int32, [c_int32, P(RacProblem), P(RacOptions), P(c_void_p), P(RacInfo)]),
    ("rac_admm_path", c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, P(RacInfo)]),
    ("rac_admm_checkpoint", c_int32, [c_void_p, c_void_p, P(c_size_t)]),
    ("rac_admm_restore", c_int32, [c_void_p, c_void_p, c_size_t]),
    ("rac_admm_destroy", None, [c_void_p]),
    ("rac_assembly", c_int32, [c_int64, c_int32, c_uint64, c_int64, c_int32, c_void_p, c_void_p,
                               c_void_p]),
    ("rac_gram", c_int32, [c_int64, c_int64, c_void_p, c_int64, c_int32, c_void_p, c_void_p]),
    ("rac_rbf_gram", c_int32, [c_int64, c_int64, c_void_p, c_int64, c_void_p, c_double,
                               c_void_p, c_void_p]),
    ("rac_assembly_noalloc", c_int32, [c_int64, c_int32, c_uint64, c_int64, c_int32, c_void_p,
                                       c_void_p, c_void_p]),
    ("rac_ws_num_params", c_int64, []),
    ("rac_ws_features", c_int32, [c_int64, c_int64, c_void_p, c_int64, c_void_p, c_double,
                                  c_double, c_void_p, P(c_double), c_void_p]),
    ("rac_ws_features_targets", c_int32, [c_int64, c_int64, c_void_p, c_int64, c_void_p, c_double,
                                          c_double, c_void_p, c_void_p, c_void_p, P(c_double),
                                          c_void_p]),
    ("rac_ws_forward", c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rac_ws_predict", c_int32, [c_int64, c_int64, c_void_p, c_int64, c_void_p, c_double, c_double,
                                 c_void_p, c_void_p, c_void_p]),
    ("rac_ws_train_step", c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_int32, c_float, c_float, c_float, c_float,
                                    P(c_float), c_void_p]),
    ("rac_ws_loss_grad", c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, P(c_float),
                                   c_void_p]),
]

_LIB = None


class RacError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        detail = ""
        if status == RAC_ERR_CUDA:
            try:
                detail = " [%s]" % load().rac_last_error().decode()
            except Exception:
                pass
        super().__init__("%s: status %d (%s)%s" % (where, status, status_string(status), detail))


def load() -> ctypes.CDLL:
    """Load the CUDA library (raises if it is missing: no fallback path)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("RAC-MBADMM CUDA library not built (%s); run "
                               "__graft_entry__.build() or python -m "
                               "paper_1907_01995_gb300.build" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def status_string(status: int) -> str:
    try:
        return load().rac_status_string(int(status)).decode()
    except Exception:  # the library may be absent when formatting an error
        return "status %d" % status


def check(status: int, where: str, allow=(RAC_OK,)) -> int:
    if status not in allow:
        raise RacError(status, where)
    return status
