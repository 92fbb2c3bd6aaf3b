"""Autotuner: pick the storage precision, gradient form and sweep-kernel grid.

Each candidate is timed end to end (setup + solve to the requested KKT
tolerance) on the caller's problem; candidates that fail or do not converge
are dropped.  Results are cached per (GPU, library build, workload key) in a
JSON file (RAC_AUTOTUNE_CACHE, default ~/.cache/rac_admm/autotune.json).
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import _lib
from . import api

DEFAULT_CANDIDATES = [("fp32", "gram"), ("bf16", "gram"), ("fp32", "residual"),
                      ("bf16", "residual")]
DEFAULT_GRIDS = {"gram": [0, 16, 32, 64, 152], "residual": [0, 64, 152]}


def _cache_path() -> str:
    return os.environ.get("RAC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "rac_admm",
                                       "autotune.json"))


def _build_id() -> str:
    try:
        with open(_lib.LIB_PATH, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return "unbuilt"


def _gpu_name(device) -> str:
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:
        return "gpu"


def _time_solve(A, b, common, storage, form, grid, reps=2):
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        try:
            with api.Handle(A, b, storage=storage, form=form, grid=grid, **common) as h:
                _, info = h.solve()
        except _lib.RacError:
            return None
        dt = time.perf_counter() - t0
        if info["status"] != 0:
            return None
        best = dt if best is None else min(best, dt)
    return best


def choose(A, b, common: dict, key: str, device=None, candidates=None, grids=None,
           use_cache: bool = True) -> dict:
    """Return {"storage", "form", "grid", "seconds", "table"} for the fastest
    candidate on this problem."""
    candidates = candidates or DEFAULT_CANDIDATES
    grids = grids or DEFAULT_GRIDS
    ck = "%s|%s|%s" % (_gpu_name(device), _build_id(), key)
    path = _cache_path()
    cache = {}
    if use_cache:
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if ck in cache:
            return cache[ck]
    table = []
    for storage, form in candidates:
        for g in grids[form]:
            t = _time_solve(A, b, common, storage, form, g)
            table.append({"storage": storage, "form": form, "grid": g, "seconds": t})
    ok = [r for r in table if r["seconds"] is not None]
    if not ok:
        raise RuntimeError("no autotuner candidate converged")
    best = min(ok, key=lambda r: r["seconds"])
    res = dict(best)
    res["table"] = table
    if use_cache:
        cache[ck] = res
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return res
