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


# ---------------------------------------------------------------- batched form
BATCH_CANDIDATES = [(32, "rac", "bf16"), (64, "rac", "bf16"), (128, "rac", "bf16"),
                    (32, "rp", "bf16"), (64, "rp", "bf16"), (128, "rp", "bf16"),
                    (64, "rp", "fp32")]


def batch_sample(work, count):
    """Indices of `count` instances spread over the work quantiles (sorted by
    work, evenly spaced ranks), so that the sample keeps the batch's mix of
    small and large instances."""
    order = sorted(range(len(work)), key=lambda i: (work[i], i))
    if count >= len(order):
        return order
    return sorted({order[int(round(k * (len(order) - 1) / (count - 1)))] for k in range(count)})


def choose_batch(probs, common: dict, key: str, device=None, candidates=None, sample=8,
                 budget_s=2.0, use_cache: bool = True) -> dict:
    """Block size, assembly (RAC or RP) and storage for rac_admm_batch on this
    family.  Every candidate gets the same device-time budget on the same
    stratified sample of the problems (batch_sample): a 30-sweep run measures
    its time per sweep, then it runs as many sweeps as the budget buys, and
    it is scored by the geometric mean of the sample's KKT measures at the
    end (so a candidate with cheaper sweeps, or with more progress per sweep,
    wins).  Time to a fixed tolerance cannot rank these duals at full size:
    the split iteration needs more than 10^4 sweeps to reach KKT 1e-3 on the
    largest ones.  Returns {"block", "assembly", "storage", "score",
    "table"}; cached per (GPU, library build, key) like choose()."""
    import math
    candidates = candidates or BATCH_CANDIDATES
    ck = "%s|%s|batch|%s" % (_gpu_name(device), _build_id(), key)
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
    work = [int(p["A"].shape[0]) * int(p["A"].shape[1]) for p in probs]
    pick = batch_sample(work, sample)
    sub = [probs[i] for i in pick]
    table = []
    for block, assembly, storage in candidates:
        kw = dict(common)
        kw.update(num_blocks=-block, assembly=assembly, storage=storage, tol=0.0)
        try:
            _, probe = api.batch(sub, max_sweeps=30, **kw)
            ms_sweep = probe[0]["t_loop_ms"] / 30.0
            sweeps = int(min(20000, max(30, budget_s * 1000.0 / max(ms_sweep, 1e-3))))
            sweeps -= sweeps % int(kw.get("refresh_every", 10))
            _, infos = api.batch(sub, max_sweeps=max(sweeps, 30), **kw)
        except _lib.RacError:
            continue
        kkts = [max(i["kkt"], 1e-300) for i in infos]
        score = math.exp(sum(math.log(k) for k in kkts) / len(kkts))
        table.append({"block": block, "assembly": assembly, "storage": storage,
                      "ms_per_sweep": ms_sweep, "sweeps": infos[0]["sweeps"], "score": score,
                      "worst_kkt": max(kkts)})
    if not table:
        raise RuntimeError("no batch autotuner candidate ran")
    best = min(table, key=lambda r: r["score"])
    res = {k: best[k] for k in ("block", "assembly", "storage", "score", "ms_per_sweep")}
    res.update({"table": table, "sample": pick, "budget_s": budget_s})
    if use_cache:
        cache[ck] = res
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return res
