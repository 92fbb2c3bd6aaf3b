#!/usr/bin/env python
"""Benchmark: time to KKT <= 1e-6 and block updates/s of RAC-MBADMM.

Workload (one "step"): the LASSO problem A 10000 x 2000 (N(0,1) columns
scaled to unit norm, x_true 5% nonzero +-U[1,3], noise 0.01, lambda1 =
0.1 ||A^T b||_inf), p = 20 blocks, beta = gamma = 1, solved from a cold start
to KKT <= 1e-6 -- setup from the resident FP64 A (storage conversion and the
Gram matrix) plus every sweep, refresh and check.  The chosen form (picked by
the autotuner among the mixed-precision forms) is timed, and the plain FP64
GPU path is timed beside it on the same problem.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time to KKT<=1e-6 & block updates/s, chosen form vs plain FP64 GPU path"
PRECISION = {
    "bf16": "BF16 storage of G = A^T A, FP32 accumulation; FP64 iterates, duals, anchor "
            "refresh and KKT",
    "fp32": "FP32 storage of G = A^T A, FP32 accumulation; FP64 iterates, duals, anchor "
            "refresh and KKT",
    "fp64": "FP64 throughout"}
WORKLOAD = dict(name="lasso_10000x2000_p20", m=10000, n=2000, p=20, lam_frac=0.1, tol=1e-6,
                seed=0, refresh_every=10)
CPU_SAMPLE_SECONDS = 12.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--solve-once", type=int, default=0, metavar="K",
                    help="run K plain solves of the workload in the default mixed-precision "
                         "form and exit (no timing; a fixed command to profile)")
    ap.add_argument("--en-once", type=int, default=0, metavar="K",
                    help="run K BF16 solves of the Elastic-Net 2000x50000 (--assembly rac or "
                         "rp) and exit (no timing; a fixed command to profile)")
    ap.add_argument("--ws-config5", type=int, nargs=2, default=None, metavar=("TRAIN", "TEST"),
                    help="learned warm start at the family's stated size: train on TRAIN "
                         "generated instances (4096 as specified), measure sweeps and time to "
                         "KKT <= 1e-6 cold and warm on TEST held-out ones (512), print one JSON "
                         "line and exit")
    ap.add_argument("--sparse-once", type=int, default=0, metavar="SWEEPS",
                    help="one BF16 solve of the sparse Elastic-Net 20000x100000 workload for "
                         "SWEEPS sweeps and exit (no timing; a fixed command to profile)")
    ap.add_argument("--path-once", type=int, default=0, metavar="K",
                    help="run K batched BF16 solves of the 64-point regularisation path "
                         "20000x5000 and exit (no timing; a fixed command to profile)")
    ap.add_argument("--rbf-once", type=int, default=0, metavar="SWEEPS",
                    help="profiling entry: the Gaussian-kernel SVM workload with the box kept "
                         "in the blocks (BF16), SWEEPS sweeps once, then exit")
    ap.add_argument("--rbf-n", type=int, default=0, metavar="N",
                    help="with --rbf-once: N samples instead of the workload's (a smaller "
                         "case for profiling)")
    ap.add_argument("--svm-batch", type=int, default=0, metavar="COUNT",
                    help="time the batched soft-margin SVM dual workload (COUNT uneven "
                         "instances, N in [500, 20000], d in [20, 1000], blocks of 64) per "
                         "sweep and exit; max(--steps, 40) sweeps are timed")
    ap.add_argument("--storage", default="bf16", choices=["fp64", "fp32", "bf16"],
                    help="storage precision of --svm-batch")
    ap.add_argument("--assembly", default="rac", choices=["rac", "rp"],
                    help="block assembly of --svm-batch (rac: random every sweep; rp: fixed "
                         "partition in a random order)")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="skip the Elastic-Net 2000x50000 and batched-SVM legs of the line")
    return ap.parse_args()


def svm_batch_leg(args) -> int:
    """Time per sweep of the batched SVM duals in one form (--storage,
    --assembly) and print it as one JSON line (a measurement mode beside the
    headline line)."""
    import torch
    K = max(args.steps, 40)
    r = svm_batch_times(args.svm_batch, torch.device("cuda", 0),
                        [(args.storage, args.assembly)], sweeps=K)
    key = "%s/%s" % (args.storage, args.assembly)
    line = dict(r[key])
    line.update({"workload": "svm_batch_%d" % args.svm_batch, "storage": args.storage,
                 "assembly": args.assembly, "sum_Nd": r["sum_Nd"], "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- extra workload legs
EN_WORKLOAD = dict(name="elastic_net_2000x50000_p100", m=2000, n=50000, p=100, tol=1e-6,
                   refresh_every=10)


def _timed_call(fn, flush, st):
    """Run fn() between CUDA events on stream st after an L2 flush; returns
    (ms, fn's result)."""
    import torch
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    out = fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def en_leg(dev, flush, st, fp64_max_sweeps=400):
    """Elastic-Net 2000 x 50000 (groups of 10 columns with rho = 0.7,
    lambda1 = 0.05 lambda_max, lambda2 = 0.1), p = 100 blocks of 500, residual
    form, time to KKT <= 1e-6 from the resident FP64 A: the BF16- and
    FP32-storage forms, the plain FP64 path and RP-MBADMM in BF16 (fixed
    blocks in a random order, inverses once), each a full solve (setup
    included).  The FP64 path is capped at fp64_max_sweeps sweeps; if it
    stops there its time per sweep and the sweeps the BF16 form needed give
    the reported estimate, marked as such."""
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    w = EN_WORKLOAD
    inst = synth.elastic_net_instance(0)
    A = torch.tensor(inst.A, device=dev).t().contiguous().t()
    b = torch.tensor(inst.b, device=dev)
    del inst.A
    common = dict(phi="l1l2", lambda1=inst.lam1, lambda2=inst.lam2, num_blocks=w["p"], beta=1.0,
                  gamma=1.0, tol=w["tol"], refresh_every=w["refresh_every"], seed=0,
                  form="residual")
    out = {"workload": w["name"], "m": w["m"], "n": w["n"], "p": w["p"], "tol": w["tol"],
           "lambda1": "0.05*lambda_max", "lambda2": 0.1}

    def solve(storage, cap, assembly):
        with api.Handle(A, b, storage=storage, max_sweeps=cap, assembly=assembly,
                        **common) as h:
            return h.solve()[1]

    for key, storage, reps, cap, assembly in (
            ("bf16", "bf16", 2, 3000, "rac"), ("fp32", "fp32", 1, 3000, "rac"),
            ("fp64", "fp64", 1, fp64_max_sweeps, "rac"),
            ("bf16_rp", "bf16", 1, 3000, "rp")):
        runs = [_timed_call(lambda: solve(storage, cap, assembly), flush, st)
                for _ in range(reps)]
        ms, info = min(runs, key=lambda r: r[0])
        out[key] = {"time_ms": ms, "sweeps": info["sweeps"], "kkt": info["kkt"],
                    "status": info["status"], "form": info["form"],
                    "block_updates_per_s": info["block_updates"] / (ms / 1000.0)}
    f64, bf = out["fp64"], out["bf16"]
    if f64["status"] == 0:
        f64["time_to_kkt_ms"] = f64["time_ms"]
    else:
        f64["time_to_kkt_ms_estimate"] = f64["time_ms"] / f64["sweeps"] * bf["sweeps"]
        f64["note"] = ("stopped at the sweep cap; estimate = its time per sweep x the sweeps "
                       "the BF16 form needed")
    ref = f64.get("time_to_kkt_ms", f64.get("time_to_kkt_ms_estimate"))
    out["speedup_bf16_vs_fp64_plain"] = ref / bf["time_ms"]
    out["speedup_fp32_vs_fp64_plain"] = ref / out["fp32"]["time_ms"]
    out["speedup_bf16_rp_vs_fp64_plain"] = ref / out["bf16_rp"]["time_ms"]
    del A, b
    torch.cuda.empty_cache()
    return out


PATH_WORKLOAD = dict(name="lasso_path_20000x5000_64", m=20000, n=5000, nlambda=64, tol=1e-6,
                     refresh_every=10)


def path_leg(dev, flush, st, peaks, sms):
    """Regularisation path: one AR(1) design 20000 x 5000 (rho = 0.5, 5% sparse
    x_true), 64 values of lambda1 geometric from lambda_max to 0.01 lambda_max,
    p = 50 blocks of 100, time to KKT <= 1e-6 for every point from the
    resident FP64 A (handle setup included).  Forms: the batched path (all
    points in one launch per sweep) in BF16 / FP32 / FP64 storage, the
    sequential warm-started loop in BF16, and the plain FP64 path (sequential,
    FP64 storage).  The roofline of the batched chain comes from a profiled
    replica (CUDA events around each launch): its useful work is the
    gradient update 2 n^2 FLOP per running point and sweep (FP32 pipe), and
    its algorithmic traffic one pass over the n x n BF16 Gram matrix per
    launch."""
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    w = PATH_WORKLOAD
    inst, lams = synth.path_instance(0, m=w["m"], n=w["n"], nlambda=w["nlambda"])
    A = torch.tensor(inst.A, device=dev).t().contiguous().t()
    b = torch.tensor(inst.b, device=dev)
    p = inst.num_blocks
    del inst.A

    def run(storage, mode, profile=False):
        with api.Handle(A, b, phi="l1l2", lambda1=float(lams[0]), lambda2=0.0, num_blocks=p,
                        tol=w["tol"], max_sweeps=3000, refresh_every=w["refresh_every"],
                        storage=storage, form="gram", path=mode, profile=profile) as h:
            return h.path(lams)[1]

    out = {"workload": w["name"], "m": w["m"], "n": w["n"], "p": p, "nlambda": w["nlambda"],
           "tol": w["tol"], "lambda1": "geometric lambda_max .. 0.01 lambda_max"}
    run("bf16", "batched")                              # warm-up (module load)
    for storage, mode, reps in (("bf16", "batched", 2), ("fp32", "batched", 1),
                                ("fp64", "batched", 1), ("bf16", "sequential", 1),
                                ("fp64", "sequential", 1)):
        runs = [_timed_call(lambda: run(storage, mode), flush, st) for _ in range(reps)]
        ms, infos = min(runs, key=lambda r: r[0])
        sw = sum(i["sweeps"] for i in infos)
        out["%s/%s" % (storage, mode)] = {
            "time_ms": ms, "sweeps_all_points": sw, "max_sweeps": max(i["sweeps"] for i in infos),
            "kkt_max": max(i["kkt"] for i in infos),
            "status": sorted({i["status"] for i in infos}), "form": infos[0]["form"],
            "block_updates_per_s": sw * p / (ms / 1000.0)}
    ref = out["fp64/sequential"]["time_ms"]
    for k in ("bf16/batched", "fp32/batched", "fp64/batched", "bf16/sequential"):
        out[k]["speedup_vs_fp64_plain"] = ref / out[k]["time_ms"]
    out["batched_vs_sequential_bf16"] = (out["bf16/sequential"]["time_ms"] /
                                         out["bf16/batched"]["time_ms"])
    # roofline of the batched BF16 chain from a profiled replica
    infos = run("bf16", "batched", profile=True)
    n = w["n"]
    launches = infos[0]["chain_launches"]
    chain_ms = infos[0]["t_chain_ms"]
    point_sweeps = sum(i["sweeps"] for i in infos)
    flops = 2.0 * n * n * point_sweeps
    peak_alu = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ach = flops / (chain_ms / 1000.0) / 1e12
    gb = n * n * 2 * launches / (chain_ms / 1000.0) / 1e9
    out["roofline_chain"] = {
        "bound": "alu", "kernel": "k_path_chain", "achieved": ach, "peak": peak_alu,
        "unit": "TFLOP/s", "frac": ach / peak_alu, "flops_model": "2 n^2 per running point and sweep",
        "launch_ms": chain_ms / max(1, launches), "launches": launches,
        "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (
            sms, peaks.get("sm_max_mhz", 2070.0)),
        "hbm_view": {"algorithmic_bytes_per_launch": n * n * 2, "achieved_gbs": gb,
                     "peak_gbs": peaks.get("hbm_gbs", 6800.0),
                     "frac": gb / peaks.get("hbm_gbs", 6800.0)},
        "refresh_ms": infos[0]["t_refresh_ms"]}
    del A, b
    torch.cuda.empty_cache()
    return out


SPARSE_WORKLOAD = dict(name="sparse_en_20000x100000_d0.005", m=20000, n=100000, density=0.005,
                       block=100, tol=1e-6, refresh_every=10)


def sparse_leg(flush, st):
    """Sparse Elastic-Net (Sec. 3.1, Table 3's regime, scaled): A 20000 x 100000
    with 0.5% N(0,1) entries per column at random rows, unit-norm columns,
    x_true 1% nonzero, lambda1 = 0.1 ||A^T b||_inf, lambda2 = 0.1, blocks of
    100, residual form on compressed columns; time to KKT <= 1e-6 from the
    host CSC (setup included; the memory pool already grown by an untimed
    one-sweep handle) in BF16 and FP32 storage and on the plain FP64 path."""
    import synth
    from paper_1907_01995_gb300 import api
    w = SPARSE_WORKLOAD
    inst = synth.sparse_en_instance(0, m=w["m"], n=w["n"], density=w["density"],
                                    nnz_frac=0.01, lam_frac=0.1, lam2=0.1, block=w["block"])
    out = {"workload": w["name"], "m": w["m"], "n": w["n"], "nnz": int(inst.A.nnz),
           "p": inst.num_blocks, "tol": w["tol"], "lambda1": "0.1*||A^T b||_inf", "lambda2": 0.1}

    def solve(storage, sweeps=2000):
        with api.Handle(inst.A, inst.b, phi="l1l2", lambda1=inst.lam1, lambda2=0.1,
                        num_blocks=inst.num_blocks, tol=w["tol"], max_sweeps=sweeps,
                        refresh_every=w["refresh_every"], storage=storage) as h:
            return h.solve()[1]

    for storage in ("bf16", "fp32", "fp64"):
        # an untimed one-sweep handle first: the device memory pool grows to this
        # form's staging regions once per process, which a steady-state solve
        # does not pay
        solve(storage, 1)
        ms, info = _timed_call(lambda: solve(storage), flush, st)
        out[storage] = {"time_ms": ms, "sweeps": info["sweeps"], "kkt": info["kkt"],
                        "status": info["status"], "form": info["form"],
                        "block_updates_per_s": info["block_updates"] / (ms / 1000.0)}
    out["speedup_bf16_vs_fp64_plain"] = out["fp64"]["time_ms"] / out["bf16"]["time_ms"]
    return out


RBF_WORKLOAD = dict(name="rbf_svm_20000x8_s100", N=20000, d=8, sigma=1.0, C=1.0, block=100,
                    tol=1e-6, refresh_every=10, split_sweeps=600)


def rbf_svm_leg(flush, st, peaks):
    """Gaussian-kernel C-SVC dual (Sec. 3.2, eq. svm; Table 8's kernel and
    block size s = 100, beta = 0.1 p): 20000 samples of 8 features with a
    spherical class boundary, sigma = 1, C = 1.  Q = diag(y) K diag(y) is
    formed on the GPU (rac_rbf_gram) and solved to KKT <= 1e-6 with the box
    kept in the block argmins (box_qp) in BF16 and FP32 storage; the split
    form (box in the z-block) is run for a bounded number of sweeps on the
    same Q for comparison.  Times are from the device-resident Q (its build
    is reported separately)."""
    import numpy as np
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    w = RBF_WORKLOAD
    X, y = synth.rbf_svm_data(0, w["N"], w["d"])
    N = w["N"]
    p = (N + w["block"] - 1) // w["block"]
    ms_q, Q = _timed_call(lambda: api.rbf_svm_matrix(X, y, w["sigma"]), flush, st)
    out = {"workload": w["name"], "N": N, "d": w["d"], "sigma": w["sigma"], "C": w["C"], "p": p,
           "beta": 0.1 * p, "tol": w["tol"], "rbf_gram_ms": ms_q}

    def solve(storage, box, sweeps):
        kw = dict(box_qp=True) if box else dict(gamma=-0.3)
        with api.Handle(H=Q, c=-np.ones(N), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=w["C"],
                        num_blocks=p, beta=0.1 * p, tol=w["tol"], max_sweeps=sweeps,
                        refresh_every=w["refresh_every"], storage=storage, **kw) as h:
            return h.solve()[1]

    for storage in ("bf16", "fp32"):
        ms, info = _timed_call(lambda: solve(storage, True, 2000), flush, st)
        out["boxqp_" + storage] = {"time_ms": ms, "sweeps": info["sweeps"], "kkt": info["kkt"],
                                   "status": info["status"], "obj": info["obj"],
                                   "box_iters_per_block_step": info["box_iters"] /
                                   max(1, info["block_updates"]),
                                   "box_capped": info["box_capped"],
                                   "ms_per_sweep": ms / max(1, info["sweeps"])}
    # the chain's roofline: one launch per sweep reads G once (n^2 storage values)
    # and each block's M (s x ld FP32); time per launch from CUDA events
    with api.Handle(H=Q, c=-np.ones(N), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=w["C"],
                    num_blocks=p, beta=0.1 * p, tol=0.0, max_sweeps=20,
                    refresh_every=w["refresh_every"], storage="bf16", box_qp=True,
                    profile=True) as h:
        info = h.solve()[1]
    ms_chain = info["t_chain_ms"] / max(1, info["chain_launches"])
    ld = ((w["block"] + 3) // 4 + (1 - ((w["block"] + 3) // 4) % 2)) * 4
    alg = N * N * 2 + N * ld * 4
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = None
    try:
        tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        t = tj.get("box_chain/bf16/gram")
        src = open(os.path.join(ROOT, t["source"]), "rb").read()
        if t.get("source_sha256") == hashlib.sha256(src).hexdigest():
            traffic = t["bytes_per_launch"] * (N / t["n_captured"]) ** 2
    except Exception:
        traffic = None
    ach = alg / (ms_chain * 1e-3) / 1e9
    out["roofline_chain"] = {"bound": "hbm", "kernel": "k_chain_box", "ms_per_launch": ms_chain,
                             "achieved": ach, "peak": peak, "unit": "GB/s",
                             "frac": ach / peak if peak else None, "traffic": traffic,
                             "algorithmic_bytes": alg,
                             "note": "latency-bound sequential chain; peak of measured"}
    ms, info = _timed_call(lambda: solve("bf16", False, w["split_sweeps"]), flush, st)
    out["split_bf16"] = {"time_ms": ms, "sweeps": info["sweeps"], "kkt": info["kkt"],
                         "status": info["status"], "obj": info["obj"],
                         "ms_per_sweep": ms / max(1, info["sweeps"])}
    del Q
    torch.cuda.empty_cache()
    return out


def rbf_once(sweeps, n_override=0):
    """One BF16 box-mode solve of the Gaussian-kernel SVM workload for a fixed
    number of sweeps (profiling entry)."""
    import numpy as np
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    w = RBF_WORKLOAD
    N = n_override if n_override > 0 else w["N"]
    X, y = synth.rbf_svm_data(0, N, w["d"])
    p = (N + w["block"] - 1) // w["block"]
    Q = api.rbf_svm_matrix(X, y, w["sigma"])
    with api.Handle(H=Q, c=-np.ones(N), E=y, d=np.zeros(1), phi="box", lo=0.0, hi=w["C"],
                    num_blocks=p, beta=0.1 * p, tol=0.0, max_sweeps=sweeps,
                    refresh_every=w["refresh_every"], storage="bf16", box_qp=True) as h:
        _, info = h.solve()
    torch.cuda.synchronize()
    print(json.dumps({"rbf_once": sweeps, "N": N, "form": info["form"], "kkt": info["kkt"],
                      "box_iters": info["box_iters"]}), flush=True)
    return 0


def en_once(k, assembly):
    """K BF16 solves of the Elastic-Net 2000 x 50000 workload (profiling entry)."""
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    w = EN_WORKLOAD
    inst = synth.elastic_net_instance(0)
    A = torch.tensor(inst.A, device="cuda").t().contiguous().t()
    b = torch.tensor(inst.b, device="cuda")
    for _ in range(k):
        with api.Handle(A, b, phi="l1l2", lambda1=inst.lam1, lambda2=inst.lam2,
                        num_blocks=inst.num_blocks, tol=w["tol"], max_sweeps=2000,
                        refresh_every=10, storage="bf16", assembly=assembly) as h:
            _, info = h.solve()
    torch.cuda.synchronize()
    print(json.dumps({"en_once": k, "form": info["form"], "sweeps": info["sweeps"]}), flush=True)
    return 0


def _ws_instance(args):
    """One member of the warm-start family (host, numpy): a worker's job."""
    import synth
    seed, kw = args
    inst = synth.warmstart_instance(seed, **kw, block=100)
    # sent as FP32 (half the bytes through the pool's pipe); the instance is
    # this matrix, solved in FP64
    import numpy as np
    return np.asfortranarray(inst.A, dtype=np.float32), inst.b, inst.lam1, inst.lam2, inst.num_blocks


def ws_config5(ntrain, ntest):
    """The learned warm start (form 4) on its family at the stated size: the
    plain solver's solutions of ntrain generated instances are the training
    targets; the network's warm start is then compared with the cold start on
    ntest held-out instances, both to KKT <= 1e-6 (sweeps and device time per
    solve).  The instances are generated on the host by a process pool
    (spawn, started before the first CUDA call) and streamed to the GPU."""
    import multiprocessing as mp
    import time

    import numpy as np

    import synth
    fam_train = synth.warmstart_family(0, ntrain)
    fam_test = synth.warmstart_family(100000, ntest)
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        import torch

        from paper_1907_01995_gb300 import api
        from paper_1907_01995_gb300 import warmstart as ws
        t0 = time.time()
        Fs, Ts = [], []
        for A, b, lam1, lam2, p in pool.imap(_ws_instance, fam_train, chunksize=4):
            Ad = torch.tensor(A, dtype=torch.float64, device="cuda").t().contiguous().t()
            bd = torch.tensor(b, device="cuda")
            with api.Handle(Ad, bd, phi="l1l2", lambda1=lam1, lambda2=lam2, num_blocks=p,
                            tol=1e-9, max_sweeps=20000, storage="bf16") as h:
                x, _ = h.solve()
            Fx, T, _ = ws.features(Ad, bd, lam1, lam2, torch.tensor(x, device="cuda"))
            Fs.append(Fx)
            Ts.append(T)
        t_targets = time.time() - t0
        Fx, T = torch.cat(Fs), torch.cat(Ts)
        del Fs, Ts
        params = ws.init_params(0)
        tr = ws.Trainer(params, lr=3e-3)
        t1 = time.time()
        hist = tr.fit(Fx, T, epochs=8, batch=8192)
        torch.cuda.synchronize()
        t_train = time.time() - t1
        ncoord = int(Fx.shape[0])
        del Fx, T
        cold, warm, tcold, twarm, rejected = [], [], [], [], 0
        for A, b, lam1, lam2, p in pool.imap(_ws_instance, fam_test, chunksize=4):
            Ad = torch.tensor(A, dtype=torch.float64, device="cuda").t().contiguous().t()
            bd = torch.tensor(b, device="cuda")
            kw = dict(phi="l1l2", lambda1=lam1, lambda2=lam2, num_blocks=p, tol=1e-6,
                      max_sweeps=20000, refresh_every=1, storage="bf16")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            with api.Handle(Ad, bd, **kw) as h:
                _, ic = h.solve()
            e1.record()
            torch.cuda.synchronize()
            tcold.append(e0.elapsed_time(e1))
            torch.cuda.synchronize()
            e0.record()
            x0 = ws.predict(Ad, bd, lam1, lam2, params)
            with api.Handle(Ad, bd, x0=x0, xi0_from_grad=1, ws_fallback=True, **kw) as h:
                _, iw = h.solve()
            e1.record()
            torch.cuda.synchronize()
            twarm.append(e0.elapsed_time(e1))
            if ic["status"] != 0 or iw["status"] != 0:
                raise RuntimeError("a held-out solve missed KKT 1e-6: %s %s" % (ic, iw))
            cold.append(ic["sweeps"])
            warm.append(iw["sweeps"])
            rejected += iw["warm_start_rejected"]
    print(json.dumps({
        "ws_config5": {"train_instances": ntrain, "test_instances": ntest,
                       "training_coordinates": ncoord, "epochs": len(hist),
                       "loss_first": hist[0], "loss_last": hist[-1],
                       "targets_s": t_targets, "train_s": t_train, "tol": 1e-6,
                       "sweeps_cold_mean": float(np.mean(cold)),
                       "sweeps_warm_mean": float(np.mean(warm)),
                       "ms_cold_mean": float(np.mean(tcold)), "ms_warm_mean": float(np.mean(twarm)),
                       "sweep_gain": float(np.mean(cold) / np.mean(warm)),
                       "time_gain": float(np.mean(tcold) / np.mean(twarm)),
                       "warm_starts_rejected": rejected}}), flush=True)
    return 0


def sparse_once(sweeps):
    """One BF16 solve of the sparse Elastic-Net workload for a fixed number of
    sweeps (profiling entry)."""
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    w = SPARSE_WORKLOAD
    inst = synth.sparse_en_instance(0, m=w["m"], n=w["n"], density=w["density"],
                                    nnz_frac=0.01, lam_frac=0.1, lam2=0.1, block=w["block"])
    with api.Handle(inst.A, inst.b, phi="l1l2", lambda1=inst.lam1, lambda2=0.1,
                    num_blocks=inst.num_blocks, tol=0.0, max_sweeps=sweeps,
                    refresh_every=w["refresh_every"], storage="bf16") as h:
        _, info = h.solve()
    torch.cuda.synchronize()
    print(json.dumps({"sparse_once": sweeps, "form": info["form"], "kkt": info["kkt"]}), flush=True)
    return 0


def path_once(k):
    """K batched BF16 solves of the 64-point path (profiling entry)."""
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    w = PATH_WORKLOAD
    inst, lams = synth.path_instance(0, m=w["m"], n=w["n"], nlambda=w["nlambda"])
    A = torch.tensor(inst.A, device="cuda").t().contiguous().t()
    b = torch.tensor(inst.b, device="cuda")
    for _ in range(k):
        with api.Handle(A, b, phi="l1l2", lambda1=float(lams[0]), num_blocks=inst.num_blocks,
                        tol=w["tol"], max_sweeps=3000, refresh_every=w["refresh_every"],
                        storage="bf16", form="gram", path="batched") as h:
            _, infos = h.path(lams)
    torch.cuda.synchronize()
    print(json.dumps({"path_once": k, "form": infos[0]["form"],
                      "point_sweeps": sum(i["sweeps"] for i in infos)}), flush=True)
    return 0


def svm_tuned(count, dev, seed=0):
    """The batch autotuner's choice for the SVM family (same budget per
    candidate on a stratified sample, scored by the KKT reached) and its
    time per sweep on the whole batch."""
    import synth
    from paper_1907_01995_gb300 import autotune
    insts = synth.svm_batch(seed, count=count)
    probs = [dict(A=s.A, b=s.b, c=s.c, E=s.E[0], d=s.d, phi="box", lo=0.0, hi=1.0)
             for s in insts]
    return autotune.choose_batch(probs, dict(beta=0.0, gamma=-0.3, refresh_every=20, seed=0),
                                 key="svm_batch_%d" % count, device=dev)


def svm_batch_times(count, dev, forms, sweeps=40, seed=0):
    """Per-sweep device time of the batched soft-margin SVM duals (count
    uneven instances, N in [500, 20000], d in [20, 1000], blocks of 64) for
    each (storage, assembly) in forms: rac_info.t_loop_ms (CUDA events on the
    batch stream around all periods, their refreshes and the checks between
    them) over `sweeps` sweeps.  Inputs are uploaded to the device once."""
    import torch

    import synth
    from paper_1907_01995_gb300 import api
    insts = synth.svm_batch(seed, count=count)
    probs = []
    for s in insts:
        A = torch.tensor(s.A, device=dev).t().contiguous().t()
        probs.append(dict(A=A, b=s.b, c=s.c, E=s.E[0], d=s.d, phi="box", lo=0.0, hi=1.0))
        s.A = None
    res = {}
    api.batch(probs, num_blocks=-64, beta=0.0, gamma=-0.3, tol=0.0, refresh_every=20,
              storage="bf16", max_sweeps=2)                  # warm-up (module load)
    for form in forms:
        storage, assembly = form[0], form[1]
        block = form[2] if len(form) > 2 else 64
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, infos = api.batch(probs, num_blocks=-block, beta=0.0, gamma=-0.3, tol=0.0,
                             refresh_every=20, storage=storage, assembly=assembly,
                             max_sweeps=sweeps)
        torch.cuda.synchronize()
        blocks = sum(i["block_updates"] for i in infos) // sweeps
        ms = infos[0]["t_loop_ms"] / sweeps
        res["%s/%s%s" % (storage, assembly, "" if block == 64 else "/b%d" % block)] = {
            "ms_per_sweep": ms, "block_updates_per_s": blocks / (ms * 1e-3),
            "blocks_per_sweep": blocks, "sweeps_timed": sweeps, "form": infos[0]["form"],
            "call_seconds": time.perf_counter() - t0}
    res["sum_Nd"] = int(sum(int(p["A"].shape[0]) * int(p["A"].shape[1]) for p in probs))
    del probs
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------- CPU oracle leg
_CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
import synth
from oracle import rac_oracle as O
w = %(w)r
inst = synth.lasso_instance(w["seed"], m=w["m"], n=w["n"], num_blocks=w["p"], lam_frac=w["lam_frac"])
P = O.problem_from_instance(inst)
st = O.initial_state(P)
budget = %(budget)r
sweeps = 0
t0 = time.perf_counter()
while True:
    O.sweep(P, st, w["p"], w["seed"], 1.0, 1.0)
    sweeps += 1
    el = time.perf_counter() - t0
    if el >= budget or sweeps >= %(max_sweeps)d:
        break
print(json.dumps({"sweeps": sweeps, "seconds": el}))
"""


def cpu_oracle_sample(budget=CPU_SAMPLE_SECONDS, max_sweeps=500, threads=1):
    """Time the FP64 oracle (as it stands) on a bounded sample: whole sweeps of
    the same LASSO workload, after its setup, on `threads` host cores (the
    oracle's BLAS calls use them; its Python loop runs on one)."""
    t = str(threads)
    env = dict(os.environ, OPENBLAS_NUM_THREADS=t, OMP_NUM_THREADS=t, MKL_NUM_THREADS=t,
               CUDA_VISIBLE_DEVICES="")
    code = _CPU_SNIPPET % {"root": ROOT, "w": WORKLOAD, "budget": budget,
                           "max_sweeps": max_sweeps}
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=900)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    bu = r["sweeps"] * WORKLOAD["p"]
    return {"value": bu / r["seconds"], "unit": "block_updates/s", "cores": threads,
            "kind": "oracle",
            "sample": "%d whole sweeps (%d block updates) of the LASSO 10000x2000 p=20 workload "
                      "after setup, FP64 numpy/scipy, %d thread(s) of %d host cores, %.1f s"
                      % (r["sweeps"], bu, threads, os.cpu_count() or 0, r["seconds"])}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    for _ in range(max(1, args.warmup)):
        cpu_oracle_sample(budget=2.0, max_sweeps=20)
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(budget=max(2.0, CPU_SAMPLE_SECONDS / max(1, args.steps)),
                                      max_sweeps=200))
    v = statistics.mean(s["value"] for s in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "block_updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * WORKLOAD["p"] / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "m": WORKLOAD["m"], "n": WORKLOAD["n"],
                       "p": WORKLOAD["p"], "note": "FP64 CPU oracle, bounded sample per step"},
            "cpu_baseline": {"value": v, "unit": "block_updates/s", "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "block_updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", gpu_index], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.split(",") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
def block_sizes(n, p):
    q, r = divmod(n, p)
    return [q + 1] * r + [q] * (p - r)


def algorithmic_bytes(kclass, m, n, p, sb, ta, gram):
    """Bytes one launch of a kernel class must move (one sweep / one refresh)."""
    fac = sum(s * s for s in block_sizes(n, p))          # sum_i s_i^2
    if kclass == "chain":
        if gram:   # every row of G once, the p factors, 4 state vectors in, 3 out
            return n * n * sb + fac * ta + 7 * n * 8
        return 2 * m * n * sb + fac * ta + 7 * n * 8    # the slab copy of A twice
    if kclass == "factor":
        return (fac * sb + fac * ta) if gram else (p * m * (n // p + 1) * sb + fac * ta)
    if kclass == "refresh":
        return 2 * m * n * 8 + (n * n * sb if gram else m * n * sb)
    if kclass == "prox":
        return 8 * n * 8
    return 0


def algorithmic_flops(kclass, m, n, p, gram):
    """Floating-point operations the method needs per launch: the block
    factorisation is the Cholesky factor of each K_S, sum_i s_i^3 / 3 flops
    (the method's own work, whatever the kernel computes to get it); the
    refresh is two FP64 GEMVs, 4 m n flops."""
    ss = block_sizes(n, p)
    if kclass == "factor":
        return sum(s ** 3 / 3.0 for s in ss)
    if kclass == "refresh":
        return 4 * m * n
    return 0


def design_flops(kclass, m, n, p, gram):
    """Flops the factor kernel of this design actually performs: the sweep
    operator on the augmented s_i x (s_i + s_{i-1}) matrix [K_S | G[S_i,
    S_{i-1}]] (one multiply-add per entry and pivot), which yields K_S^{-1}
    and the lookahead P_i together."""
    ss = block_sizes(n, p)
    if kclass == "factor" and gram:
        return sum(2 * s * s * (s + (ss[i - 1] if i else 0)) for i, s in enumerate(ss))
    return algorithmic_flops(kclass, m, n, p, gram)


def roofline_for(kclass, ms_per_launch, w, sb, ta, gram, peaks, sms):
    """Roofline entry of one kernel class.  The Gram-form factor is FP32
    multiply-add work (bound "alu", peak = SMs x 128 FP32 lanes x 2 flop x the
    maximum SM clock); the chain is bound by the bytes it must read ("hbm",
    the measured copy bandwidth); the refresh by this part's FP64 pipe
    (nominal 1.25 TFLOP/s)."""
    m, n, p = w["m"], w["n"], w["p"]
    sec = ms_per_launch / 1000.0
    if kclass == "factor":
        fl = algorithmic_flops("factor", m, n, p, gram)
        dfl = design_flops("factor", m, n, p, gram)
        fp64 = sb == 8
        peak = 1.25 if fp64 else sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = fl / sec / 1e12
        return {"bound": "alu", "kernel": kclass, "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "flops_per_launch": fl,
                "flops_model": "Cholesky of every block, sum_i s_i^3/3",
                "design_flops_per_launch": dfl,
                "design_frac": dfl / sec / 1e12 / peak,
                "launch_ms": ms_per_launch,
                "peak_source": ("nominal FP64 1.25 TFLOP/s" if fp64 else
                                "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (
                                    sms, peaks.get("sm_max_mhz", 2070.0))),
                "note": "one CTA per block: a launch keeps p = %d of %d SMs busy" % (p, sms)}
    if kclass == "refresh":
        fl = algorithmic_flops("refresh", m, n, p, gram)
        ach = fl / sec / 1e12
        return {"bound": "alu", "kernel": kclass, "achieved": ach, "peak": 1.25,
                "unit": "TFLOP/s", "frac": ach / 1.25, "flops_per_launch": fl,
                "launch_ms": ms_per_launch, "peak_source": "nominal FP64 1.25 TFLOP/s"}
    ab = algorithmic_bytes(kclass, m, n, p, sb, ta, gram)
    peak = peaks.get("hbm_gbs", 6800.0)
    ach = ab / sec / 1e9
    return {"bound": "hbm", "kernel": kclass, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "algorithmic_bytes_per_launch": ab, "launch_ms": ms_per_launch,
            "peak_source": "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"}


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.svm_batch:
        return svm_batch_leg(args)
    if args.path_once:
        return path_once(args.path_once)
    if args.en_once:
        return en_once(args.en_once, args.assembly)
    if args.ws_config5:
        return ws_config5(*args.ws_config5)
    if args.sparse_once:
        return sparse_once(args.sparse_once)
    if args.rbf_once:
        return rbf_once(args.rbf_once, args.rbf_n)
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_1907_01995_gb300 import api
    from paper_1907_01995_gb300 import autotune

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    gpu_index = vis.split(",")[local] if vis and vis.split(",")[0].isdigit() else str(local)

    w = WORKLOAD
    inst = synth.lasso_instance(w["seed"], m=w["m"], n=w["n"], num_blocks=w["p"],
                                lam_frac=w["lam_frac"])
    A = torch.tensor(inst.A, device=dev)            # column-major copy below
    A = A.t().contiguous().t()
    b = torch.tensor(inst.b, device=dev)
    common = dict(phi="l1l2", lambda1=inst.lam1, num_blocks=w["p"], beta=1.0, tol=w["tol"],
                  max_sweeps=5000, refresh_every=w["refresh_every"], seed=w["seed"])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run(storage, form, profile=False, **extra):
        kw = dict(common)
        kw.update(extra)
        with api.Handle(A, b, storage=storage, form=form, profile=profile, **kw) as h:
            z, info = h.solve()
        return z, info

    if args.solve_once:
        for _ in range(args.solve_once):
            _, info = run("bf16", "gram")
        torch.cuda.synchronize()
        print(json.dumps({"solve_once": args.solve_once, "form": info["form"],
                          "sweeps": info["sweeps"], "kkt": info["kkt"]}), flush=True)
        return 0
    # autotuner: the chosen mixed-precision form (cached per workload)
    choice = autotune.choose(A, b, common, key=w["name"], device=dev)
    storage, form, grid = choice["storage"], choice["form"], choice["grid"]

    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        run(storage, form, grid=grid)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = ClockSampler(gpu_index)
    step_ms, infos = [], []
    for _ in range(args.steps):
        flush.zero_()                                  # L2 flush between steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        _, info = run(storage, form, grid=grid)       # the product path (CUDA graphs)
        e1.record(st)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(info)
    clocks = clk.stop()
    # the same steps again with every kernel class bracketed by CUDA events on
    # the library's stream (direct launches): per-kernel device times
    prof_infos, prof_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        _, info = run(storage, form, profile=True, grid=grid)
        e1.record(st)
        torch.cuda.synchronize()
        prof_ms.append(e0.elapsed_time(e1))
        prof_infos.append(info)
    total_ms = sum(step_ms)
    bu = sum(i["block_updates"] for i in infos)
    if world > 1:
        t = torch.tensor([total_ms, float(bu)], device=dev, dtype=torch.float64)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_ms_max, bu_all = float(tmax[0]), float(t[1])
    else:
        total_ms_max, bu_all = total_ms, float(bu)
    value = bu_all / (total_ms_max / 1000.0)

    # other forms on the same problem, each a full solve to the same KKT:
    # the plain FP64 GPU path (FP64 storage; its chain is the grid-barrier
    # chain, since the one-cluster chain is FP32/BF16-only), the FP32-storage
    # form of config 2, and the chosen storage on the grid-barrier chain (which
    # separates the chain design's share of the speed-up from precision's)
    def time_form(reps, storage_, form_, **extra):
        run(storage_, form_, **extra)
        ms_, info_ = [], None
        for _ in range(reps):
            t_, (_, info_) = _timed_call(lambda: run(storage_, form_, **extra), flush, st)
            ms_.append(t_)
        return ms_, info_

    fp64_ms, fp64_info = time_form(args.fp64_steps, "fp64", "gram")
    fp32_ms, fp32_info = time_form(args.fp64_steps, "fp32", "gram")
    grid_ms, grid_info = time_form(args.fp64_steps, storage, form, chain="grid")

    # end to end through the C-ABI with pinned host buffers
    A_h = torch.empty((w["n"], w["m"]), dtype=torch.float64, pin_memory=True)
    A_h.copy_(torch.from_numpy(np.ascontiguousarray(inst.A.T)))
    A_h = A_h.t()                                      # column-major host view
    b_h = torch.from_numpy(inst.b.copy()).pin_memory()
    z_h = torch.empty(w["n"], dtype=torch.float64, pin_memory=True)
    e2e_s, e2e_bu, e2e_info = [], 0, None
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with api.Handle(A_h, b_h, storage=storage, form=form, grid=grid, **common) as h:
            _, e2e_info = h.solve(z_h)
        e2e_s.append(time.perf_counter() - t0)
        e2e_bu += e2e_info["block_updates"]
    periods = math.ceil(e2e_info["sweeps"] / w["refresh_every"]) + 1

    # roofline of the dominant kernel class, from the live event timings
    sb = {"fp64": 8, "fp32": 4, "bf16": 2}[storage]
    ta = 8 if storage == "fp64" else 4
    gram = infos[-1]["form"].startswith("gram")
    cls_ms = {c: sum(i["t_%s_ms" % c] for i in prof_infos) for c in
              ("assembly", "factor", "chain", "prox", "refresh")}
    launches = {"chain": sum(i["chain_launches"] for i in prof_infos)}
    launches["factor"] = launches["prox"] = launches["chain"]
    launches["refresh"] = sum(math.ceil(i["sweeps"] / w["refresh_every"]) for i in prof_infos)
    dom = max(("factor", "chain", "prox", "refresh"), key=lambda c: cls_ms[c])
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = {c: roofline_for(c, cls_ms[c] / max(1, launches[c]), w, sb, ta, gram, peaks, sms)
            for c in ("factor", "chain", "refresh")}
    # DRAM traffic per launch from the committed ncu capture, if it was taken
    # on the kernels as they are now (source hash)
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f)
        for c, ent in roof.items():
            t = tj.get("%s/%s/%s" % (c, storage, "gram" if gram else "residual"))
            ent["traffic"] = None
            if t:
                src = open(os.path.join(ROOT, t["source"]), "rb").read()
                if t.get("source_sha256") == hashlib.sha256(src).hexdigest():
                    ent["traffic"] = t["bytes_per_launch"]
    except Exception:
        for ent in roof.values():
            ent.setdefault("traffic", None)

    extra = {}
    if rank == 0 and world == 1 and not args.no_extra_legs:
        try:
            extra["elastic_net_2000x50000"] = en_leg(dev, flush, st)
        except Exception as ex:  # report, never fake
            extra["elastic_net_2000x50000"] = {"failed": str(ex)[:300]}
        try:
            extra["lasso_path_20000x5000_64"] = path_leg(dev, flush, st, peaks, sms)
        except Exception as ex:
            extra["lasso_path_20000x5000_64"] = {"failed": str(ex)[:300]}
        try:
            extra["sparse_en_20000x100000"] = sparse_leg(flush, st)
        except Exception as ex:
            extra["sparse_en_20000x100000"] = {"failed": str(ex)[:300]}
        try:
            extra["rbf_svm_20000"] = rbf_svm_leg(flush, st, peaks)
        except Exception as ex:
            extra["rbf_svm_20000"] = {"failed": str(ex)[:300]}
        try:
            tuned = svm_tuned(256, dev)
            forms = [("bf16", "rp"), ("bf16", "rac"), ("fp32", "rp"), ("fp64", "rp"),
                     ("fp64", "rac")]
            pick = (tuned["storage"], tuned["assembly"], tuned["block"])
            if pick[2] != 64 or (pick[0], pick[1]) not in forms:
                forms.append(pick)
            extra["svm_batch_256"] = svm_batch_times(256, dev, forms, sweeps=40)
            extra["svm_batch_256"]["autotuner"] = tuned
        except Exception as ex:
            extra["svm_batch_256"] = {"failed": str(ex)[:300]}

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        try:
            cpu = cpu_oracle_sample()
            cpu_all = cpu_oracle_sample(threads=ncores)
        except Exception as ex:  # report, never fake
            cpu = {"value": None, "unit": "block_updates/s", "cores": 1, "kind": "oracle",
                   "sample": "failed: %s" % str(ex)[:200]}

    if world > 1:
        dist.barrier()
    if rank == 0:
        ttk = statistics.mean(step_ms)
        f64 = statistics.mean(fp64_ms)
        def form_entry(ms_list, info_):
            t_ = statistics.mean(ms_list)
            return {"time_to_kkt_ms": t_, "sweeps": info_["sweeps"],
                    "block_updates_per_s": info_["block_updates"] / (t_ / 1000.0),
                    "form": info_["form"], "kkt": info_["kkt"], "status": info_["status"]}

        line = {
            "metric": METRIC, "value": value, "unit": "block_updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ttk,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "fp32": "f32", "fp64": "f64"}[storage],
            "data": "synthetic",
            "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "p": w["p"],
                       "lambda1": "0.1*||A^T b||_inf", "tol": w["tol"],
                       "form": infos[-1]["form"], "grid": grid,
                       "precision": PRECISION[storage],
                       "anchor": "FP64 refresh every %d sweeps" % w["refresh_every"],
                       "l2": "512 MB buffer written between timed steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_kkt_ms": ttk, "sweeps": infos[-1]["sweeps"], "kkt": infos[-1]["kkt"],
            "fp64_plain": form_entry(fp64_ms, fp64_info),
            "fp32_form": form_entry(fp32_ms, fp32_info),
            "chosen_storage_grid_chain": form_entry(grid_ms, grid_info),
            "speedup_vs_fp64_plain": f64 / ttk,
            "speedup_fp32_form_vs_fp64_plain": f64 / statistics.mean(fp32_ms),
            "cpu_baseline_all_cores": cpu_all,
            "workloads": extra,
            "kernel_ms_per_step": {c: v / len(prof_infos) for c, v in cls_ms.items()},
            "profiled_ms_per_step": statistics.mean(prof_ms),
            "roofline": roof.get(dom, roof["chain"]),
            "roofline_chain": roof["chain"],
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_bu / sum(e2e_s), "unit": "block_updates/s",
                    "time_to_kkt_ms": 1000.0 * statistics.mean(e2e_s),
                    "h2d_bytes_per_step": (w["m"] * w["n"] + w["m"]) * 8,
                    "d2h_bytes_per_step": w["n"] * 8 + periods * 52},
            "clocks": clocks,
            "gpu_launches": sum(i["kernel_launches"] + i["setup_launches"] for i in infos),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
