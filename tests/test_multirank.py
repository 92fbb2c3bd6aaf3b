"""Multi-rank path of the batched form on CPU (gloo, world size 2).

Each rank solves its LPT shard of independent problems and the results are
gathered on the host.  The per-rank solver here is the FP64 oracle (this test
exercises the sharding and gathering logic, which needs no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import rac_oracle as O
from paper_1907_01995_gb300.shard import lpt_shards, run_sharded


def test_lpt_shards_cover_and_balance():
    work = [5, 1, 9, 3, 3, 7, 2, 8]
    for world in (1, 2, 3, 8):
        sh = lpt_shards(work, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(work)))
        loads = [sum(work[i] for i in s) for s in sh]
        assert max(loads) - min(loads) <= max(work)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problems():
    insts = [synth.small_instance(i, 30 + 7 * i, 12 + 3 * i, 3) for i in range(5)]
    probs = [dict(A=s.A, b=s.b, lam1=s.lam1) for s in insts]
    work = [s.m * s.n for s in insts]
    return probs, work


def _oracle_batch(probs):
    xs, infos = [], []
    for p in probs:
        P = O.problem_from_data(p["A"], p["b"], "l1l2", p["lam1"])
        st, info = O.solve(P, 3, seed=0, tol=1e-10, max_sweeps=5000)
        xs.append(st.z)
        infos.append({"sweeps": info["sweeps"], "kkt": info["kkt"]})
    return xs, infos


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs, work = _problems()
    xs, infos = run_sharded(probs, work, _oracle_batch, rank, world)
    if rank == 0:
        q.put([x.tolist() for x in xs])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_matches_single_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    probs, _ = _problems()
    ref, _ = _oracle_batch(probs)
    assert len(got) == len(ref)
    for a, b in zip(got, ref):
        assert np.array_equal(np.asarray(a), b)
