"""The sharded batched form through the product path: two ranks (spawned
processes, gloo on the host) each solve their LPT shard of independent LASSO
problems with rac_admm_batch on the GPU, and the gathered results equal the
oracle's coordinate-descent solutions.  The ranks share one GPU here; their
kernels never wait on each other (the only exchange is the host gather)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import synth  # noqa: E402
from oracle import rac_oracle as O  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problems():
    insts = [synth.small_instance(40 + i, 60 + 11 * i, 24 + 6 * i, 4, lam2=0.05) for i in range(7)]
    probs = [dict(A=s.A, b=s.b, phi="l1l2", lambda1=s.lam1, lambda2=0.05) for s in insts]
    work = [s.m * s.n for s in insts]
    return insts, probs, work


def _gpu_batch(probs):
    from paper_1907_01995_gb300 import api
    zs, infos = api.batch(probs, num_blocks=-8, beta=1.0, tol=1e-10, max_sweeps=20000,
                          refresh_every=10, storage="fp64")
    return zs, [{"status": i["status"], "sweeps": i["sweeps"]} for i in infos]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1907_01995_gb300.shard import lpt_shards, run_sharded
    _, probs, work = _problems()
    xs, infos = run_sharded(probs, work, _gpu_batch, rank, world)
    if rank == 0:
        q.put(([x.tolist() for x in xs], infos, lpt_shards(work, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_batch_on_the_product_path():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, infos, shards = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(len(s) > 0 for s in shards)          # both ranks had work
    insts, _, _ = _problems()
    assert len(got) == len(insts)
    for x, inf, s in zip(got, infos, insts):
        assert inf["status"] == 0, inf
        ref = O.cd_enet(s.A, s.b, s.lam1, 0.05)
        x = np.asarray(x)
        assert np.abs(x - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max())
        assert np.array_equal(x != 0, ref != 0)
