"""The bench's multi-rank host logic on CPU ranks (gloo, world size 2): the
job time is the slowest rank's, throughput counts every rank's units, and
each rank recovers its own replica.  No GPU involved."""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2506_09594_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    ms = bench.max_over_ranks(dist, ms_local, "cpu")
    w = synth.WORKLOADS["tubal64_r5"]
    _, M, _, _ = synth.make_problem(w, seed=bench.replica_seed(w.seed, rank))
    digest = float(np.abs(M).sum())
    gathered = [None] * world
    dist.all_gather_object(gathered, digest)
    out.put((rank, ms, bench.job_rate(50, world, ms * 1e-3), gathered, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ms, rate, gathered, env in res:
        assert ms == 15.0                              # max over ranks
        assert rate == pytest.approx(50 * 2 / 0.015)   # units of both ranks / slowest time
        assert gathered[0] != gathered[1]              # distinct replicas
        assert env == (2, rank, rank)
