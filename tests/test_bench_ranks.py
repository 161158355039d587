"""Host logic of the multi-rank benchmark (replicas only), on CPU with gloo.

Every rank advances its own independent replica; the only collectives are
the host barrier and the maximum of the elapsed times, so a world of two
gloo ranks on CPU exercises all of it."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # rank r pretends its timed region took 1 + r seconds
        t = bench.max_over_ranks(1.0 + rank, world)
        v = bench.job_throughput(world, 1000.0, t)
        r, w, l = bench.dist_env()
        # the replica of each rank comes from its own seed
        x, _, kw = bench.system(1 + rank)
        out.put((rank, t, v, (r, w, l), kw["seed"], float(x.sum())))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # every rank sees the slowest rank's time
    assert [r[1] for r in res] == [2.0, 2.0]
    # whole-job value: both ranks' units over the slowest time
    assert res[0][2] == pytest.approx(2 * 1000.0 / 2.0)
    assert [r[3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    # independent replicas: different seeds, different placements
    assert res[0][4] != res[1][4]
    assert res[0][5] != res[1][5]


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(1, 10.0, 2.0) == 5.0
    bench.barrier(1)


def test_reference_arm_other_ranks_exit(monkeypatch):
    """Under torchrun only rank 0 runs the reference arm; the others exit 0
    without work."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps = 1
        warmup = 0
    assert bench.run_reference(A()) == 0
