"""The multi-rank path of bench.py on the CPU: two gloo ranks (torch.distributed), no GPU.

Each rank of `bench.py --gpus N` solves its own instance of the workload (no collective on the data
path); the job's time is the slowest rank's, and the whole-job rate counts every rank's points.  The
checks: ranks get distinct, reproducible workloads; max_over_ranks returns the maximum on every rank;
job_rate is the aggregate.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w = bench.rank_workload(24, rank)
        elapsed = 10.0 + 5.0 * rank                      # the slower rank sets the job's time
        m = bench.max_over_ranks(elapsed)
        seeds = [None] * world
        dist.all_gather_object(seeds, w.seed)
        rate = bench.job_rate(w.npoints, 3, world, m)
        out.put((rank, m, seeds, rate, w.npoints))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
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
    for rank, m, seeds, rate, npts in res:
        assert m == 15.0                                 # max over ranks, seen by every rank
        assert len(set(seeds)) == world                  # independent instances
        assert rate == pytest.approx(npts * 3 * world / 15.0 / 1e6)
    assert res[0][2] == res[1][2]


def test_single_process_has_no_collective():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    w0, w1 = bench.rank_workload(16, 0), bench.rank_workload(16, 1)
    assert w0.seed != w1.seed and w0.dims == w1.dims
