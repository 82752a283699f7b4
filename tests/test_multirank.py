"""The multi-rank host logic of the benchmark on CPU ranks (gloo, world size 2):
every rank runs an independent replica (no data-path collective); the job's
time is the slowest rank's and its throughput counts every rank's points."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    mx = bench.max_over_ranks(my_ms, dist, "cpu")
    val = bench.whole_job_mpoints(world, 1_000_000, 100, mx)
    q.put((rank, mx, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, mx, val in res:
        assert mx == 15.0                           # the slowest rank's time, on every rank
        assert val == pytest.approx(2 * 1_000_000 * 100 / 0.015 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_mpoints(1, 5242880, 10, 1.0) == pytest.approx(52428.8)
