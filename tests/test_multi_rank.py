"""Replica path of bench.py on CPU: world_size-2 gloo ranks, each timing its
own reconstructions; the job value is all ranks' units over the slowest
rank's time, with no data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        value, tmax = bench.job_throughput(1.0 + rank, 50 * 3)
        q.put((rank, ws, r, local, value, tmax))
    finally:
        dist.destroy_process_group()


def test_two_rank_throughput_is_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ws, r, local, value, tmax in res:
        assert (ws, r, local) == (world, rank, rank)
        assert tmax == 2.0                      # the slowest rank (rank 1: 2 s)
        assert value == world * 150 / 2.0       # all ranks' iterations / max time


def test_single_process_throughput():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.job_throughput(0.5, 100) == (200.0, 0.5)
