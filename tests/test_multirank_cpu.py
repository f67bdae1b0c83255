"""The benchmark's multi-rank path (replicas, weak scaling) on CPU ranks with gloo: the job
time is the slowest rank's and the value counts every rank's work."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = [1.0 + rank, 10.0 - rank, 0.5 * (rank + 1), 3.0]
    got = bench.max_over_ranks(mine, "cpu")
    q.put((rank, got, bench.whole_job_gflops(world, 6.0, got[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, got, value in res:
        assert got == [2.0, 10.0, 1.0, 3.0]
        assert value == pytest.approx(2 * 6.0 / (2.0 / 1e3))
