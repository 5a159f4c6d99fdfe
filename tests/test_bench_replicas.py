"""Host logic of the N > 1 bench path on CPU: two gloo ranks, each an
independent replica, agree on the slowest rank's time and on the whole-job
rate (units of all ranks over that time)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [1.5, 2.5][rank]           # rank 1 is the slow one
        bench.barrier(world)
        t = bench.max_over_ranks(world, seconds, device="cpu")
        bench.barrier(world)
        q.put((rank, t, bench.replica_rate(world, 100, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
            pytest.fail("gloo rank did not finish")
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, t, rate in res:
        assert t == 2.5
        assert rate == pytest.approx(2 * 100 / 2.5)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1, 3.0) == 3.0
    assert bench.replica_rate(1, 10, 2.0) == 5.0
