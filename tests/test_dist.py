"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.

Each rank runs an independent replica (no data-path collective); the job's time is the
slowest rank's and its throughput counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    bench.init_dist(world, "gloo")
    w, r, _ = bench.dist_env()
    seconds = [2.0, 5.0][r]                     # rank 1 is the slow one
    value, t = bench.combine(100.0, seconds, w)
    bench.barrier(w)
    q.put((r, value, t))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, value, t in out:
        assert t == pytest.approx(5.0)
        assert value == pytest.approx(2 * 100.0 / 5.0)


def test_single_rank_is_identity():
    import bench
    v, t = bench.combine(10.0, 2.0, 1)
    assert (v, t) == (5.0, 2.0)
