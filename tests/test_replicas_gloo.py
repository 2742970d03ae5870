"""The multi-GPU path of the benchmark is replicas only (the exact sweep does not shard): each
rank solves its own cavity and the job's time is the slowest rank's.  Its host logic, run as
two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        slow = bench.max_over_ranks(1.5 + rank, device="cpu")   # rank 1 is the slow replica
        value = bench.replica_throughput(1000, w, slow)
        q.put((r, lr, w, slow, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 0, 2), (1, 1, 2)]
    for o in out:
        assert o[3] == pytest.approx(2.5)            # both ranks see the slowest time
        assert o[4] == pytest.approx(2 * 1000 / 2.5)  # all ranks' units over that time


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_throughput(10, 1, 2.0) == 5.0
