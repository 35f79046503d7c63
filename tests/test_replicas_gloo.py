"""The benchmark's multi-GPU mode is replicas only (the coupling step does
not shard): every rank steps its own instance and the job's throughput is
all ranks' particle-steps over the slowest rank's time.  This checks that
aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        slow = bench.max_over_ranks(1.0 + 2.0 * rank, world)       # rank 1 is the slow replica
        value = bench.job_throughput(world, 1000, 10, slow)
        dist.barrier()
        q.put((rank, slow, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slow, value in got:
        assert slow == 3.0                      # both ranks see the slowest time
        assert value == pytest.approx(2 * 1000 * 10 / 3.0)


def test_one_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_throughput(1, 4_000_000, 100, 0.05) == pytest.approx(8e9)
