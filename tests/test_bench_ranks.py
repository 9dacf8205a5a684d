"""bench.py's multi-rank reduction on CPU: two gloo ranks (replicas) report
different timed regions; both take the slowest, and the job's throughput
counts every rank's solves over that time."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [30.0, 45.5][rank]
    slow = bench.slowest_rank_ms(ms, world, "cpu")
    val = bench.job_gflops(world, 2.0e9, 10, slow)
    q.put((rank, slow, val))
    dist.destroy_process_group()


def test_two_replica_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, val in res:
        assert slow == 45.5
        assert val == pytest.approx(2 * 2.0e9 * 10 / 45.5e-3 / 1e9)


def test_single_rank_is_its_own_time():
    import bench
    assert bench.slowest_rank_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_gflops(1, 1e9, 4, 2.0) == pytest.approx(2000.0)
