"""The multi-replica path of bench.py on CPU: two gloo ranks, each with its own time, must agree
on the slowest rank's time and on the whole-job rate (the GPU run of the same code uses NCCL)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", init_method="env://")
    try:
        r, w, local = bench.dist_env()
        ms = 100.0 + 25.0 * r                       # rank 1 is the slower replica
        slowest = bench.max_over_ranks(ms, "cpu")
        rate = bench.job_throughput(1000, slowest / 1e3, w)
        q.put((r, w, local, slowest, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_take_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = 100.0 + 25.0 * (world - 1)
    for r, (rank, w, local, slowest, rate) in enumerate(out):
        assert (rank, w, local) == (r, world, r)
        assert slowest == slow
        assert rate == pytest.approx(1000 * world / (slow / 1e3))


def test_single_rank_is_its_own_max():
    import bench

    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_throughput(10, 2.0, 1) == 5.0
