"""The bench's multi-rank host logic on CPU with two gloo ranks (one process per GPU on a B300 node;
here the same code with the collective's tensor on the CPU): the job's time is the slowest rank's,
throughput counts every rank's units, and the reference arm runs on rank 0 alone."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank durations: rank r took 1 + r s on its timed region and 10 - r s on another
        mx = bench.max_over_ranks([1.0 + rank, 10.0 - rank], world, "cpu")
        rate = bench.job_rate(world, 20, mx[0])
        dist.barrier()
        # the reference arm: every rank but 0 returns at once, without building the workload
        sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"]
        ret = bench.main() if rank != 0 else None
        out.put((rank, mx, rate, ret))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_count_every_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, mx, rate, ret in res:
        assert mx == [2.0, 10.0]          # max over ranks of each entry
        assert rate == pytest.approx(world * 20 / 2.0)
    assert res[1][3] == 0                 # rank 1 left the reference arm with status 0


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.job_rate(1, 10, 2.0) == 5.0
