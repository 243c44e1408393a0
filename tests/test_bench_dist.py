"""The multi-rank aggregation bench.py uses (max time over ranks, whole-job throughput), on 2 gloo ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 100.0 + 25.0 * rank  # rank 1 is the slow one
        got = bench.max_over_ranks(mine, dist, "cpu")
        q.put((rank, got, bench.job_throughput(world, 4, 1e9, got)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, thr in out:
        assert got == 125.0  # both ranks see the slowest rank's time
        assert thr == pytest.approx(2 * 4 * 1e9 / 0.125 / 1e9)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.job_throughput(1, 10, 2e9, 1000.0) == pytest.approx(20.0)
