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


def _run_reference(env_rank, env_world):
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK=str(env_rank), LOCAL_RANK=str(env_rank), WORLD_SIZE=str(env_world),
               MASTER_ADDR="127.0.0.1")
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--gpus", str(env_world)], cwd=root, env=env, capture_output=True,
                          text=True, timeout=600)


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_reference(1, 2)
    assert r.returncode == 0 and r.stdout.strip() == "", r.stderr[-2000:]


def test_reference_arm_line():
    import json

    r = _run_reference(0, 1)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "G add-min/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    for key in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
                "dtype", "data", "config"):
        assert key in line, key
