"""The benchmark's multi-rank bookkeeping, run as two gloo ranks on the CPU:
times are the slowest rank's, end-to-end rates the slowest rank's times the
rank count, and the whole-job value counts every rank's symbols."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0 + rank, 20.0 - rank]
    got_max = bench.ranks_max(ms, dist, "cpu")
    got_min = bench.ranks_min([5.0 * (rank + 1)], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got_max, got_min))


def test_two_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got_max, got_min in res:
        assert got_max == [11.0, 20.0]
        assert got_min == [5.0]


def test_whole_job_value_counts_all_ranks():
    import bench
    one = bench.whole_job_gbps(1 << 20, 10, 1, 2.0)
    assert bench.whole_job_gbps(1 << 20, 10, 4, 2.0) == pytest.approx(4 * one)
    assert one == pytest.approx(2.0 * (1 << 20) * 10 / 2e-3 / 1e9)
    assert bench.ranks_max([3, 1], None, "cpu") == [3.0, 1.0]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
