"""The N > 1 path of bench.py on CPU: replicas on world_size-2 gloo ranks.

Each rank runs its own independent products (no data-path collective); the
only exchange is the timing: the job's time is the slowest rank's, and the
whole-job rate counts the products of every rank.  The reference arm runs on
rank 0 only; the other ranks exit without work.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
    tmax = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(world, 10, tmax)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, tmax, rate))


def test_max_over_ranks_and_whole_job_rate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, rate in out:
        assert tmax == 150.0
        assert abs(rate - 2 * 10 / 0.150) < 1e-9


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert abs(bench.whole_job_rate(1, 4, 500.0) - 8.0) < 1e-12


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
