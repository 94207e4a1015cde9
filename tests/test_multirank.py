"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): every rank
runs its own replica, the job's time is the slowest rank's (an all-reduce of
the elapsed times with MAX) and the whole-job throughput counts every rank's
node updates.  Under torchrun the reference arm runs on rank 0 alone; the
other ranks exit 0 without work."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, seconds, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(seconds[rank], dist, "cpu")
    value = bench.whole_job_mlups(1_000_000 * 50, world, t)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, value))


def test_slowest_rank_sets_the_job_time():
    world, seconds = 2, [0.25, 0.4]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, seconds, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in res:
        assert t == 0.4
        assert value == pytest.approx(2 * 1_000_000 * 50 / 0.4 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3, None, "cpu") == 0.3
    assert bench.whole_job_mlups(2_000_000, 1, 0.5) == pytest.approx(4.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "3", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
