"""Host logic of bench.py's multi-rank form, on CPU with two gloo ranks:
disjoint per-rank workloads, the max-over-ranks time, the whole-job rate, and
the reference arm's rank-0-only rule."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = [w.seed for w in bench.workload(rank, 4)]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        rate = bench.whole_job_rate(64 * 10, world, t)
        q.put((rank, gathered, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_work_and_max_time():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(world, port, q), nprocs=world, join=True, start_method="spawn")
    out = sorted(q.get() for _ in range(world))
    for rank, gathered, t, rate in out:
        assert gathered[0] == [0, 1, 2, 3] and gathered[1] == [4, 5, 6, 7]
        assert t == 2.5  # the slowest rank's time, on every rank
        assert rate == pytest.approx(64 * 10 * 2 / 2.5)


def test_single_process_helpers():
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.whole_job_rate(640, 1, 2.0) == 320.0
    assert [w.seed for w in bench.workload(0, 3)] == [0, 1, 2]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_traffic_fingerprints_resolve():
    """Every kernel and device function a traffic figure depends on is found
    in the kernel file, so the fingerprint is well defined; a change to any
    of them changes it."""
    src = open(os.path.join(ROOT, bench.KERNEL_FILE)).read()
    for t in bench.TRAFFIC.values():
        for name in (t["kernel"],) + tuple(t["helpers"]):
            text = bench._definition(src, name)
            assert text is not None and text.rstrip().endswith("}")
            assert name + "(" in text.splitlines()[0] or name + "(" in text.splitlines()[1]
        fp = bench.kernel_fingerprint(t["kernel"], t["helpers"])
        assert fp is not None and len(fp) == 40
        assert fp != bench.kernel_fingerprint(t["kernel"], t["helpers"][:-1])
