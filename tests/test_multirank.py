"""The benchmark's multi-GPU host logic on two CPU ranks (gloo): replicas of the filter, each
rank on its own packets, the job's time the slowest rank's, the rate summed over ranks.  No GPU
and no data-path collective: packets are independent (replicas only)."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist)   # rank r took 10 + 5 r ms
        q.put((rank, slowest, bench.ring_seed(rank), bench.job_rate(world, 100, slowest / 1e3)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_the_slowest_time_and_sum_the_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [15.0, 15.0]            # every rank reports the slowest rank's time
    assert got[0][2] != got[1][2]                         # each replica filters its own packets
    assert got[0][3] == got[1][3] == pytest.approx(2 * 100 / 0.015)   # whole-job frames/s


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_rate(1, 200, 0.25) == 800.0


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the CPU reference arm prints from rank 0 alone; rank 1 exits at once."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
