"""The benchmark's multi-rank logic on the CPU (gloo, two ranks): the job's
step time is the slowest rank's, its throughput counts every rank's rays,
and the reference arm runs on rank 0 alone.  The path itself shards into
replicas with no collective, so these are all the ranks share."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = 1.5 + rank            # rank 1 is the slower one
    got = bench.max_over_ranks(ms, dist)
    out.put((rank, got, bench.job_throughput(world, 3_000_000, got)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]               # both ranks see the slowest time
    assert res[0][2] == pytest.approx(2 * 3_000_000 / 2500)  # 2 ranks x 3 M rays in 2.5 ms: 2400 Mrays/s


def test_one_rank_needs_no_collective():
    assert bench.max_over_ranks(1.25, None) == 1.25
    assert bench.job_throughput(1, 5_702_033, 1.372) == pytest.approx(5_702_033 / 1372)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""
