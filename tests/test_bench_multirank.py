"""Host logic of bench.py for N > 1 ranks (replicas), on CPU with the gloo backend.

Every rank reconstructs its own instances (disjoint seeds), the step time is the maximum over
ranks, and the whole-job value counts all ranks' instances.  The reference arm runs on rank 0
only; the other ranks exit without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, 16)
        local_ms = 2.0 + 3.0 * rank  # rank 1 is slower
        ms = bench.max_over_ranks(local_ms, world)
        q.put((rank, seeds, ms, bench.whole_job_value(world, 16, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, ms0, v0), (r1, s1, ms1, v1) = res
    assert (r0, r1) == (0, 1)
    assert not set(s0) & set(s1) and len(s0) == len(s1) == 16  # disjoint instances per rank
    assert ms0 == ms1 == 5.0                                     # slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 16 / 5e-3)              # all instances / slowest time


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.rank_seeds(0, 4) == [0, 1, 2, 3]
    assert bench.whole_job_value(1, 16, 2.0) == pytest.approx(8000.0)


def test_reference_arm_rank_nonzero_exits_quietly():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_gpus_flag_starts_or_refuses_ranks():
    """bench.py --gpus N never silently runs fewer ranks: without WORLD_SIZE it starts N ranks
    itself, with a WORLD_SIZE that differs from N it refuses (exit status 2, no measurement)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_plan(1, {}) == ("run", 1)
    assert bench.rank_plan(4, {}) == ("spawn", 4)
    assert bench.rank_plan(2, {"WORLD_SIZE": "2"}) == ("run", 2)
    how, msg = bench.rank_plan(8, {"WORLD_SIZE": "1"})
    assert how == "refuse" and "--gpus 8" in msg
    env = dict(os.environ, WORLD_SIZE="3", RANK="0", LOCAL_RANK="0", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "1"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2
    assert "WORLD_SIZE=3" in json.loads(r.stdout.strip().splitlines()[-1])["error"]
