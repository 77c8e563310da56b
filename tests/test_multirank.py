"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
runs its own replica, the ranks meet at a barrier around the timed region,
the time reported is the maximum over the ranks and the throughput counts
every rank's node updates (weak scaling, no data-path collective)."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo")
    try:
        assert r.world == world and r.rank == rank
        r.barrier()
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
        ms_max = r.maxall(ms)
        value = bench.weak_scaling_value(1000, 10, ms_max, r.world)
        r.barrier()
        q.put((rank, ms_max, value))
    finally:
        r.close()


def test_two_ranks_max_time_and_whole_job_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, value in out:
        assert ms_max == 15.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.015 / 1e6)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    env_backup = {k: os.environ.pop(k, None) for k in ("WORLD_SIZE", "RANK")}
    try:
        r = bench.Ranks("gloo")
        assert r.world == 1 and r.dist is None
        r.barrier()
        assert r.maxall(3.5) == 3.5
        assert bench.weak_scaling_value(100, 4, 2.0, 1) == pytest.approx(100 * 4 / 0.002 / 1e6)
    finally:
        for k, v in env_backup.items():
            if v is not None:
                os.environ[k] = v


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
