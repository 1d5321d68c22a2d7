"""The bench's multi-GPU host logic on CPU with two gloo ranks: every rank
runs its own problem, the timing is the maximum over ranks, and the whole-job
rate aggregates all ranks (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as tmp       # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    d = bench.init_dist(ws, "gloo")
    ms = 100.0 + 50.0 * r                        # rank 1 is the slow one
    tmax = bench.max_over_ranks(d, ms)
    rate = bench.job_rate(ws, 1000, 3, tmax)
    d.barrier()
    q.put((r, ws, tmax, rate))
    d.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_sum_the_work():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ws, tmax, rate in out:
        assert ws == 2 and tmax == 150.0
        assert abs(rate - 2 * 1000 * 3 / 0.150) < 1e-6


def test_single_process_has_no_collective():
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 12.5) == 12.5


def test_reference_arm_under_torchrun_prints_once_from_rank_zero():
    # `bench.py --impl reference` launched as two ranks: rank 0 times the
    # oracle and prints one JSON line, the other rank exits 0 without work.
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-seconds", "0.5"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
