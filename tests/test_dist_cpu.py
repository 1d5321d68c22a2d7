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
