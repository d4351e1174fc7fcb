"""The multi-rank timing path of bench.py (replicas: one keyframe per rank, no data-path
collective) on two CPU processes over gloo: the barrier, the MAX reduction of the step time
and the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.rank_barrier(dist)
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
        slowest = bench.max_ms_over_ranks(dist, ms, "cpu")
        value = bench.job_throughput(world, 1, 20, slowest)
        out.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]  # both ranks see the slowest time
    # 2 ranks x 20 steps of one keyframe in 15 ms
    assert res[0][2] == pytest.approx(2 * 20 / 0.015)


def test_single_process_is_identity():
    import bench
    assert bench.max_ms_over_ranks(None, 12.5, "cpu") == 12.5
    bench.rank_barrier(None)
    assert bench.job_throughput(1, 6, 10, 100.0) == pytest.approx(600.0)
