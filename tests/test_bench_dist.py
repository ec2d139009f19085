"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) combine their timed
regions as the max over ranks, and the job's throughput counts the points of every rank."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        local_ms = 10.0 + 5.0 * rank           # rank 1 is the slower replica
        total_ms, value = bench.job_throughput(local_ms, ws, 1_000_000, torch.device("cpu"))
        q.put((rank, total_ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_all_points():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, total_ms, value in res:
        assert total_ms == 15.0                 # the slowest replica's timed region
        assert value == pytest.approx(2 * 1_000_000 / 15e-3 / 1e9)


def test_single_rank_is_unchanged():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    total_ms, value = bench.job_throughput(8.0, 1, 4_000_000, torch.device("cpu"))
    assert total_ms == 8.0 and value == pytest.approx(4_000_000 / 8e-3 / 1e9)
