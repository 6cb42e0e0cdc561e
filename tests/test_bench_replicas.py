"""The multi-rank host logic of bench.py (replicas, one LP per rank) on two
CPU ranks over gloo: distinct seeds per rank, and the job time is the slowest
rank's (max over ranks)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local = [3.5, 7.25][rank]
        slowest = bench.max_over_ranks(local, dist, "cpu")
        out.put((rank, bench.replica_seed(rank), slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_seed_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [0, 1]          # one LP per rank
    assert all(g[2] == 7.25 for g in got)          # every rank sees the slowest time


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(1.5, None, "cpu") == 1.5
