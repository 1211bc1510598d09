"""The benchmark's multi-rank reduction (replicas only: the max of the timed
region over ranks) on two gloo ranks on the CPU."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local = 0.5 + rank  # rank 1 is the slow one
        q.put((rank, bench.max_over_ranks_dist(local, world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 1.5, 1: 1.5}
    assert all(p.exitcode == 0 for p in procs)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks_dist(3.25, 1, "cpu") == 3.25
