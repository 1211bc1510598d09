"""The benchmark's multi-rank paths on two gloo ranks on the CPU: the max of
the timed region over ranks (replicas), and the ensemble's case partition
(each rank advances its share of the independent grids; the job's node
updates are summed over ranks and divided by the slowest rank's time)."""
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


def _partition_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2311_10827_gb300 import workloads as wl
        sizes = [wl.ensemble_case(s)["n"] ** 2 for s in range(256)]
        mine = bench.partition_cases(sizes, world)[rank]
        local_nodes = sum(sizes[i] for i in mine)
        local_s = 0.25 * (rank + 1)  # rank 1 is the slow one
        nodes, dt = bench.combine_ranks(local_nodes, local_s, world, "cpu")
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        q.put((rank, mine, local_nodes, nodes, dt, everyone))
    finally:
        dist.destroy_process_group()


def test_ensemble_partition_two_gloo_ranks():
    from paper_2311_10827_gb300 import workloads as wl
    sizes = [wl.ensemble_case(s)["n"] ** 2 for s in range(256)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    got = {r[0]: r[1:] for r in (q.get(timeout=5) for _ in range(2))}
    assert all(p.exitcode == 0 for p in procs)
    m0, n0, tot0, dt0, all0 = got[0]
    m1, n1, tot1, dt1, all1 = got[1]
    # every case on exactly one rank, and both ranks agree on the split
    assert sorted(m0 + m1) == list(range(256)) and not set(m0) & set(m1)
    assert all0 == all1 == [m0, m1]
    # the job's node updates per step: the sum over ranks, on both ranks
    assert n0 + n1 == sum(sizes) == tot0 == tot1
    # balanced by node count within the largest grid
    assert abs(n0 - n1) <= max(sizes)
    # the job ends with its slowest rank
    assert dt0 == dt1 == 0.5
