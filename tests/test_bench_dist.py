"""Host-side logic of the multi-GPU bench path on CPU: two gloo ranks, each with
its own timed region; the job time is the max over ranks and the value counts
the elements of every rank (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_total = [100.0, 250.0][rank]                 # rank 1 is the slow one
    ms_step, value = bench.aggregate(ms_total, 1_000_000, 10, world, dist, "cpu")
    q.put((rank, ms_step, value))
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, ms_step, value in res:
        assert ms_step == pytest.approx(25.0)
        assert value == pytest.approx(2 * 1_000_000 / 25e-3 / 1e6)


def test_aggregate_single_rank():
    import bench
    ms, v = bench.aggregate(50.0, 6_000_000, 100, 1)
    assert ms == 0.5 and v == pytest.approx(12000.0)


def _weak_worker(rank, world, port, q):
    """One rank of the weak-scaling path on CPU: its own seeded mesh of the bench
    workload (a small cube here), integrated by the FP64 oracle as the rank's
    step, timed, then the job time (max over ranks) and the whole-job value from
    bench.aggregate; the mesh's checksum goes to rank 0 to show the ranks' problems
    are independent shards, not copies."""
    import time

    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    mesh, coefs = bench.workload(rank, n_cubes=4)            # 384 elements per rank
    t = time.perf_counter()
    A, b, flags = oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh, coefs)
    ms = (time.perf_counter() - t) * 1e3
    ms_step, value = bench.aggregate(ms, len(mesh), 1, world, dist, "cpu")
    sums = torch.tensor([float(mesh.sum()), float(np.abs(A).sum())], dtype=torch.float64)
    gathered = [torch.zeros_like(sums) for _ in range(world)]
    dist.all_gather(gathered, sums)
    q.put((rank, ms, ms_step, value, len(mesh), [g.tolist() for g in gathered], bool(np.isfinite(A).all()),
           int(flags.sum())))
    dist.destroy_process_group()


def test_weak_scaling_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_weak_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    slowest = max(r[1] for r in res)
    for rank, ms, ms_step, value, n, gathered, finite, nflags in res:
        assert n == 384 and finite and nflags == 0
        assert ms_step == pytest.approx(slowest)
        assert value == pytest.approx(2 * n / (slowest * 1e-3) / 1e6)
        # every rank sees both checksums, and the two shards differ
        assert gathered == res[0][5]
        assert gathered[0] != gathered[1]
