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
