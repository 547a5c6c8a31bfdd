"""Host-side logic of bench.py's replica mode (N > 1): every rank times its own
replica, the job time is the slowest rank's and the throughput counts every
rank's work.  Run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]
    out[rank] = bench.aggregate(ms, 1000.0, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    for r in range(2):
        ms, thr = out[r]
        assert ms == pytest.approx(150.0)
        assert thr == pytest.approx(2 * 1000.0 / 0.150)


def test_aggregate_single_process():
    import bench
    ms, thr = bench.aggregate(200.0, 500.0, "cpu")
    assert ms == 200.0 and thr == pytest.approx(2500.0)
