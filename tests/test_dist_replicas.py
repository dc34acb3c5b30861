"""The replica path of bench.py on CPU: two gloo ranks, the whole-job time is the slowest rank's
and the rate counts every rank's units (weak scaling, no collective on the data path).  A replica
that dies before the timing reduction is detected on the host: the surviving rank's reduction
fails with an error within the process group's short timeout instead of waiting forever."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    elapsed = [120.0, 150.0][rank]              # rank 1 is the slow replica
    m = bench.max_over_ranks(elapsed, ws)
    out[rank] = (m, bench.whole_job_rate(23 * 5, ws, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_max_time_and_rate():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(2):
            m, rate = out[r]
            assert m == 150.0
            assert rate == pytest.approx(2 * 23 * 5 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 1, 1000.0) == pytest.approx(10.0)



def _rank_dies(rank, ws, port, out):
    import datetime

    import torch.distributed as dist

    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws)})
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(0)                             # the failed replica leaves without reducing
    import time
    t0 = time.time()
    try:
        bench.max_over_ranks(120.0, ws)
        out[rank] = ("no error", time.time() - t0)
    except Exception as e:                      # gloo reports the lost peer or the timeout
        out[rank] = (type(e).__name__, time.time() - t0)
    os._exit(0)


def test_dead_replica_is_detected_not_waited_on():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        kind, secs = out[0]
        assert kind != "no error" and secs < 60.0
