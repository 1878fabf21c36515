"""The multi-GPU path is replicas only: each rank analyses its own copy of
the workload and the job's figures are the slowest rank's time and the sum
of all ranks' rays.  This checks that reduction (bench.job_totals) with two
gloo ranks on the CPU, and that a rank that raises ends its process group
with an error on the other rank instead of hanging it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.job_totals(1.5 + rank, 1000.0 * (rank + 1), torch.device("cpu"))
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    port = _port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == out[1] == (2.5, 3000.0)


def _failing(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        raise SystemExit(3)                       # a rank that leaves before the collective
    import bench
    try:
        bench.job_totals(1.0, 1.0, torch.device("cpu"))
        out[rank] = "completed"
    except Exception as e:                        # the surviving rank learns of it
        out[rank] = "error: " + type(e).__name__


def test_lost_rank_is_reported_not_hung():
    port = _port()
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_failing, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=60)
        for p in procs:
            if p.is_alive():
                p.kill()
                pytest.fail("a rank hung")
        assert procs[1].exitcode == 3
        assert out.get(0, "").startswith("error")
