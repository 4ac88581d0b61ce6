"""bench.py's multi-GPU path runs independent replicas (the scheme has no data-path exchange):
the job's throughput is all ranks' updates over the slowest rank's time.  Checked here with
two gloo ranks on the CPU (no GPU, no NCCL)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    local_ms = [80.0, 125.0][rank]  # rank 1 is the slow one
    value, ms = bench.replica_throughput(local_ms, pts_per_rank=1000, steps=10)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_time_and_summed_work():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        value, ms = res[r]
        assert ms == pytest.approx(125.0)
        assert value == pytest.approx(2 * 1000 * 10 / 0.125)


def test_single_process_is_local_time():
    sys.path.insert(0, ROOT)
    import bench

    value, ms = bench.replica_throughput(50.0, pts_per_rank=200, steps=5)
    assert ms == 50.0 and value == pytest.approx(200 * 5 / 0.05)
