"""The multi-GPU mode is replicas only: every rank runs its own copy of the
workload and the job's numbers are the slowest rank's time and the sum of
the ranks' cell-steps.  This checks that reduction on two CPU ranks (gloo)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = [12.5, 20.0][rank]
        cells = [1000, 3000][rank]
        out[rank] = bench.aggregate_ranks(ms, cells, ws, "cpu")
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_to_slowest_time_and_total_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        assert out[0] == out[1] == (20.0, 4000.0)


def test_single_rank_is_the_identity():
    import bench
    assert bench.aggregate_ranks(3.5, 17, 1, "cpu") == (3.5, 17.0)
