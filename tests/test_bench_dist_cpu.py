"""The bench's multi-rank aggregation (max time over ranks, summed work) on two
CPU processes with the gloo backend."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    work = 1e9 * (rank + 1)
    ms_max, value = bench.aggregate(ms_local, work, dist, "cpu")
    out[rank] = (ms_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, value = out[r]
        assert ms_max == pytest.approx(150.0)
        assert value == pytest.approx(3e9 / 0.150)


def test_single_process_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(200.0, 4e9) == (200.0, pytest.approx(2e10))
