"""The replica timing of bench.py across ranks (gloo, world size 2, CPU): the slowest rank's
time is taken and the throughput counts every rank's work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    t = bench.max_over_ranks(1.0 + rank)          # rank 1 is slower
    rate = bench.aggregate_rate(10.0, ws, t)
    out[rank] = (t, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_rate():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert out[0] == out[1] == (2.0, 10.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.aggregate_rate(7.0, 1, 2.0) == 3.5
