"""Multi-GPU form of bench.py is replicas only: each rank solves its own copy
and rank 0 reports all ranks' solves over the slowest rank's time.  The
cross-rank reduction is host logic, checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 5.0][rank]
    value, slowest = bench.reduce_timing(elapsed, steps=10, world=world, dist=dist, device="cpu")
    out[rank] = (value, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_timing_reduction():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, slowest = res[r]
        assert slowest == 5.0
        assert value == pytest.approx(2 * 10 / 5.0)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(4.0, steps=8, world=1) == (2.0, 4.0)
