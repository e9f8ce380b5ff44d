"""Multi-rank bench aggregation (replicas) on CPU with the gloo backend:
value = ranks x steps / slowest rank's time, and only rank 0 prints."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank  # rank 1 is slower
    ms_max, value = bench.aggregate_ranks(ms, 20, world)
    out[rank] = (ms_max, value)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms_max, value = out[r]
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 20 / 0.150)


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate_ranks(50.0, 10, 1) == (50.0, pytest.approx(200.0))
