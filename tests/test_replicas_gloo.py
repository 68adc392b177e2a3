"""The multi-GPU path of bench.py is independent replicas: no data-path
collective, one MAX reduction of the step time across ranks.  Exercised here
with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [0.004, 0.005][rank]          # seconds per step measured by each rank
    slowest = bench.max_over_ranks(local, dist, torch.device("cpu"))
    out[rank] = (slowest, bench.replica_throughput(slowest, world))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_step():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        slowest, value = out[r]
        assert slowest == pytest.approx(0.005)
        assert value == pytest.approx(2 / 0.005)
