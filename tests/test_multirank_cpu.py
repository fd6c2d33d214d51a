"""The multi-GPU path is replicas only (the single-grid PSATD step has no exchange):
each rank advances its own grid, the job time is the slowest rank's.  Checked here
with two gloo ranks on CPU (no GPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]                      # rank 1 is the slow one
    value, t_max = bench.replica_throughput(ms, 1000, 10, world, torch.device("cpu"))
    out[rank] = (value, t_max)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t_max = res[rank]
        assert t_max == 150.0
        assert value == pytest.approx(world * 1000 * 10 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    value, t_max = bench.replica_throughput(50.0, 2048 * 2048, 100, 1, torch.device("cpu"))
    assert t_max == 50.0 and value == pytest.approx(2048 * 2048 * 100 / 0.05)
