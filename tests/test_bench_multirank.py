"""Host logic of the multi-GPU bench path on CPU: two gloo ranks agree on the
slowest rank's time and on the whole-job throughput (replicas, weak scaling)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = [2.0, 3.5][rank]          # rank 1 is the slow one
    value, tmax = bench.job_value(secs, 10, world, torch.device("cpu"))
    bench.barrier(world)
    out[rank] = (value, tmax)
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank_and_the_job_total():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, tmax = out[r]
        assert tmax == 3.5
        assert value == pytest.approx(world * 10 / 3.5)
