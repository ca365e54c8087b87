"""The benchmark's multi-rank aggregation on two gloo ranks (CPU): the timed
region is the slowest rank's, and the value counts the units of every rank
(independent ensemble replicas, no data-path collective)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 3.0][rank]
    tmax = bench.max_over_ranks(seconds, world)
    value = bench.whole_job_rate(20 * 10, world, tmax)
    out[rank] = (tmax, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        tmax, value = out[r]
        assert tmax == 3.0
        assert value == pytest.approx(20 * 10 * 2 / 3.0)
