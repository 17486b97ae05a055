"""The bench's N > 1 path runs independent replicas and reduces only the clock:
the job's seconds per iteration are the slowest rank's time over the
iterations one replica ran (not divided by the number of replicas), and the
aggregate throughput counts every replica's iterations.  Checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = [3.0, 5.0][rank]
    out[rank] = bench.job_seconds_per_iter(t_local, steps=4, world=world)
    dist.destroy_process_group()


def test_replica_timing_takes_slowest_rank():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        value, t_max, agg = out[rank]
        assert t_max == pytest.approx(5.0)
        assert value == pytest.approx(5.0 / 4)
        assert agg == pytest.approx(2 * 4 / 5.0)


def test_single_rank_needs_no_process_group():
    assert bench.job_seconds_per_iter(2.0, steps=4, world=1) == (0.5, 2.0, 2.0)
