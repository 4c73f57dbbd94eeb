"""The N > 1 path of bench.py (independent replicas, one per rank) on CPU with
world_size-2 gloo: the job time is the slowest rank's on every rank, and the
reported throughput is all ranks' DOF-updates over that time."""
import os
import socket

import pytest
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
    try:
        local_s = 0.010 + 0.005 * rank      # rank 1 is the slower replica
        job_s = bench.max_over_ranks(local_s, dist, device="cpu")
        out[rank] = (job_s, bench.replica_throughput(world, 4096000, 10, job_s))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        job_s, value = out[r]
        assert job_s == pytest.approx(0.015)
        assert value == pytest.approx(2 * 4096000 * 5 * 10 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.25, None) == 0.25
    assert bench.replica_throughput(1, 100, 2, 1.0) == 1000
