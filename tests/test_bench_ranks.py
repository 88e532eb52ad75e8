"""The benchmark's multi-rank arithmetic on CPU ranks (gloo, world size 2).

The path shards by replicas only (no exchange step); what ranks share is the
barrier and the max-over-ranks time that turns per-rank work into whole-job
throughput.  Two gloo ranks run that code here.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        seconds = [1.5, 2.5][rank]  # rank 1 is the slowest
        slowest = bench.allreduce_max(seconds, world, "cpu")
        out[rank] = (slowest, bench.job_throughput(16, world, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][0] == pytest.approx(2.5)
        assert res[r][1] == pytest.approx(16 * 2 / 2.5)


def test_single_rank_is_identity():
    assert bench.allreduce_max(3.0, 1, "cpu") == 3.0
    assert bench.job_throughput(10, 1, 2.0) == 5.0
