"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2):
max-over-ranks timing and whole-job throughput for independent
reconstructions per rank (weak scaling, no data-path collective)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 2.0 + rank  # rank 1 is the slower one
        ms = bench.reduce_max(ms_local, dist)
        value = bench.job_throughput(1.0e9, world, ms)
        dist.barrier()
        out[rank] = (ms, value, bench.dist_env())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_throughput():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value, env = res[rank]
        assert ms == 3.0
        assert value == pytest.approx(1.0e9 * 2 / 3.0e-3)
        assert env == (rank, world, 0)


def test_single_process_reduce_is_identity():
    assert bench.reduce_max(1.5, None) == 1.5
    assert bench.job_throughput(10.0, 1, 1000.0) == 10.0
