"""Depth sharding on CPU ranks (gloo, world sizes 2 and 3): the slice assignment, ragged and empty
slices, and the gather order.  Each rank back-projects its own depth planes with the FP64 oracle
(stand-in for the GPU plan of its slice) and the gathered volume must equal the single-process
volume plane for plane."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2501_05244_gb300.sharding import depth_slices, gather_planes


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slices_are_contiguous_ragged_and_cover_every_depth():
    for Z, world in ((128, 8), (5, 2), (7, 3), (1, 2), (0, 3), (3, 3)):
        sl = depth_slices(Z, world)
        assert len(sl) == world and sl[0][0] == 0 and sl[-1][1] == Z
        assert all(a1 == b0 for (_, a1), (b0, _) in zip(sl, sl[1:]))
        sizes = [b - a for a, b in sl]
        assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        depth_slices(4, 0)


def _case(Z):
    r = np.random.default_rng(3)
    N, L, F, pitch = 8, 40, 3, 0.02
    xy = r.uniform(-0.079, 0.079, (L, 2))
    P = r.standard_normal((L, F)) + 1j * r.standard_normal((L, F))
    om = 2 * math.pi * np.array([3e9, 4e9, 5e9])
    depths = np.linspace(0.3, 0.9, Z)
    return P, xy, (0.0, 0.0), pitch, N, depths, om


def _worker(rank, world, port, Z, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P, xy, c, pitch, N, depths, om = _case(Z)
        z0, z1 = depth_slices(Z, world)[rank]
        if z1 > z0:
            local = O.nursd_forward(P, xy, c, pitch, N, depths[z0:z1], om)
        else:
            local = np.zeros((0, N, N), np.complex128)
        full = gather_planes(torch.from_numpy(local.astype(np.complex64)), Z, rank, world, dist)
        out[rank] = full.numpy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,Z", [(2, 5), (3, 7), (2, 1)])
def test_gathered_volume_equals_the_single_process_volume(world, Z):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, Z, out), nprocs=world, join=True)
        res = dict(out)
    P, xy, c, pitch, N, depths, om = _case(Z)
    ref = O.nursd_forward(P, xy, c, pitch, N, depths, om).astype(np.complex64)
    for rank in range(world):
        assert res[rank].shape == (Z, N, N)
        assert np.array_equal(res[rank], ref)  # the gather moves values, it does not compute


def test_single_rank_gather_is_identity():
    x = torch.randn(4, 3, 3, dtype=torch.complex64)
    assert gather_planes(x, 4, 0, 1, None) is x
    with pytest.raises(ValueError):
        gather_planes(x, 5, 0, 1, None)
