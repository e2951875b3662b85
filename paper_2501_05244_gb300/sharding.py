"""Depth sharding of one reconstruction over several GPUs, one process per GPU.

The operator has no exchange between depth planes (each plane is Eq. RSD_conv of the same spectrum
with its own transfer function, summed over frequency): rank r builds a plan for a contiguous slice
of the depths -- its slice of the transfer-function table, the one large per-depth array -- and
reconstructs those planes from the same relay samples and histograms; the planes are then gathered
in depth order.  The gather is the only collective: an all_gather of equal-sized, zero-padded
slices (NCCL for CUDA tensors, gloo for host tensors), after which every rank holds the volume.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def depth_slices(Z: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous slices [z0, z1) of Z depths over `world` ranks, sizes differing by at most one (the
    first Z % world ranks take one more); ranks beyond Z get an empty slice."""
    if Z < 0 or world < 1:
        raise ValueError("need Z >= 0 and world >= 1")
    base, extra = divmod(Z, world)
    out, z0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z0, z0 + n))
        z0 += n
    return out


def gather_planes(local, Z: int, rank: int, world: int, dist, group=None):
    """All-gather of the ranks' plane slices [Z_r][...] into the full [Z][...] volume on every rank.

    Slices are padded to the largest slice size so that every rank contributes a tensor of one shape;
    the padding is dropped again in rank (= depth) order.  `dist` is torch.distributed (or None for a
    single rank)."""
    import torch

    slices = depth_slices(Z, world)
    z0, z1 = slices[rank]
    if local.shape[0] != z1 - z0:
        raise ValueError(f"rank {rank} holds {local.shape[0]} planes, its slice is {z1 - z0}")
    if dist is None or world == 1:
        return local
    zmax = max(b - a for a, b in slices)
    pad = torch.zeros((zmax,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    wire = torch.view_as_real(pad) if pad.is_complex() else pad  # collectives carry real values
    parts = [torch.empty_like(wire) for _ in range(world)]
    dist.all_gather(parts, wire.contiguous(), group=group)
    if pad.is_complex():
        parts = [torch.view_as_complex(p) for p in parts]
    return torch.cat([parts[r][: b - a] for r, (a, b) in enumerate(slices)], dim=0)


class DepthShardedPlan:
    """A plan over this rank's slice of the depths; reconstruct() returns the whole gathered volume."""

    def __init__(self, N: int, pitch: float, center, depths, omega, weight=None, rank: int = 0, world: int = 1,
                 dist=None, group=None, **plan_kw):
        from .nursd import Plan

        self.depths = np.ascontiguousarray(depths, dtype=np.float64)
        self.Z, self.N, self.rank, self.world, self.dist, self.group = len(self.depths), int(N), rank, world, dist, group
        self.slice = depth_slices(self.Z, world)[rank]
        z0, z1 = self.slice
        self.plan = (Plan(N, pitch, center, self.depths[z0:z1], omega, weight, **plan_kw) if z1 > z0 else None)
        self._magnitude = bool(plan_kw.get("magnitude", False))

    def reconstruct(self, xy, hist, stream=None):
        """Positions + histograms -> the full [Z][N][N] volume (this rank's planes, then the gather)."""
        import torch

        if self.plan is not None:
            local = self.plan.reconstruct(xy, hist, stream=stream)
        else:
            dtype = torch.float32 if self._magnitude else torch.complex64
            local = torch.empty((0, self.N, self.N), dtype=dtype, device=xy.device)
        return gather_planes(local, self.Z, self.rank, self.world, self.dist, self.group)

    def close(self):
        if self.plan is not None:
            self.plan.close()
