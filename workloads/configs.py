"""Workload definitions (geometry + seeded inputs) for the NURSD benchmarks.

Sizes follow the five workloads the operator is measured on:

* tiny   : 1,024 uniform-random relay samples on a 1 m x 1 m plane, 256-bin
           histograms at 16 ps of 3 on-axis point scatterers (0.6/0.9/1.2 m),
           16 frequencies, 32x32x16 voxels over 0.5-1.5 m.
* mid    : 4,096 samples, 64x64x16 voxels (a multi-tile parity size).
* spad   : 65,536 keystone samples (16x16 spots x 16x16 SPAD pixels through a
           pinhole onto a 2 m x 2 m plane tilted 20 deg), 1,024 bins at 4 ps,
           128 frequencies, 256x256x128 voxels over 0.5-3 m.
* batched: 64 reconstructions of 4,096-65,536 samples, 512 bins at 8 ps,
           64 frequencies, 128x128x64 voxels.
* grad   : 65,536 samples, 128 frequencies, 128x128x64 voxels.

Frequency grid: F contiguous bins of a zero-padded length-``t_pad`` DFT whose
spacing 1/(t_pad*dt) makes the band 3.906 GHz wide around f_c = c/lambda_c
(lambda_c = 6 cm everywhere).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .generators import (C_LIGHT, Geometry, relay_keystone, relay_lattice, relay_uniform,
                         simulate_histograms)

BASE_SEED = 20250105


def geometry_c1() -> Geometry:
    return Geometry(name="tiny-1k", N=32, pitch=1.0 / 32, center=(0.0, 0.0),
                    depths=np.linspace(0.5, 1.5, 16), T=256, dt=16e-12, t0=0.5 / C_LIGHT,
                    lambda_c=0.06, t_pad=256, F=16)


def geometry_mid() -> Geometry:
    return Geometry(name="mid-4k", N=64, pitch=1.0 / 64, center=(0.0, 0.0),
                    depths=np.linspace(0.5, 1.5, 16), T=256, dt=16e-12, t0=0.5 / C_LIGHT,
                    lambda_c=0.06, t_pad=256, F=16)


def geometry_c2(t0: float | None = None) -> Geometry:
    return Geometry(name="spad-65k", N=256, pitch=2.0 / 256, center=(0.0, 0.0),
                    depths=np.linspace(0.5, 3.0, 128), T=1024, dt=4e-12,
                    t0=(0.9 / C_LIGHT if t0 is None else t0), lambda_c=0.06, t_pad=8192, F=128)


def geometry_c4() -> Geometry:
    return Geometry(name="batched-64", N=128, pitch=2.0 / 128, center=(0.0, 0.0),
                    depths=np.linspace(0.5, 3.0, 64), T=512, dt=8e-12, t0=0.9 / C_LIGHT,
                    lambda_c=0.06, t_pad=2048, F=64)


def geometry_c5() -> Geometry:
    return Geometry(name="grad-65k", N=128, pitch=2.0 / 128, center=(0.0, 0.0),
                    depths=np.linspace(0.5, 3.0, 64), T=1024, dt=4e-12, t0=0.9 / C_LIGHT,
                    lambda_c=0.06, t_pad=8192, F=128)


def srsd_depths_c3b(Z: int = 128) -> np.ndarray:
    """SRSD depth planes: Z planes from 1 m to 4 m (endpoints included)."""
    return np.linspace(1.0, 4.0, Z)


def srsd_pitches_c3b(depths: np.ndarray) -> np.ndarray:
    """SRSD output pitch growing linearly with depth: 8 mm at 1 m -> 32 mm at 4 m."""
    return 8e-3 * np.asarray(depths, dtype=np.float64) / 1.0


def batch_sizes_c4(B: int = 64, lo: int = 4096, hi: int = 65536, seed: int = BASE_SEED + 4) -> np.ndarray:
    """Relay-sample counts drawn log-uniformly in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=B))).astype(np.int64)


@dataclass
class Workload:
    geom: Geometry
    xy: np.ndarray          # float32 [L][2]
    hist: np.ndarray        # float32 [L][T]
    sources: np.ndarray     # float64 [S][3]


def workload_c1(seed: int = BASE_SEED + 1) -> Workload:
    g = geometry_c1()
    xy = relay_uniform(1024, 0.5, seed=seed)
    src = np.array([[0.0, 0.0, 0.6], [0.0, 0.0, 0.9], [0.0, 0.0, 1.2]])
    h = simulate_histograms(xy, src, np.ones(3), g.T, g.dt, g.t0, seed=seed + 100)
    return Workload(g, xy, h, src)


def workload_mid(seed: int = BASE_SEED + 11) -> Workload:
    g = geometry_mid()
    xy = relay_uniform(4096, 0.5, seed=seed)
    src = np.array([[0.1, -0.05, 0.7], [-0.15, 0.1, 1.0], [0.05, 0.2, 1.3]])
    h = simulate_histograms(xy, src, np.ones(3), g.T, g.dt, g.t0, seed=seed + 100)
    return Workload(g, xy, h, src)


def _c2_scene(xy: np.ndarray, seed: int):
    rng = np.random.default_rng(seed)
    src = np.stack([rng.uniform(-0.7, 0.7, 5), rng.uniform(-0.7, 0.7, 5), rng.uniform(1.0, 2.5, 5)], axis=1)
    alb = rng.uniform(0.5, 1.0, 5)
    d = np.sqrt((xy[:, None, 0].astype(np.float64) - src[None, :, 0]) ** 2
                + (xy[:, None, 1].astype(np.float64) - src[None, :, 1]) ** 2 + src[None, :, 2] ** 2)
    return src, alb, float(d.min())


def workload_c2(seed: int = BASE_SEED + 2, with_hist: bool = True) -> Workload:
    """65,536 keystone samples; t0 puts the nearest one-way path at bin 32."""
    xy = relay_keystone(seed=seed)
    src, alb, dmin = _c2_scene(xy, seed + 7)
    dt = 4e-12
    g = geometry_c2(t0=dmin / C_LIGHT - 32 * dt)
    h = simulate_histograms(xy, src, alb, g.T, g.dt, g.t0, seed=seed + 100) if with_hist else None
    return Workload(g, xy, h, src)


def workload_c2_lattice(seed: int = BASE_SEED + 2, with_hist: bool = True) -> Workload:
    """The spad-65k scene sampled on the 256x256 output lattice itself."""
    g0 = geometry_c2()
    xy = relay_lattice(g0.N, g0.pitch, g0.center)
    src, alb, dmin = _c2_scene(xy, seed + 7)
    g = geometry_c2(t0=dmin / C_LIGHT - 32 * g0.dt)
    h = simulate_histograms(xy, src, alb, g.T, g.dt, g.t0, seed=seed + 100) if with_hist else None
    return Workload(g, xy, h, src)


def workload_c5(seed: int = BASE_SEED + 5, with_hist: bool = True) -> Workload:
    """65,536 keystone samples reconstructed on the 128^2 x 64 grid of the gradient workload."""
    xy = relay_keystone(seed=seed)
    src, alb, dmin = _c2_scene(xy, seed + 7)
    g0 = geometry_c5()
    g = Geometry(name=g0.name, N=g0.N, pitch=g0.pitch, center=g0.center, depths=g0.depths, T=g0.T, dt=g0.dt,
                 t0=dmin / C_LIGHT - 32 * g0.dt, lambda_c=g0.lambda_c, t_pad=g0.t_pad, F=g0.F)
    h = simulate_histograms(xy, src, alb, g.T, g.dt, g.t0, seed=seed + 100) if with_hist else None
    return Workload(g, xy, h, src)


def batch_layouts_c4(sizes, seed: int = BASE_SEED + 40):
    """Relay layouts of the batched workload: even items uniform-random on the 2 m
    aperture, odd items the keystone layout subsampled (seeded) to the item's size."""
    rng = np.random.default_rng(seed)
    key = relay_keystone(seed=seed + 1)
    out = []
    for b, L in enumerate(np.asarray(sizes)):
        if b % 2 == 0:
            out.append(relay_uniform(int(L), 0.985, seed=seed + 100 + b))
        else:
            out.append(key[rng.choice(len(key), int(L), replace=False)])
    return out


def batch_scenes_c4(B: int, seed: int = BASE_SEED + 41):
    """Per-item point scenes (5 sources at 1-2.5 m) of the batched workload."""
    rng = np.random.default_rng(seed)
    scenes = []
    for _ in range(B):
        src = np.stack([rng.uniform(-0.7, 0.7, 5), rng.uniform(-0.7, 0.7, 5), rng.uniform(1.0, 2.5, 5)], axis=1)
        scenes.append((src, rng.uniform(0.5, 1.0, 5)))
    return scenes
