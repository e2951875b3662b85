"""Seeded generators of synthetic NLOS inputs (no reconstruction arithmetic).

Everything here stands in for the paper's measured datasets (Sec. 7-8 use
public NLOS captures and a SPAD-array prototype, Supp. B), which are not
available: relay-sample layouts on a planar relay wall, Poisson photon-count
histograms of point scatterers, and random complex test vectors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: speed of light in vacuum [m/s]; used only to simulate photon arrival times.
C_LIGHT = 299_792_458.0


@dataclass(frozen=True)
class Geometry:
    """Acquisition and reconstruction geometry of one workload.

    N x N output lateral lattice of pitch ``pitch`` centred at ``center`` on the
    relay plane (z = 0); ``depths`` are the reconstruction planes z_v (Eq. 3);
    histograms have ``T`` bins of width ``dt`` starting at ``t0``; the phasor
    field has central wavelength ``lambda_c`` and ``F`` frequency components
    taken from a zero-padded length-``t_pad`` DFT grid (Eq. PFPacket).
    """

    name: str
    N: int
    pitch: float
    center: tuple
    depths: np.ndarray = field(compare=False)
    T: int
    dt: float
    t0: float
    lambda_c: float
    t_pad: int
    F: int
    upsample: int = 2
    kernel_width: int = 6

    @property
    def Z(self) -> int:
        return int(len(self.depths))

    @property
    def M(self) -> int:
        """Convolution size (2N: covers every relay-to-voxel offset)."""
        return 2 * self.N

    @property
    def aperture(self) -> float:
        return self.N * self.pitch


# ----------------------------------------------------------------- layouts ---

def relay_uniform(L: int, half_extent: float, center=(0.0, 0.0), seed: int = 0) -> np.ndarray:
    """``L`` relay samples uniform-random in a square of half-width ``half_extent``.

    Returns float32 [L][2] (x, y) in metres.
    """
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-half_extent, half_extent, size=(L, 2))
    xy += np.asarray(center, dtype=np.float64)[None, :]
    return xy.astype(np.float32)


def relay_lattice(N: int, pitch: float, center=(0.0, 0.0), dtype=np.float32) -> np.ndarray:
    """All N*N points of the output lattice c + pitch*(m, n), m, n in [-N/2, N/2).

    Row-major (y outer, x inner); [N*N][2] of ``dtype`` (float32 by default).
    """
    m = (np.arange(N) - N // 2) * pitch
    X, Y = np.meshgrid(m + center[0], m + center[1], indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1).astype(dtype)


def relay_keystone(n_spots: int = 16, n_pix: int = 16, half_extent: float = 0.985,
                   tilt_deg: float = 20.0, cam_dist: float = 2.0, fov: float = 0.8,
                   jitter: float = 1e-3, center=(0.0, 0.0), seed: int = 0) -> np.ndarray:
    """Perspective-distorted SPAD-array layout (keystone) on a tilted relay plane.

    A virtual (n_spots*n_pix)^2 sensor (n_spots^2 illumination spots, each with
    an n_pix^2 SPAD array) is projected through a pinhole ``cam_dist`` metres
    from the plane centre onto a plane tilted by ``tilt_deg``.  The footprint is
    rescaled to fit inside +-``half_extent``, and each spot's group of pixels
    gets a seeded uniform jitter of +-``jitter`` metres.  float32 [L][2].
    """
    n = n_spots * n_pix
    idx = (np.arange(n) + 0.5) / n - 0.5
    a, b = np.meshgrid(idx, idx, indexing="xy")
    t = math.radians(tilt_deg)
    cam = np.array([0.0, -cam_dist * math.sin(t), cam_dist * math.cos(t)])
    fwd = -cam / np.linalg.norm(cam)
    right = np.array([1.0, 0.0, 0.0])
    up = np.cross(fwd, right)
    d = fwd[None, None, :] + fov * (a[..., None] * right[None, None, :] + b[..., None] * up[None, None, :])
    s = -cam[2] / d[..., 2]
    p = cam[None, None, :] + s[..., None] * d
    xy = p[..., :2]
    lo = xy.reshape(-1, 2).min(axis=0)
    hi = xy.reshape(-1, 2).max(axis=0)
    mid = 0.5 * (lo + hi)
    scale = half_extent / (0.5 * float(np.max(hi - lo)))
    xy = (xy - mid) * scale
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter, jitter, size=(n_spots, n_spots, 2))
    spot = np.arange(n) // n_pix
    xy = xy + jit[spot[:, None], spot[None, :]]
    xy = xy.reshape(-1, 2) + np.asarray(center)[None, :]
    return xy.astype(np.float32)


# -------------------------------------------------------------- histograms ---

def simulate_histograms(xy: np.ndarray, sources: np.ndarray, albedo: np.ndarray, T: int,
                        dt: float, t0: float, peak_counts: float = 100.0,
                        background: float = 0.01, fwhm: float = 65e-12,
                        seed: int = 0, chunk: int = 4096) -> np.ndarray:
    """Poisson photon counts H(x_l, t_n) of phasor-field point sources.

    Each source at ``sources[s]`` (x, y, z) emits a Gaussian pulse of FWHM
    ``fwhm`` (65 ps, the system response of Supp. B) that reaches relay sample
    x_l after the one-way time |x_s - x_l| / c with amplitude albedo / r^2.
    The expected counts are scaled so the brightest bin has ``peak_counts``,
    a uniform background of ``background * peak_counts`` is added, and the
    counts are Poisson-sampled.  float32 [L][T].
    """
    xy = np.asarray(xy, dtype=np.float64)
    L = xy.shape[0]
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    t = t0 + dt * np.arange(T)
    mean = np.zeros((L, T), dtype=np.float64)
    for s0 in range(0, L, chunk):
        s1 = min(L, s0 + chunk)
        acc = np.zeros((s1 - s0, T))
        for src, alb in zip(np.asarray(sources, dtype=np.float64), albedo):
            d = np.sqrt((xy[s0:s1, 0] - src[0]) ** 2 + (xy[s0:s1, 1] - src[1]) ** 2 + src[2] ** 2)
            amp = alb / d ** 2
            acc += amp[:, None] * np.exp(-((t[None, :] - d[:, None] / C_LIGHT) ** 2) / (2 * sig * sig))
        mean[s0:s1] = acc
    mx = mean.max()
    if mx > 0:
        mean *= peak_counts / mx
    mean += background * peak_counts
    rng = np.random.default_rng(seed)
    return rng.poisson(mean).astype(np.float32)


# ---------------------------------------------------------- random vectors ---

def random_phasors(L: int, F: int, seed: int = 0) -> np.ndarray:
    """Complex standard-normal phasors, complex64 [L][F]."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((L, F)) + 1j * rng.standard_normal((L, F))).astype(np.complex64) / np.float32(math.sqrt(2))


def random_spectrum(M: int, F: int, seed: int = 0) -> np.ndarray:
    """Complex standard-normal spectrum, complex64 [M ky][M kx][F] (f fastest)."""
    rng = np.random.default_rng(seed)
    s = rng.standard_normal((M, M, F)) + 1j * rng.standard_normal((M, M, F))
    return (s / math.sqrt(2)).astype(np.complex64)


def random_plane_points(Z: int, K: int, half_extent: float, center=(0.0, 0.0), seed: int = 0) -> np.ndarray:
    """``K`` uniform-random (x, y) voxel positions on each of ``Z`` planes, float32 [Z][K][2]."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(-half_extent, half_extent, size=(Z, K, 2)) + np.asarray(center)[None, None, :]
    return p.astype(np.float32)


def lattice_plane_points(Z: int, N: int, pitch: float, center=(0.0, 0.0)) -> np.ndarray:
    """The N*N lattice voxels repeated on each of ``Z`` planes, float32 [Z][N*N][2]."""
    lat = relay_lattice(N, pitch, center)
    return np.broadcast_to(lat[None], (Z,) + lat.shape).copy()


def device_histograms(xy, sources, albedo, T: int, dt: float, t0: float, peak_counts: float = 100.0,
                      background: float = 0.01, fwhm: float = 65e-12, seed: int = 0, device="cuda"):
    """:func:`simulate_histograms` generated on a torch device (for multi-GB batches).

    Same model (Gaussian pulses at the one-way delays, amplitude albedo / r^2,
    peak scaled to ``peak_counts`` over this call, 1% uniform background,
    Poisson counts), drawn with a seeded torch generator.  ``xy`` is a float32
    tensor [L][2] on ``device``; returns float32 [L][T] on ``device``.
    """
    import torch

    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    t = t0 + dt * torch.arange(T, device=device, dtype=torch.float64)
    xyd = xy.to(torch.float64)
    mean = torch.zeros((xy.shape[0], T), device=device, dtype=torch.float64)
    for src, alb in zip(np.asarray(sources, dtype=np.float64), np.asarray(albedo, dtype=np.float64)):
        d = torch.sqrt((xyd[:, 0] - src[0]) ** 2 + (xyd[:, 1] - src[1]) ** 2 + src[2] ** 2)
        mean += (alb / d ** 2)[:, None] * torch.exp(-((t[None, :] - d[:, None] / C_LIGHT) ** 2) / (2 * sig * sig))
    mx = mean.max()
    if float(mx) > 0:
        mean *= peak_counts / mx
    mean += background * peak_counts
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.poisson(mean.to(torch.float32), generator=g)
