"""FP64 CPU oracle of the NURSD / SRSD operator (arXiv 2501.05244).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline legs of ``bench.py``; never by the CUDA product path.

Everything is a direct, unfused statement of the paper's definitions in FP64:
non-uniform and scaled transforms are explicit sums (matrix products of
explicit exponentials), uniform length-M DFTs of the transfer function use
``numpy.fft`` as a textbook routine.  Conventions (readings of the paper where it
is ambiguous or silent):

* index sets I_L = {l : -L/2 <= l < L/2} (Sec. 4.1), row-major arrays with x
  fastest: ``U[f][ky][kx]``, ``V[z][my][mx]``;
* forward DFTs carry e^{-i}, the temporal transform e^{-i w t}, and the
  back-propagation kernel is G = e^{+i k r} / r (Eq. 3), so a delay tau gives a
  phasor e^{-i w tau} that G cancels at focus;
* relay positions map to theta = 2 pi (x - c) / (M delta) in [-pi/2, pi/2]
  (the rescaling to [-pi, pi) of Sec. 6);
* the phasor-field band-pass uses sigma_w = w_c / 5 (Eq. PFPacket read in
  frequency units) on F contiguous bins of a zero-padded length-t_pad DFT.

Parity status: every public function below is pinned by ``tests/test_oracle_*``
(closed forms, brute force, on-lattice equality with direct back-projection,
adjoint identity, finite differences).
"""
from __future__ import annotations

import math

import numpy as np

C = 299_792_458.0  # speed of light [m/s]

__all__ = [
    "C", "index_set", "phasor_frequencies", "temporal_dft", "relay_theta",
    "nudft_type1", "nudft_type1_modes", "nudft_type2", "rsd_kernel", "transfer_function",
    "transfer_functions", "propagate", "propagate_depth", "nursd_forward", "fbp_direct",
    "propagate_points", "idft_grid", "scaled_dft_matrix", "srsd_from_grid", "srsd_forward",
    "adjoint_spectrum", "nursd_adjoint", "nursd_loss", "nursd_gradients",
    "adjoint_spectrum_depthwise", "nudft_type1_lattice", "gradients_from_w", "position_loss_differences",
    "downsampling_bound", "subsample_grid", "upsample_nearest", "upsample_linear", "frustum_volume", "frustum_extra_volume", "data_compression", "lateral_resolution",
    "voxel_lattice", "propagate_per_frequency", "illumination_mask", "propagate_illuminated", "transient_frames",
    "nursd_forward_illuminated", "nursd_transient_frames", "fbp_direct_per_frequency",
    "srsd_spectra", "srsd_points", "nu_sfft_spectra", "nu_sfft_forward",
    "rsd_kernel_3d", "nursd3d_plane", "nursd3d_forward",
]


# --------------------------------------------------------------- notation ---

def index_set(L: int) -> np.ndarray:
    """I_L = {l in Z : -L/2 <= l < L/2} (Sec. 4.1, used for modes and lattices)."""
    return np.arange(-(L // 2), L - L // 2)


# ------------------------------------------------- a1: temporal transform ---

def phasor_frequencies(lambda_c: float, dt: float, t_pad: int, F: int):
    """Frequencies and Gaussian weights of the phasor-field kernel (Eq. PFPacket).

    lambda_c = 2 pi c / w_c; the filter is exp(-(w - w_c)^2 / (2 sigma^2)) with
    sigma = w_c / 5 (the paper's sigma = c / (5 lambda_c) read as a frequency).
    The F frequencies are contiguous bins of a length-``t_pad`` DFT of step
    ``dt``: w_f = 2 pi (f0 + f) / (t_pad dt), f0 = round(f_c t_pad dt) - F/2.
    Returns (omega [F] rad/s, weight [F]).
    """
    f_c = C / lambda_c
    f0 = math.floor(f_c * t_pad * dt + 0.5) - F // 2
    omega = 2.0 * math.pi * (f0 + np.arange(F, dtype=np.float64)) / (t_pad * dt)
    omega_c = 2.0 * math.pi * f_c
    sigma = omega_c / 5.0
    weight = np.exp(-((omega - omega_c) ** 2) / (2.0 * sigma * sigma))
    return omega, weight


def temporal_dft(h: np.ndarray, t0: float, dt: float, omega: np.ndarray, weight: np.ndarray) -> np.ndarray:
    """Phasors P[l, f] = w_f * sum_n h_l[n] exp(-i w_f (t0 + n dt)) (Eq. PF_Response).

    The virtual response is the histogram convolved with the phasor-field
    illumination; in the frequency domain that is the histogram's DTFT at w_f
    times the filter weight.  h: [L][T] -> complex128 [L][F].
    """
    h = np.asarray(h, dtype=np.float64)
    t = t0 + dt * np.arange(h.shape[1], dtype=np.float64)
    E = np.exp(-1j * t[:, None] * np.asarray(omega, dtype=np.float64)[None, :])
    return (h @ E) * np.asarray(weight, dtype=np.float64)[None, :]


# ------------------------------------------- a2-a5: non-uniform transforms ---

def relay_theta(xy: np.ndarray, center, pitch: float, M: int) -> np.ndarray:
    """Rescale metric positions to the NUFFT's periodic domain (Sec. 6).

    theta = 2 pi (x - c) / (M delta): the M-point lattice c + delta*I_M maps to
    2 pi I_M / M, so the aperture |x - c| <= N delta / 2 lands in [-pi/2, pi/2].
    """
    xy = np.asarray(xy, dtype=np.float64)
    c = np.asarray(center, dtype=np.float64)
    return 2.0 * math.pi * (xy - c[None, :]) / (M * pitch)


def nudft_type1(P: np.ndarray, theta: np.ndarray, M: int) -> np.ndarray:
    """Type-1 non-uniform DFT, U_f[ky, kx] = sum_l P[l, f] exp(-i (kx th_x + ky th_y)).

    (Sec. 6, NUFFT-1) evaluated exactly for every mode (kx, ky) in I_M^2 by the
    separable product of explicit exponentials.  P: [L][F] -> [F][M][M].
    """
    P = np.asarray(P, dtype=np.complex128)
    k = index_set(M).astype(np.float64)
    Ex = np.exp(-1j * k[:, None] * theta[None, :, 0])  # [kx][l]
    Ey = np.exp(-1j * k[:, None] * theta[None, :, 1])  # [ky][l]
    U = np.empty((P.shape[1], M, M), dtype=np.complex128)
    for f in range(P.shape[1]):
        U[f] = (Ey * P[None, :, f]) @ Ex.T
    return U


def nudft_type1_modes(P: np.ndarray, theta: np.ndarray, kxy: np.ndarray) -> np.ndarray:
    """Type-1 sum at selected modes only: out[q, f] = sum_l P[l, f] e^{-i k_q . theta_l}."""
    kxy = np.asarray(kxy, dtype=np.float64)
    E = np.exp(-1j * (kxy[:, 0:1] * theta[None, :, 0] + kxy[:, 1:2] * theta[None, :, 1]))
    return E @ np.asarray(P, dtype=np.complex128)


def nudft_type2(U: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Type-2 non-uniform DFT, u[l, f] = sum_k U_f[k] exp(+i (kx th_x + ky th_y)).

    (Sec. 6, NUFFT-2: the adjoint of type 1.)  U: [F][M][M] -> [L][F].
    """
    U = np.asarray(U, dtype=np.complex128)
    M = U.shape[-1]
    k = index_set(M).astype(np.float64)
    Ex = np.exp(1j * k[:, None] * theta[None, :, 0])  # [kx][l]
    Ey = np.exp(1j * k[:, None] * theta[None, :, 1])  # [ky][l]
    out = np.empty((theta.shape[0], U.shape[0]), dtype=np.complex128)
    for f in range(U.shape[0]):
        out[:, f] = np.sum(Ey * (U[f] @ Ex), axis=0)
    return out


# ------------------------------------------- a6-a7: RSD propagation -------

def rsd_kernel(M: int, pitch: float, z: float, k: float) -> np.ndarray:
    """Propagation kernel G(j delta, z) = exp(+i k r) / r on the M x M offsets j in I_M^2.

    r = sqrt((jx delta)^2 + (jy delta)^2 + z^2) (Eq. RSD_conv); [jy][jx].
    """
    j = index_set(M).astype(np.float64) * pitch
    r = np.sqrt(j[None, :] ** 2 + j[:, None] ** 2 + z * z)
    return np.exp(1j * k * r) / r


def transfer_function(g: np.ndarray) -> np.ndarray:
    """Transfer function Ghat[k] = sum_{j in I_M^2} g[j] exp(-2 pi i k.j / M), k in I_M^2.

    (The FFT{G} factor of Eq. 4.)  A plain length-M 2D DFT with centred index
    sets, computed with numpy.fft (shifts move index 0 to the front and back).
    """
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(g)))


def transfer_functions(depths, omega, M: int, pitch: float, confocal: bool = False) -> np.ndarray:
    """Ghat[z][f][ky][kx] for every depth plane and frequency (k_f = w_f / c).

    confocal: every relay point both illuminates and detects, so the phasor-field point source
    radiates e^{i 2 k r} (Supp., confocal systems) and the kernel takes k_con = 2 k_f.
    """
    depths = np.asarray(depths, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    kmul = 2.0 if confocal else 1.0
    out = np.empty((len(depths), len(omega), M, M), dtype=np.complex128)
    for iz, z in enumerate(depths):
        for f, w in enumerate(omega):
            out[iz, f] = transfer_function(rsd_kernel(M, pitch, z, kmul * w / C))
    return out


def _idft_crop_matrix(M: int, N: int) -> np.ndarray:
    """B[m, k] = exp(+2 pi i k m / M) for m in I_N, k in I_M."""
    m = index_set(N).astype(np.float64)
    k = index_set(M).astype(np.float64)
    return np.exp(2j * math.pi * np.outer(m, k) / M)


def propagate(U: np.ndarray, Ghat: np.ndarray, N: int) -> np.ndarray:
    """NURSD-1 propagation and coherent frequency sum (Eq. NURSD1 with Eq. PF_RSD_Defn).

    Y_z(k) = sum_f U_f(k) Ghat_{z,f}(k), then the inverse DFT evaluated on the
    N x N output lattice: V_z[m] = M^-2 sum_k Y_z(k) exp(+2 pi i k.m / M),
    m in I_N^2.  U: [F][M][M], Ghat: [Z][F][M][M] -> V: [Z][N][N].
    """
    M = U.shape[-1]
    Y = np.einsum("fyx,zfyx->zyx", U, Ghat)
    B = _idft_crop_matrix(M, N)
    return np.stack([B @ Y[z] @ B.T for z in range(Y.shape[0])]) / (M * M)


def propagate_depth(U: np.ndarray, z: float, omega, pitch: float, N: int) -> np.ndarray:
    """One depth plane of :func:`propagate`, building Ghat_{z,f} one frequency at a time."""
    M = U.shape[-1]
    Y = np.zeros((M, M), dtype=np.complex128)
    for f, w in enumerate(np.asarray(omega, dtype=np.float64)):
        Y += U[f] * transfer_function(rsd_kernel(M, pitch, z, w / C))
    B = _idft_crop_matrix(M, N)
    return (B @ Y @ B.T) / (M * M)


def nursd_forward(P, xy, center, pitch: float, N: int, depths, omega, confocal: bool = False) -> np.ndarray:
    """The full NURSD-1 operator: phasors at irregular relay samples -> V[z][my][mx].

    IFFT{ NUFFT-1{P_F(x_l)} . FFT{G(m delta, n delta, z_v)} } (Eq. NURSD1), with the
    frequency integral of Eq. PF_RSD_Defn taken as the sum over the F phasor bins;
    confocal as in :func:`transfer_functions`.
    """
    M = 2 * N
    U = nudft_type1(P, relay_theta(xy, center, pitch, M), M)
    return propagate(U, transfer_functions(depths, omega, M, pitch, confocal), N)


def fbp_direct(P, xy, omega, vox, chunk: int = 256) -> np.ndarray:
    """Direct back-projection (the gold-standard sum of Eq. PF_RSD_Defn's inner integral).

    V(x_v) = sum_f sum_l P[l, f] exp(+i k_f |x_v - x_l|) / |x_v - x_l|, relay
    samples on z = 0, voxels ``vox`` [V][3] (x, y, z).  Costs L*F per voxel.
    """
    P = np.asarray(P, dtype=np.complex128)
    xy = np.asarray(xy, dtype=np.float64)
    vox = np.asarray(vox, dtype=np.float64)
    k = np.asarray(omega, dtype=np.float64) / C
    out = np.zeros(vox.shape[0], dtype=np.complex128)
    for v0 in range(0, vox.shape[0], chunk):
        v = vox[v0:v0 + chunk]
        r = np.sqrt((v[:, None, 0] - xy[None, :, 0]) ** 2 + (v[:, None, 1] - xy[None, :, 1]) ** 2
                    + v[:, None, 2] ** 2)
        acc = np.zeros(v.shape[0], dtype=np.complex128)
        for f in range(P.shape[1]):
            acc += (np.exp(1j * k[f] * r) / r) @ P[:, f]
        out[v0:v0 + chunk] = acc
    return out


# ------------------------------- per-frequency forms: illumination, video ---

def voxel_lattice(center, pitch: float, N: int, depths) -> np.ndarray:
    """Voxel positions x_v = (c_x + mx delta, c_y + my delta, z) of V[z][my][mx], m in I_N: [Z][N][N][3]."""
    m = index_set(N).astype(np.float64) * pitch
    Z = len(depths)
    out = np.empty((Z, N, N, 3))
    out[..., 0] = center[0] + m[None, None, :]
    out[..., 1] = center[1] + m[None, :, None]
    out[..., 2] = np.asarray(depths, dtype=np.float64)[:, None, None]
    return out


def propagate_per_frequency(U: np.ndarray, Ghat: np.ndarray, N: int) -> np.ndarray:
    """Each frequency's reconstruction before the coherent sum (Eq. RSD_conv per frequency).

    V_{z,f}[m] = M^-2 sum_k U_f(k) Ghat_{z,f}(k) exp(+2 pi i k.m / M), m in I_N^2.
    U: [F][M][M], Ghat: [Z][F][M][M] -> [Z][F][N][N].
    """
    M = U.shape[-1]
    B = _idft_crop_matrix(M, N)
    Z, F = Ghat.shape[0], Ghat.shape[1]
    out = np.empty((Z, F, N, N), dtype=np.complex128)
    for z in range(Z):
        for f in range(F):
            out[z, f] = B @ (U[f] * Ghat[z, f]) @ B.T / (M * M)
    return out


def illumination_mask(xp, vox: np.ndarray, omega) -> np.ndarray:
    """Illumination phase mask of Eq. PF_RSD_Defn, exp(+i k_f |x_p - x_v|), at voxels vox [...][3].

    The sign follows the temporal transform's e^{-i w t}: the path x_p -> x_v delays the
    phasor by e^{-i k |x_p - x_v|}, which this mask cancels.  Returns [F][...].
    """
    xp = np.asarray(xp, dtype=np.float64)
    d = np.sqrt(np.sum((np.asarray(vox, dtype=np.float64) - xp) ** 2, axis=-1))
    k = np.asarray(omega, dtype=np.float64) / C
    return np.exp(1j * k.reshape((-1,) + (1,) * d.ndim) * d[None])


def propagate_illuminated(U: np.ndarray, Ghat: np.ndarray, N: int, xp, center, pitch: float, depths,
                          omega) -> np.ndarray:
    """Single-illumination reconstruction (Eq. PF_RSD_Defn for one illumination point x_p).

    V_z[m] = sum_f exp(+i k_f |x_p - x_v|) V_{z,f}[m]: the illumination mask varies per voxel and
    frequency, so the frequency sum follows each frequency's inverse transform.  -> [Z][N][N].
    """
    Vf = propagate_per_frequency(U, Ghat, N)
    vox = voxel_lattice(center, pitch, N, depths)  # [Z][N][N][3]
    A = illumination_mask(xp, vox, omega)  # [F][Z][N][N]
    return np.einsum("fzyx,zfyx->zyx", A, Vf)


def transient_frames(U: np.ndarray, Ghat: np.ndarray, N: int, times, omega) -> np.ndarray:
    """Time-resolved frames of the propagating virtual wave (Eq. Video_Voxel_Freq_Offset).

    V_{t,z}[m] = sum_f exp(+i w_f t) V_{z,f}[m] for each time t (seconds, on the measurement's
    clock).  -> [T][Z][N][N].
    """
    Vf = propagate_per_frequency(U, Ghat, N)
    w = np.asarray(omega, dtype=np.float64)
    A = np.exp(1j * np.outer(np.asarray(times, dtype=np.float64), w))  # [T][F]
    return np.einsum("tf,zfyx->tzyx", A, Vf)


def nursd_forward_illuminated(P, xy, center, pitch: float, N: int, depths, omega, xp) -> np.ndarray:
    """Phasors at irregular relay samples -> single-illumination volume V[z][my][mx]."""
    M = 2 * N
    U = nudft_type1(P, relay_theta(xy, center, pitch, M), M)
    return propagate_illuminated(U, transfer_functions(depths, omega, M, pitch), N, xp, center, pitch, depths,
                                 omega)


def nursd_transient_frames(P, xy, center, pitch: float, N: int, depths, omega, times) -> np.ndarray:
    """Phasors at irregular relay samples -> frames V[t][z][my][mx]."""
    M = 2 * N
    U = nudft_type1(P, relay_theta(xy, center, pitch, M), M)
    return transient_frames(U, transfer_functions(depths, omega, M, pitch), N, times, omega)


def fbp_direct_per_frequency(P, xy, omega, vox, chunk: int = 256) -> np.ndarray:
    """Direct back-projection of each frequency on its own (Eq. PF_RSD_Defn's inner integral).

    R_f(x_v) = sum_l P[l, f] exp(+i k_f |x_v - x_l|) / |x_v - x_l|, relay samples on z = 0,
    voxels ``vox`` [V][3].  -> [V][F].
    """
    P = np.asarray(P, dtype=np.complex128)
    xy = np.asarray(xy, dtype=np.float64)
    vox = np.asarray(vox, dtype=np.float64)
    k = np.asarray(omega, dtype=np.float64) / C
    out = np.zeros((vox.shape[0], P.shape[1]), dtype=np.complex128)
    for v0 in range(0, vox.shape[0], chunk):
        v = vox[v0:v0 + chunk]
        r = np.sqrt((v[:, None, 0] - xy[None, :, 0]) ** 2 + (v[:, None, 1] - xy[None, :, 1]) ** 2
                    + v[:, None, 2] ** 2)
        for f in range(P.shape[1]):
            out[v0:v0 + chunk, f] = (np.exp(1j * k[f] * r) / r) @ P[:, f]
    return out


# ------------------------------------------- a8: arbitrary output voxels ---

def propagate_points(U: np.ndarray, Ghat: np.ndarray, theta_v: np.ndarray) -> np.ndarray:
    """NURSD-2/3 output: V_z(x_v) = M^-2 sum_k Y_z(k) exp(+i k . theta_v) (Eqs. NURSD2-3).

    Y_z as in :func:`propagate`; ``theta_v`` [Z][K][2] are the per-plane voxel
    positions rescaled like relay samples.  Returns [Z][K].
    """
    M = U.shape[-1]
    Y = np.einsum("fyx,zfyx->zyx", U, Ghat)
    out = np.empty(theta_v.shape[:2], dtype=np.complex128)
    for z in range(Y.shape[0]):
        out[z] = nudft_type2(Y[z][None], theta_v[z])[:, 0] / (M * M)
    return out


# ------------------------------------------------------------ a9: SRSD ----

def idft_grid(U: np.ndarray) -> np.ndarray:
    """Gridded field u_f[n] = M^-2 sum_k U_f(k) exp(+2 pi i k.n / M), n in I_M^2.

    The regular-grid input that SRSD requires (Supp. C, SRSD on non-uniform
    acquisition: interpolate to a regular grid, here by the NUFFT-1 spectrum).
    """
    M = U.shape[-1]
    B = _idft_crop_matrix(M, M)
    return np.stack([B @ U[f] @ B.T for f in range(U.shape[0])]) / (M * M)


def scaled_dft_matrix(M: int, s: float) -> np.ndarray:
    """A[kappa, n] = exp(-2 pi i kappa n / (M s)), kappa, n in I_M (scaled DFT, Sec. 4.1).

    s = 1/alpha is the ratio of output to input pitch.
    """
    k = index_set(M).astype(np.float64)
    return np.exp(-2j * math.pi * np.outer(k, k) / (M * s))


def srsd_from_grid(u: np.ndarray, depths, scales, omega, pitch: float, N: int) -> np.ndarray:
    """Scaled RSD on a gridded input (Eq. SRSD_conv / SFFT, fusion form of Supp. C).

    Per depth z with scale s_z: Phat_{z,f} = A_z u_f A_z^T (the scaled DFT as an
    explicit sum), Y_z = sum_f Phat_{z,f} . Ghat^(s)_{z,f} where Ghat^(s) is the
    DFT of G sampled at pitch s_z delta, and V_z = M^-2 IDFT crop to I_N^2.
    The output of plane z lies on the lattice c + s_z delta I_N^2.
    u: [F][M][M] -> [Z][N][N].
    """
    M = u.shape[-1]
    B = _idft_crop_matrix(M, N)
    out = np.empty((len(depths), N, N), dtype=np.complex128)
    for iz, (z, s) in enumerate(zip(np.asarray(depths, float), np.asarray(scales, float))):
        A = scaled_dft_matrix(M, s)
        Y = np.zeros((M, M), dtype=np.complex128)
        for f, w in enumerate(np.asarray(omega, dtype=np.float64)):
            Y += (A @ u[f] @ A.T) * transfer_function(rsd_kernel(M, s * pitch, z, w / C))
        out[iz] = (B @ Y @ B.T) / (M * M)
    return out


def srsd_forward(P, xy, center, pitch: float, N: int, depths, scales, omega) -> np.ndarray:
    """SRSD of non-uniform relay samples: NUFFT-1 spectrum -> grid -> scaled RSD."""
    M = 2 * N
    U = nudft_type1(P, relay_theta(xy, center, pitch, M), M)
    return srsd_from_grid(idft_grid(U), depths, scales, omega, pitch, N)


def srsd_spectra(u: np.ndarray, depths, scales, omega, pitch: float) -> np.ndarray:
    """The scaled spectra of :func:`srsd_from_grid` before its inverse transform.

    Y^S_z = sum_f (A_z u_f A_z^T) . Ghat^(s_z)_{z,f}, A_z the scaled DFT with s_z and Ghat^(s_z)
    the DFT of G sampled at pitch s_z delta.  u: [F][M][M] -> [Z][M][M].
    """
    M = u.shape[-1]
    out = np.empty((len(depths), M, M), dtype=np.complex128)
    for iz, (z, s) in enumerate(zip(np.asarray(depths, float), np.asarray(scales, float))):
        A = scaled_dft_matrix(M, s)
        Y = np.zeros((M, M), dtype=np.complex128)
        for f, w in enumerate(np.asarray(omega, dtype=np.float64)):
            Y += (A @ u[f] @ A.T) * transfer_function(rsd_kernel(M, s * pitch, z, w / C))
        out[iz] = Y
    return out


def srsd_points(P, xy, center, pitch: float, N: int, depths, scales, omega, vox_xy) -> np.ndarray:
    """SRSD + NURSD-2 (Eq. NURSD2_SRSD): the scaled reconstruction at arbitrary voxels of each plane.

    V_z(x_v) = M^-2 sum_kappa Y^S_z(kappa) exp(+i kappa . theta_v) with theta_v = 2 pi (x_v - c) /
    (M s_z delta): the type-2 sum on plane z's scaled lattice, whose lattice points
    c + s_z delta m give back the SRSD output.  vox_xy: [Z][K][2] metres -> [Z][K].
    """
    M = 2 * N
    U = nudft_type1(P, relay_theta(xy, center, pitch, M), M)
    Y = srsd_spectra(idft_grid(U), depths, scales, omega, pitch)
    vox = np.asarray(vox_xy, dtype=np.float64)
    out = np.empty(vox.shape[:2], dtype=np.complex128)
    for iz, s in enumerate(np.asarray(scales, float)):
        theta = 2 * math.pi * (vox[iz] - np.asarray(center, dtype=np.float64)) / (M * s * pitch)
        out[iz] = nudft_type2(Y[iz][None], theta)[:, 0] / (M * M)
    return out


def nu_sfft_spectra(P, xy, center, pitch: float, N: int, depths, scales, omega) -> np.ndarray:
    """Scaled spectra of the non-uniform-input SRSD (NU-SFFT, Supp. C, SRSD on non-uniform acquisition).

    The scaled DFT taken directly at the relay samples instead of a gridded input:
    Phat_{z,f}(kappa) = sum_l P[l, f] exp(-i kappa . theta_l / s_z), kappa in I_M^2, theta_l the
    rescaled positions of Sec. 6; then Y_z = sum_f Phat_{z,f} . Ghat^(s_z)_{z,f} as in SRSD.
    P [L][F] -> [Z][M][M], M = 2N.
    """
    M = 2 * N
    theta = relay_theta(xy, center, pitch, M)
    out = np.empty((len(depths), M, M), dtype=np.complex128)
    for iz, (z, s) in enumerate(zip(np.asarray(depths, float), np.asarray(scales, float))):
        Ph = nudft_type1(P, theta / s, M)
        Y = np.zeros((M, M), dtype=np.complex128)
        for f, w in enumerate(np.asarray(omega, dtype=np.float64)):
            Y += Ph[f] * transfer_function(rsd_kernel(M, s * pitch, z, w / C))
        out[iz] = Y
    return out


def nu_sfft_forward(P, xy, center, pitch: float, N: int, depths, scales, omega) -> np.ndarray:
    """NU-SFFT reconstruction: :func:`nu_sfft_spectra`, then V_z = M^-2 IDFT crop to I_N^2 (plane z on the
    lattice c + s_z delta I_N^2, like SRSD).  -> [Z][N][N]."""
    M = 2 * N
    Y = nu_sfft_spectra(P, xy, center, pitch, N, depths, scales, omega)
    B = _idft_crop_matrix(M, N)
    return np.stack([B @ Y[iz] @ B.T for iz in range(Y.shape[0])]) / (M * M)


# ------------------------------------------------ 3D NURSD (non-planar relays) ---

def rsd_kernel_3d(M: int, pitch: float, Mz: int, dz: float, k: float) -> np.ndarray:
    """G(j delta, jz dz) = exp(+i k r) / r on the offsets j in I_M^2, jz in I_Mz: [jz][jy][jx], r = sqrt((jx delta)^2 +
    (jy delta)^2 + (jz dz)^2), with G = 0 at the zero offset where r = 0 (a reading: the paper leaves it undefined)."""
    j = index_set(M).astype(np.float64) * pitch
    jz = index_set(Mz).astype(np.float64) * dz
    r = np.sqrt(jz[:, None, None] ** 2 + j[None, :, None] ** 2 + j[None, None, :] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.exp(1j * k * r) / r
    g[r == 0.0] = 0.0
    return g


def nursd3d_plane(P, xyz, center, pitch: float, N: int, z0: float, dz: float, Mz: int, omega) -> np.ndarray:
    """Stage 1 of 3D NURSD (Eq. 3D_NURSD, with Eq. 3d_rsd): each frequency's field on the N x N lattice of plane z0.

    The 3D type-1 sum U_f(k) = sum_l P[l, f] exp(-i k . theta_l) over k in I_M^2 x I_Mz with
    theta_l = (2 pi (x_l - c_x) / (M delta), 2 pi (y_l - c_y) / (M delta), 2 pi (z_l - z0) / (Mz dz)), times the 3D
    DFT of the sampled kernel (rsd_kernel_3d), inverse-transformed and evaluated at the slice z = z0 and the
    lattice m in I_N^2: W_f[m] = (M^2 Mz)^-1 sum_k U_f(k) Ghat_f(k) exp(+2 pi i (kx mx + ky my) / M).
    P [L][F], xyz [L][3] metres -> [F][N][N].
    """
    M = 2 * N
    P = np.asarray(P, dtype=np.complex128)
    xyz = np.asarray(xyz, dtype=np.float64)
    c = np.asarray(center, dtype=np.float64)
    th = np.stack([2 * math.pi * (xyz[:, 0] - c[0]) / (M * pitch), 2 * math.pi * (xyz[:, 1] - c[1]) / (M * pitch),
                   2 * math.pi * (xyz[:, 2] - z0) / (Mz * dz)], axis=1)
    k = index_set(M).astype(np.float64)
    kz = index_set(Mz).astype(np.float64)
    Ex = np.exp(-1j * np.outer(k, th[:, 0]))   # [kx][l]
    Ey = np.exp(-1j * np.outer(k, th[:, 1]))   # [ky][l]
    Ez = np.exp(-1j * np.outer(kz, th[:, 2]))  # [kz][l]
    B = _idft_crop_matrix(M, N)                # [m][k]
    out = np.empty((P.shape[1], N, N), dtype=np.complex128)
    for f, w in enumerate(np.asarray(omega, dtype=np.float64)):
        U = np.einsum("zl,yl,xl,l->zyx", Ez, Ey, Ex, P[:, f])  # explicit 3D non-uniform sum
        g = rsd_kernel_3d(M, pitch, Mz, dz, w / C)
        G = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(g)))  # the 3D DFT (a library routine)
        Wk = np.sum(U * G, axis=0) / Mz  # the slice z = z0 of the inverse transform along kz
        out[f] = (B @ Wk @ B.T) / (M * M)
    return out


def nursd3d_forward(P, xyz, center, pitch: float, N: int, z0: float, dz: float, Mz: int, depths, omega) -> np.ndarray:
    """3D NURSD: stage 1 to plane z0 (:func:`nursd3d_plane`), then stage 2, the standard RSD of that plane to each
    depth (the planar operator with the plane's lattice field as relay samples, distances depths - z0, Supp. C).
    -> [Z][N][N]."""
    W = nursd3d_plane(P, xyz, center, pitch, N, z0, dz, Mz, omega)  # [F][N][N]
    lat = voxel_lattice(center, pitch, N, [0.0])[0, :, :, :2].reshape(-1, 2)  # row y, column x
    Pl = W.reshape(W.shape[0], -1).T  # [N*N][F] in the lattice's order
    return nursd_forward(Pl, lat, center, pitch, N, np.asarray(depths, dtype=np.float64) - z0, omega)


# --------------------------------------------------- a10-a11: adjoint, grad ---

def adjoint_spectrum(V: np.ndarray, Ghat: np.ndarray) -> np.ndarray:
    """R_f(k) = sum_z conj(Ghat_{z,f}(k)) Vt_z(k), Vt_z(k) = M^-2 sum_{m in I_N^2} V_z[m] e^{-2 pi i k.m/M}.

    The adjoint of :func:`propagate` up to the type-1 step.  V: [Z][N][N] -> [F][M][M].
    """
    M = Ghat.shape[-1]
    D = np.conj(_idft_crop_matrix(M, V.shape[-1])).T  # [k][m] = e^{-2 pi i k m / M}
    Vt = np.stack([D @ V[z] @ D.T for z in range(V.shape[0])]) / (M * M)
    return np.einsum("zfyx,zyx->fyx", np.conj(Ghat), Vt)


def nursd_adjoint(V, xy, center, pitch: float, N: int, depths, omega) -> np.ndarray:
    """A^H of :func:`nursd_forward`: V [Z][N][N] -> phasors [L][F].

    Type-2 is the adjoint of type-1 (Sec. 6), so A^H = NUFFT-2 o conj(Ghat) o DFT.
    """
    M = 2 * N
    Ghat = transfer_functions(depths, omega, M, pitch)
    return nudft_type2(adjoint_spectrum(np.asarray(V, np.complex128), Ghat),
                       relay_theta(xy, center, pitch, M))


def nursd_loss(P, xy, center, pitch, N, depths, omega, V_target) -> float:
    """L = || A(P, x) - V_target ||^2 over the complex output volume."""
    r = nursd_forward(P, xy, center, pitch, N, depths, omega) - V_target
    return float(np.sum(np.abs(r) ** 2))


def nursd_gradients(P, xy, center, pitch, N, depths, omega, V_target):
    """Analytic gradients of :func:`nursd_loss`.

    grad_P = 2 A^H (A P - V_t) (the conjugate-Wirtinger convention for a real
    loss of complex inputs); with R_f the adjoint spectrum of the residual,
    dL/dx_l = (2 pi / (M delta)) * 2 Re sum_f P[l,f] conj(sum_k i kx R_f(k) e^{i k.theta_l})
    and likewise for y.  Returns (grad_P [L][F] complex, grad_xy [L][2] real).
    """
    M = 2 * N
    P = np.asarray(P, dtype=np.complex128)
    theta = relay_theta(xy, center, pitch, M)
    Ghat = transfer_functions(depths, omega, M, pitch)
    resid = propagate(nudft_type1(P, theta, M), Ghat, N) - V_target
    R = adjoint_spectrum(resid, Ghat)
    grad_P = 2.0 * nudft_type2(R, theta)
    k = index_set(M).astype(np.float64)
    dx = nudft_type2(1j * k[None, None, :] * R, theta)
    dy = nudft_type2(1j * k[None, :, None] * R, theta)
    scale = 2.0 * math.pi / (M * pitch)
    gx = 2.0 * np.real(np.sum(P * np.conj(dx), axis=1)) * scale
    gy = 2.0 * np.real(np.sum(P * np.conj(dy), axis=1)) * scale
    return grad_P, np.stack([gx, gy], axis=1)


def adjoint_spectrum_depthwise(V: np.ndarray, depths, omega, pitch: float) -> np.ndarray:
    """:func:`adjoint_spectrum` building Ghat_{z,f} one (z, f) at a time (no full table in memory).

    V: [Z][N][N] -> R [F][M][M], M = 2N.
    """
    V = np.asarray(V, dtype=np.complex128)
    N = V.shape[-1]
    M = 2 * N
    D = np.conj(_idft_crop_matrix(M, N)).T
    omega = np.asarray(omega, dtype=np.float64)
    R = np.zeros((len(omega), M, M), dtype=np.complex128)
    for iz, z in enumerate(np.asarray(depths, dtype=np.float64)):
        Vt = (D @ V[iz] @ D.T) / (M * M)
        for f, w in enumerate(omega):
            R[f] += np.conj(transfer_function(rsd_kernel(M, pitch, z, w / C))) * Vt
    return R


def nudft_type1_lattice(P: np.ndarray, n_xy: np.ndarray, M: int) -> np.ndarray:
    """:func:`nudft_type1` for samples on the lattice, theta = 2 pi n / M with integer n in I_M.

    Then exp(-i k.theta) = exp(-2 pi i k.n / M), so the sum is the M x M DFT of the
    gridded samples (computed with numpy.fft).  P: [L][F], n_xy: [L][2] ints -> [F][M][M].
    """
    P = np.asarray(P, dtype=np.complex128)
    n_xy = np.asarray(n_xy)
    U = np.empty((P.shape[1], M, M), dtype=np.complex128)
    for f in range(P.shape[1]):
        grid = np.zeros((M, M), dtype=np.complex128)
        np.add.at(grid, (n_xy[:, 1] + M // 2, n_xy[:, 0] + M // 2), P[:, f])
        U[f] = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(grid)))
    return U


def gradients_from_w(R: np.ndarray, P_rows: np.ndarray, theta_rows: np.ndarray, pitch: float):
    """Gradients at selected samples given the adjoint spectrum R of w = 2 dL/d conj(V).

    grad_P[l] = sum_k R_f(k) e^{i k.theta_l} (= A^H w), and
    grad_x[l] = (2 pi / (M delta)) Re sum_f P[l,f] conj(sum_k i kx R_f(k) e^{i k.theta_l})
    (likewise y).  R: [F][M][M]; P_rows [S][F]; theta_rows [S][2].
    """
    M = R.shape[-1]
    k = index_set(M).astype(np.float64)
    gP = nudft_type2(R, theta_rows)
    dx = nudft_type2(1j * k[None, None, :] * R, theta_rows)
    dy = nudft_type2(1j * k[None, :, None] * R, theta_rows)
    scale = 2.0 * math.pi / (M * pitch)
    P_rows = np.asarray(P_rows, dtype=np.complex128)
    gx = np.real(np.sum(P_rows * np.conj(dx), axis=1)) * scale
    gy = np.real(np.sum(P_rows * np.conj(dy), axis=1)) * scale
    return gP, np.stack([gx, gy], axis=1)


def position_loss_differences(residual, P_rows, xy_rows, axes, h: float, center, pitch: float, N: int, depths,
                              omega) -> np.ndarray:
    """Central differences of L = ||A(P, x) - V_t||^2 in one coordinate of one relay sample each.

    Moving sample l changes only its own term of the forward sum (Eq. NURSD1), so with the residual
    r = A(P, x) - V_t, L(x + d) - L(x - d) = 2 Re <r, dV+ - dV-> + ||dV+||^2 - ||dV-||^2, where
    dV+ - dV- is the single-sample forward at x_l + h e minus that at x_l - h e: its NUDFT term
    P_lf (e^{-i k.theta+} - e^{-i k.theta-}), the contraction with Ghat_{z,f} summed over f, and the
    IDFT crop of each plane.  The inner product with r is taken on the spectrum side against
    Rt_z = B^H r_z conj(B) (B the crop's matrix).  The quadratic terms differ by O(h^3), i.e.
    O(h^2) relative to the difference, and are left out.  Ghat is built one depth at a time.

    residual [Z][N][N]; P_rows [S][F]; xy_rows [S][2] metres; axes [S] in {0, 1} -> [S]
    (L(x + h e) - L(x - h e)) / (2 h).
    """
    M = 2 * N
    r = np.asarray(residual, dtype=np.complex128)
    P_rows = np.asarray(P_rows, dtype=np.complex128)
    xy_rows = np.asarray(xy_rows, dtype=np.float64)
    axes = np.asarray(axes, dtype=int)
    S = len(axes)
    k = index_set(M).astype(np.float64)
    B = _idft_crop_matrix(M, N)
    dE = np.empty((S, M, M), dtype=np.complex128)  # e^{-i k.theta+} - e^{-i k.theta-}, [s][ky][kx]
    for s_ in range(S):
        d = np.zeros(2)
        d[axes[s_]] = h
        tp = relay_theta((xy_rows[s_] + d)[None], center, pitch, M)[0]
        tm = relay_theta((xy_rows[s_] - d)[None], center, pitch, M)[0]
        ep = np.outer(np.exp(-1j * k * tp[1]), np.exp(-1j * k * tp[0]))
        em = np.outer(np.exp(-1j * k * tm[1]), np.exp(-1j * k * tm[0]))
        dE[s_] = ep - em
    acc = np.zeros(S)
    omega = np.asarray(omega, dtype=np.float64)
    for iz, z in enumerate(np.asarray(depths, dtype=np.float64)):
        Gz = np.stack([transfer_function(rsd_kernel(M, pitch, z, w / C)) for w in omega])  # [F][M][M]
        H = np.tensordot(P_rows, Gz, axes=(1, 0))  # [S][M][M]: sum_f P_lf Ghat_{z,f}
        Rt = np.conj(B).T @ r[iz] @ np.conj(B)  # [ky][kx]
        acc += 2.0 * np.real(np.einsum("yx,syx->s", np.conj(Rt), dE * H)) / (M * M)
    return acc / (2.0 * h)


# --------------------------- subsampled acquisition (Methods: Sampling Criteria) ---

def downsampling_bound(dx, dz):
    """Largest lateral downsampling factor of Eq. upsample2: lambda_sx / lambda_sz = 2 |z_r - z_0| / |x_r - x_0|.

    A point source at lateral offset dx and depth offset dz from a relay point may be sampled D times
    more coarsely along the relay than the Nyquist pitch of the depth axis when D is below this ratio.
    """
    return 2.0 * abs(dz) / abs(dx)


def subsample_grid(P, D: int) -> np.ndarray:
    """Keep every D-th relay sample per axis (the compression step): [N][N][F] -> [Nc][Nc][F], Nc = ceil(N / D),
    kept sample (i, j) being grid sample (D i, D j)."""
    return np.asarray(P)[::D, ::D]


def upsample_nearest(Pc, N: int, D: int) -> np.ndarray:
    """Nearest-neighbour interpolation back to the N x N grid (step 2 of the compression algorithm).

    Grid sample n takes the kept sample nearest to it, at D i with i = round(n / D); a sample halfway
    between two kept ones takes the lower, and samples past the last kept one take the last.
    [Nc][Nc][F] -> [N][N][F].
    """
    Pc = np.asarray(Pc)
    nc = Pc.shape[0]
    n = np.arange(N)
    i = np.minimum(np.ceil(n / D - 0.5).astype(int), nc - 1)
    return Pc[i][:, i]


def upsample_linear(Pc, N: int, D: int) -> np.ndarray:
    """Separable linear interpolation back to the N x N grid between the kept samples D i and D (i + 1);
    past the last kept sample the value is held.  [Nc][Nc][F] -> [N][N][F] (complex128)."""
    Pc = np.asarray(Pc, dtype=np.complex128)
    nc = Pc.shape[0]
    n = np.arange(N, dtype=np.float64)
    i0 = np.minimum(np.floor(n / D).astype(int), nc - 1)
    i1 = np.minimum(i0 + 1, nc - 1)
    t = np.where(i1 > i0, n / D - i0, 0.0)
    rows = (1.0 - t)[:, None, None] * Pc[i0] + t[:, None, None] * Pc[i1]  # along y (first axis)
    return (1.0 - t)[None, :, None] * rows[:, i0] + t[None, :, None] * rows[:, i1]


# ------------------------------------------------ plan-level closed forms ---

def frustum_volume(x_in: float, alpha: float, z: float) -> float:
    """V_F = z x_in^2 + z^2 x_in / alpha + z^3 / (3 alpha^2) (Sec. 4.2, Supp. A.2)."""
    return z * x_in ** 2 + z ** 2 * x_in / alpha + z ** 3 / (3.0 * alpha ** 2)


def frustum_extra_volume(alpha: float, z: float) -> float:
    """Delta V = V_F - V_C = (1/alpha + 1/(3 alpha^2)) z^3 with x_in = z (Eq. Vol_Frustum)."""
    return (1.0 / alpha + 1.0 / (3.0 * alpha ** 2)) * z ** 3


def data_compression(N: int, T: int, D: int, F: int) -> float:
    """N^2 T / ((N/D)^2 * 2F): histograms vs subsampled complex phasors (Sec. 7.2, data savings)."""
    return (N * N * T) / ((N / D) ** 2 * 2.0 * F)


def lateral_resolution(lambda_c: float, z: float, D: float) -> float:
    """Delta x = 1.22 lambda_c z / D (Eq. Focusing_Res)."""
    return 1.22 * lambda_c * z / D
