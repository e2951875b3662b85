"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here re-types an oracle formula to compare it with itself: each check
uses brute-force loops, a closed form, a textbook library routine (scipy
convolution, numpy FFT), a physical special case (exact focus of a point
source, on-lattice equality with direct back-projection), an identity
(adjointness, finite differences) or a value printed in the paper.
"""
import cmath
import math
import os

import numpy as np
import pytest
from scipy.signal import convolve2d

import oracle as O
from workloads import (geometry_c1, relay_lattice, relay_uniform, random_phasors, workload_c1)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ------------------------------------------------------------------ a1 -----

def test_frequency_band_matches_workload_statement():
    # 16 bins of a 256-point DFT at 16 ps span 3.906 GHz around f_c = c / 6 cm.
    om, w = O.phasor_frequencies(0.06, 16e-12, 256, 16)
    f = om / (2 * math.pi)
    assert np.allclose(np.diff(f), 1.0 / (256 * 16e-12), rtol=1e-12)
    assert abs(f[-1] - f[0] + (f[1] - f[0]) - 3.90625e9) < 1.0
    fc = 299_792_458.0 / 0.06
    assert abs(0.5 * (f[7] + f[8]) - fc) <= (f[1] - f[0])


def test_frequency_weight_fwhm_is_that_of_sigma_fc_over_5():
    # Sample the filter finely and measure its full width at half maximum; a
    # Gaussian with sigma = f_c / 5 has FWHM = 2 sqrt(2 ln 2) f_c / 5.
    om, w = O.phasor_frequencies(0.06, 1e-12, 2 ** 20, 20000)
    f = om / (2 * math.pi)
    above = f[w >= 0.5]
    fwhm = above[-1] - above[0]
    fc = 299_792_458.0 / 0.06
    assert abs(fwhm - 2 * math.sqrt(2 * math.log(2)) * fc / 5) < 2 * (f[1] - f[0])
    assert abs(f[np.argmax(w)] - fc) <= (f[1] - f[0])


def test_temporal_dft_brute_force_small():
    L, T, F = 3, 7, 4
    h = rng.standard_normal((L, T))
    om = rng.uniform(1e10, 4e10, F)
    wt = rng.uniform(0.2, 1.0, F)
    t0, dt = 1.3e-9, 7e-12
    got = O.temporal_dft(h, t0, dt, om, wt)
    for l in range(L):
        for f in range(F):
            s = 0j
            for n in range(T):
                s += h[l, n] * cmath.exp(-1j * om[f] * (t0 + n * dt))
            assert abs(got[l, f] - wt[f] * s) < 1e-12 * (1 + abs(s))


def test_temporal_dft_of_a_gaussian_pulse_matches_its_fourier_transform():
    # A well-sampled Gaussian pulse centred at tau has DTFT ~ (sqrt(2 pi) s / dt) e^{-w^2 s^2/2} e^{-i w tau}
    # (Poisson summation; aliasing is below 1e-30 for dt << s).  Pins the sign and the time origin.
    dt, T, t0 = 4e-12, 1024, 2.0e-9
    s = 65e-12 / (2 * math.sqrt(2 * math.log(2)))
    tau = t0 + 400.3 * dt
    t = t0 + dt * np.arange(T)
    h = np.exp(-((t - tau) ** 2) / (2 * s * s))[None, :]
    om, w = O.phasor_frequencies(0.06, dt, 8192, 64)
    got = O.temporal_dft(h, t0, dt, om, np.ones_like(om))[0]
    want = math.sqrt(2 * math.pi) * s / dt * np.exp(-(om ** 2) * s * s / 2) * np.exp(-1j * om * tau)
    assert rel(got, want) < 1e-10


# -------------------------------------------------------------- a2-a5 ------

def test_type1_brute_force_tiny():
    L, M, F = 4, 6, 2
    th = rng.uniform(-math.pi, math.pi, (L, 2))
    P = rng.standard_normal((L, F)) + 1j * rng.standard_normal((L, F))
    U = O.nudft_type1(P, th, M)
    for f in range(F):
        for iy, ky in enumerate(range(-M // 2, M // 2)):
            for ix, kx in enumerate(range(-M // 2, M // 2)):
                s = sum(P[l, f] * cmath.exp(-1j * (kx * th[l, 0] + ky * th[l, 1])) for l in range(L))
                assert abs(U[f, iy, ix] - s) < 1e-12


def test_type1_on_lattice_is_the_fft_of_the_gridded_samples():
    M, F = 16, 3
    n = rng.choice(M * M, 40, replace=False)
    ny, nx = n // M - M // 2, n % M - M // 2
    th = 2 * math.pi * np.stack([nx, ny], axis=1) / M
    P = rng.standard_normal((40, F)) + 1j * rng.standard_normal((40, F))
    U = O.nudft_type1(P, th, M)
    for f in range(F):
        grid = np.zeros((M, M), complex)
        grid[ny + M // 2, nx + M // 2] = P[:, f]
        want = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(grid)))
        assert rel(U[f], want) < 1e-13


def test_type2_brute_force_and_adjointness():
    L, M, F = 5, 4, 2
    th = rng.uniform(-math.pi, math.pi, (L, 2))
    U = rng.standard_normal((F, M, M)) + 1j * rng.standard_normal((F, M, M))
    u = O.nudft_type2(U, th)
    for l in range(L):
        for f in range(F):
            s = 0j
            for iy, ky in enumerate(range(-M // 2, M // 2)):
                for ix, kx in enumerate(range(-M // 2, M // 2)):
                    s += U[f, iy, ix] * cmath.exp(1j * (kx * th[l, 0] + ky * th[l, 1]))
            assert abs(u[l, f] - s) < 1e-12
    P = rng.standard_normal((L, F)) + 1j * rng.standard_normal((L, F))
    lhs = np.vdot(O.nudft_type1(P, th, M), U)
    rhs = np.vdot(P, O.nudft_type2(U, th))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_type1_selected_modes_equal_full_sum():
    L, M, F = 30, 8, 3
    th = rng.uniform(-math.pi / 2, math.pi / 2, (L, 2))
    P = rng.standard_normal((L, F)) + 1j * rng.standard_normal((L, F))
    U = O.nudft_type1(P, th, M)
    kxy = np.array([[-4, -4], [3, -1], [0, 0], [-2, 3]])
    got = O.nudft_type1_modes(P, th, kxy)
    want = np.stack([U[:, ky + M // 2, kx + M // 2] for kx, ky in kxy])
    assert rel(got, want) < 1e-13


# -------------------------------------------------------------- a6-a7 ------

def test_transfer_function_brute_force():
    M = 4
    g = O.rsd_kernel(M, 0.1, 0.5, 40.0)
    G = O.transfer_function(g)
    for iy, ky in enumerate(range(-2, 2)):
        for ix, kx in enumerate(range(-2, 2)):
            s = 0j
            for jy_i, jy in enumerate(range(-2, 2)):
                for jx_i, jx in enumerate(range(-2, 2)):
                    s += g[jy_i, jx_i] * cmath.exp(-2j * math.pi * (kx * jx + ky * jy) / M)
            assert abs(G[iy, ix] - s) < 1e-12
    # the kernel itself: e^{ikr}/r at offset (jx, jy) = (1, -2) cells
    r = math.sqrt(0.1 ** 2 + 0.2 ** 2 + 0.25)
    assert abs(g[0, 3] - cmath.exp(40j * r) / r) < 1e-14


def _lattice_case(N=8, pitch=0.02, L=25, F=3, Z=2, seed=5):
    r = np.random.default_rng(seed)
    lat = relay_lattice(N, pitch, (0.1, -0.05), dtype=np.float64)
    xy = lat[r.choice(N * N, L, replace=False)]
    P = r.standard_normal((L, F)) + 1j * r.standard_normal((L, F))
    om = np.array([2 * math.pi * 3e9, 2 * math.pi * 4e9, 2 * math.pi * 5.5e9])[:F]
    depths = np.array([0.3, 0.55])[:Z]
    return dict(P=P, xy=xy, center=(0.1, -0.05), pitch=pitch, N=N, depths=depths, omega=om)


def pin_on_lattice_equals_direct_backprojection(case=None):
    """max relative error of NURSD-1 vs direct back-projection for on-lattice samples."""
    c = case or _lattice_case()
    V = O.nursd_forward(c["P"], c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    m = O.index_set(c["N"]) * c["pitch"]
    X, Y = np.meshgrid(m + c["center"][0], m + c["center"][1], indexing="xy")
    err = 0.0
    for iz, z in enumerate(c["depths"]):
        vox = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
        d = O.fbp_direct(c["P"], c["xy"], c["omega"], vox).reshape(X.shape)
        err = max(err, rel(V[iz], d))
    return err


def test_on_lattice_nursd_equals_direct_backprojection():
    # The paper's NURSD-1 = RSD equivalence on the full uniform grid (Sec. 8.1), and
    # RSD on a lattice is exactly the direct back-projection sum (M = 2N: no wrap).
    assert pin_on_lattice_equals_direct_backprojection() < 1e-12


def test_on_lattice_nursd_equals_scipy_linear_convolution():
    c = _lattice_case(N=6, L=20, F=2, Z=1)
    N, M = c["N"], 2 * c["N"]
    V = O.nursd_forward(c["P"], c["xy"], c["center"], c["pitch"], N, c["depths"], c["omega"])[0]
    idx = np.rint((c["xy"] - np.array(c["center"])) / c["pitch"]).astype(int) + N // 2
    want = np.zeros((N, N), complex)
    for f in range(2):
        grid = np.zeros((N, N), complex)
        grid[idx[:, 1], idx[:, 0]] = c["P"][:, f]
        g = O.rsd_kernel(M, c["pitch"], c["depths"][0], c["omega"][f] / O.C)  # offsets I_M
        full = convolve2d(grid, g, mode="full")
        # full[a] = sum_b grid[b] g[a - b]; array index b <-> n = b - N/2, c <-> j = c - N,
        # so output lattice point m sits at a = m + 3N/2, i.e. the block [N, 2N).
        want += full[N:2 * N, N:2 * N]
    assert rel(V, want) < 1e-12


def test_point_source_focus_closed_form():
    # Analytic phasors of a point source, P = e^{-i k d}/d, focus exactly:
    # V(x_s) = F * sum_l 1/d_l^2 (all phases cancel).
    xy = relay_uniform(300, 0.5, seed=3).astype(np.float64)
    om, _ = O.phasor_frequencies(0.06, 16e-12, 256, 16)
    xs = np.array([0.07, -0.12, 0.8])
    d = np.sqrt((xy[:, 0] - xs[0]) ** 2 + (xy[:, 1] - xs[1]) ** 2 + xs[2] ** 2)
    P = np.exp(-1j * np.outer(d, om / O.C)) / d[:, None]
    v = O.fbp_direct(P, xy, om, xs[None, :])[0]
    assert abs(v - 16 * np.sum(1 / d ** 2)) < 1e-10 * abs(v)


def test_confocal_point_source_focus_closed_form():
    # Confocal acquisition: the relay point illuminates and detects, the round trip gives
    # P = e^{-2 i k d} / d, and the confocal kernel e^{+2 i k r} / r refocuses it exactly on the
    # lattice: V(x_s) = F sum_l 1/d_l^2.  The ordinary kernel leaves e^{-i k d} in every term.
    c = _lattice_case()
    iz, mx, my = 1, 1, -2
    xs = (c["center"][0] + mx * c["pitch"], c["center"][1] + my * c["pitch"], c["depths"][iz])
    d = np.sqrt((c["xy"][:, 0] - xs[0]) ** 2 + (c["xy"][:, 1] - xs[1]) ** 2 + xs[2] ** 2)
    k = np.asarray(c["omega"]) / O.C
    P = np.exp(-2j * np.outer(d, k)) / d[:, None]
    V = O.nursd_forward(P, c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"], confocal=True)
    got = V[iz, my + c["N"] // 2, mx + c["N"] // 2]
    want = len(k) * np.sum(1 / d ** 2)
    assert abs(got - want) < 1e-12 * want
    V1 = O.nursd_forward(P, c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    assert abs(V1[iz, my + c["N"] // 2, mx + c["N"] // 2] - want) > 1e-3 * want


def test_confocal_on_lattice_equals_direct_sum_with_doubled_wavenumber():
    c = _lattice_case()
    V = O.nursd_forward(c["P"], c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"], confocal=True)
    vox = O.voxel_lattice(c["center"], c["pitch"], c["N"], c["depths"]).reshape(-1, 3)
    d = O.fbp_direct(c["P"], c["xy"], 2 * np.asarray(c["omega"]), vox)
    assert rel(V.ravel(), d) < 1e-12


def test_reconstruction_of_simulated_scatterers_focuses_on_them():
    # End to end through the temporal transform: the max-intensity projection of the
    # tiny workload's three on-axis scatterers (0.6/0.9/1.2 m) peaks at the centre of
    # the lateral lattice and within one depth plane of each scatterer.
    wl = workload_c1()
    g = wl.geom
    om, wt = O.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    P = O.temporal_dft(wl.hist, g.t0, g.dt, om, wt)
    V = O.nursd_forward(P, wl.xy, g.center, g.pitch, g.N, g.depths, om)
    I = np.abs(V)
    prof = I[:, g.N // 2 - 1:g.N // 2 + 1, g.N // 2 - 1:g.N // 2 + 1].max(axis=(1, 2))
    dz = g.depths[1] - g.depths[0]
    for zs in (0.6, 0.9, 1.2):
        iz = int(np.argmin(np.abs(g.depths - zs)))
        # the lateral maximum on the plane nearest the scatterer is on-axis (within one voxel)
        my, mx = np.unravel_index(np.argmax(I[iz]), I[iz].shape)
        assert abs(my - g.N // 2) <= 1 and abs(mx - g.N // 2) <= 1, (zs, my, mx)
    # the depth profile has local maxima near each scatterer
    peaks = [iz for iz in range(1, g.Z - 1) if prof[iz] >= prof[iz - 1] and prof[iz] >= prof[iz + 1]]
    for zs in (0.6, 0.9, 1.2):
        assert min(abs(g.depths[p] - zs) for p in peaks) <= 1.5 * dz


def test_lateral_psf_width_is_of_the_diffraction_limit_order():
    # Eq. Focusing_Res: Delta x = 1.22 lambda z / D.  Loose (factor 2) check of the
    # half-maximum width of the reconstructed analytic point source.
    N, pitch = 64, 1.0 / 64
    xy = relay_lattice(N, pitch, dtype=np.float64)
    om, wt = O.phasor_frequencies(0.06, 16e-12, 256, 16)
    zs = 0.8
    d = np.sqrt(xy[:, 0] ** 2 + xy[:, 1] ** 2 + zs ** 2)
    P = np.exp(-1j * np.outer(d, om / O.C)) * wt[None, :]
    m = O.index_set(N) * pitch
    vox = np.stack([m, np.zeros(N), np.full(N, zs)], axis=1)
    prof = np.abs(O.fbp_direct(P, xy, om, vox))
    above = m[prof >= 0.5 * prof.max()]
    fwhm = above[-1] - above[0] + pitch
    dx = O.lateral_resolution(0.06, zs, 1.0)
    assert 0.5 * dx < fwhm < 2.0 * dx


# ------------------------------------------- single illumination, video ---

def _two_way_phasors(xy, xs, xp, omega):
    """Analytic phasors of a point scatterer x_s lit from x_p: e^{-i k (|x_s - x_p| + d_l)} / d_l."""
    d = np.sqrt((xy[:, 0] - xs[0]) ** 2 + (xy[:, 1] - xs[1]) ** 2 + xs[2] ** 2)
    dp = float(np.linalg.norm(np.asarray(xs) - np.asarray(xp)))
    k = np.asarray(omega) / O.C
    return np.exp(-1j * np.outer(d + dp, k)) / d[:, None], d, dp


def test_per_frequency_direct_sum_adds_up_to_direct_backprojection():
    c = _lattice_case()
    vox = np.array([[0.11, -0.02, 0.4], [0.05, -0.09, 0.7]])
    per_f = O.fbp_direct_per_frequency(c["P"], c["xy"], c["omega"], vox)
    assert rel(per_f.sum(axis=1), O.fbp_direct(c["P"], c["xy"], c["omega"], vox)) < 1e-13


def test_illuminated_on_lattice_equals_direct_sum_with_the_mask():
    # On the lattice each frequency's reconstruction is exactly the direct sum, so the
    # illuminated volume is the mask-weighted sum of the per-frequency direct sums.
    c = _lattice_case()
    xp = (0.12, 0.0, 0.0)
    V = O.nursd_forward_illuminated(c["P"], c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"], xp)
    vox = O.voxel_lattice(c["center"], c["pitch"], c["N"], c["depths"]).reshape(-1, 3)
    R = O.fbp_direct_per_frequency(c["P"], c["xy"], c["omega"], vox)  # [V][F]
    A = O.illumination_mask(xp, vox, c["omega"])  # [F][V]
    assert rel(V.ravel(), np.einsum("fv,vf->v", A, R)) < 1e-12


def test_illuminated_point_scatterer_focuses_in_closed_form():
    # Two-way phasors e^{-i k (|x_s - x_p| + d_l)} / d_l: at x_s both the detection kernel and
    # the illumination mask cancel their phases, so V(x_s) = F sum_l 1 / d_l^2 exactly; a
    # wrong mask sign leaves e^{-2 i k |x_s - x_p|} in every term.
    c = _lattice_case()
    xp = (0.12, 0.0, 0.0)
    iz, mx, my = 1, 2, -1
    xs = (c["center"][0] + mx * c["pitch"], c["center"][1] + my * c["pitch"], c["depths"][iz])
    P, d, _ = _two_way_phasors(c["xy"], xs, xp, c["omega"])
    V = O.nursd_forward_illuminated(P, c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"], xp)
    want = len(c["omega"]) * np.sum(1 / d ** 2)
    got = V[iz, my + c["N"] // 2, mx + c["N"] // 2]
    assert abs(got - want) < 1e-12 * want


def test_transient_frame_at_time_zero_is_the_collapsed_forward():
    c = _lattice_case()
    Vt = O.nursd_transient_frames(c["P"], c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"],
                                  [0.0])
    V = O.nursd_forward(c["P"], c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    assert rel(Vt[0], V) < 1e-12


def test_transient_frames_of_a_point_scatterer_in_closed_form():
    # Without the illumination mask the frame at time t keeps e^{i w (t - tau_p)}, tau_p the
    # illumination delay: frame(x_s, t) = sum_f e^{i w_f (t - tau_p)} * sum_l 1 / d_l^2, which
    # peaks (F sum 1/d^2) when the virtual wave reaches x_s, t = tau_p.
    c = _lattice_case()
    xp = (0.12, 0.0, 0.0)
    iz, mx, my = 0, -3, 2
    xs = (c["center"][0] + mx * c["pitch"], c["center"][1] + my * c["pitch"], c["depths"][iz])
    P, d, dp = _two_way_phasors(c["xy"], xs, xp, c["omega"])
    tau = dp / O.C
    times = [tau, tau + 37e-12, tau - 120e-12]
    Vt = O.nursd_transient_frames(P, c["xy"], c["center"], c["pitch"], c["N"], c["depths"], c["omega"], times)
    s = np.sum(1 / d ** 2)
    for i, t in enumerate(times):
        want = s * sum(cmath.exp(1j * w * (t - tau)) for w in c["omega"])
        assert abs(Vt[i, iz, my + c["N"] // 2, mx + c["N"] // 2] - want) < 1e-12 * s * len(c["omega"])


# ------------------------------------------------------------------ a8 -----

def test_type2_output_at_lattice_voxels_equals_lattice_crop():
    c = _lattice_case()
    N, M = c["N"], 2 * c["N"]
    U = O.nudft_type1(c["P"], O.relay_theta(c["xy"], c["center"], c["pitch"], M), M)
    Gh = O.transfer_functions(c["depths"], c["omega"], M, c["pitch"])
    V = O.propagate(U, Gh, N)
    lat = relay_lattice(N, c["pitch"], c["center"], dtype=np.float64)
    th = O.relay_theta(lat, c["center"], c["pitch"], M)
    Vp = O.propagate_points(U, Gh, np.broadcast_to(th, (len(c["depths"]),) + th.shape))
    assert rel(Vp, V.reshape(len(c["depths"]), -1)) < 1e-12


# ------------------------------------------------------------------ a9 -----

def test_idft_grid_recovers_on_lattice_samples():
    c = _lattice_case(N=6, L=12, F=2)
    N, M = c["N"], 2 * c["N"]
    U = O.nudft_type1(c["P"], O.relay_theta(c["xy"], c["center"], c["pitch"], M), M)
    u = O.idft_grid(U)
    idx = np.rint((c["xy"] - np.array(c["center"])) / c["pitch"]).astype(int) + M // 2
    want = np.zeros((2, M, M), complex)
    for f in range(2):
        want[f, idx[:, 1], idx[:, 0]] = c["P"][:, f]
    assert rel(u, want) < 1e-12


def _bluestein(x, s):
    """Independent chirp-z evaluation of sum_n x[n] e^{-2 pi i kappa n/(M s)} (n, kappa in I_M)."""
    M = len(x)
    n = np.arange(-M // 2, M // 2)
    a = 1.0 / (M * s)
    chirp = np.exp(-1j * math.pi * a * n ** 2)
    d = np.arange(-(M - 1), M)
    b = np.exp(1j * math.pi * a * d ** 2)
    Lc = 1 << int(math.ceil(math.log2(3 * M)))
    conv = np.fft.ifft(np.fft.fft(x * chirp, Lc) * np.fft.fft(b, Lc))
    # out[kappa] = chirp(kappa) * sum_n (x chirp)[n] b[kappa - n]; index of (kappa - n) in b is kappa - n + M - 1
    return chirp * conv[np.arange(M) + M - 1]


def test_scaled_dft_matches_independent_chirp_z_and_reduces_to_dft():
    M = 16
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    for s in (1.0, 1.37, 2.5, 4.096):
        A = O.scaled_dft_matrix(M, s)
        assert rel(A @ x, _bluestein(x, s)) < 1e-12
    A1 = O.scaled_dft_matrix(M, 1.0)
    assert rel(A1 @ x, np.fft.fftshift(np.fft.fft(np.fft.ifftshift(x)))) < 1e-13


def test_srsd_with_unit_scale_equals_nursd():
    c = _lattice_case()
    N, M = c["N"], 2 * c["N"]
    xy = c["xy"] + np.random.default_rng(9).uniform(-0.4, 0.4, c["xy"].shape) * c["pitch"]
    V1 = O.nursd_forward(c["P"], xy, c["center"], c["pitch"], N, c["depths"], c["omega"])
    Vs = O.srsd_forward(c["P"], xy, c["center"], c["pitch"], N, c["depths"], np.ones(len(c["depths"])), c["omega"])
    assert rel(Vs, V1) < 1e-12


def test_srsd_with_input_on_the_scaled_lattice_equals_direct_sum():
    # If the gridded input is non-zero only at n that are multiples of s, the
    # trigonometric interpolant of G on the scaled lattice is sampled at lattice
    # points, so SRSD equals the direct sum  sum_n u[n] G(m s delta - n delta).
    N, M, pitch, s, z = 8, 16, 0.02, 2.0, 0.4
    om = np.array([2 * math.pi * 4e9, 2 * math.pi * 5e9])
    r = np.random.default_rng(11)
    u = np.zeros((2, M, M), complex)
    pts = [(-4, 2), (0, 0), (2, -2), (-2, -4)]
    for f in range(2):
        for nx, ny in pts:
            u[f, ny + M // 2, nx + M // 2] = r.standard_normal() + 1j * r.standard_normal()
    V = O.srsd_from_grid(u, [z], [s], om, pitch, N)[0]
    m = O.index_set(N)
    want = np.zeros((N, N), complex)
    for f in range(2):
        k = om[f] / O.C
        for nx, ny in pts:
            dx = (m[None, :] * s - nx) * pitch
            dy = (m[:, None] * s - ny) * pitch
            rr = np.sqrt(dx ** 2 + dy ** 2 + z * z)
            want += u[f, ny + M // 2, nx + M // 2] * np.exp(1j * k * rr) / rr
    assert rel(V, want) < 1e-12


def test_srsd_points_on_each_scaled_lattice_equal_the_srsd_volume():
    # Eq. NURSD2_SRSD at voxels c + s_z delta m of plane z's own lattice is the SRSD output there.
    c = _lattice_case()
    N = c["N"]
    xy = c["xy"] + np.random.default_rng(12).uniform(-0.4, 0.4, c["xy"].shape) * c["pitch"]
    scales = np.array([1.3, 2.25])
    V = O.srsd_forward(c["P"], xy, c["center"], c["pitch"], N, c["depths"], scales, c["omega"])
    r = np.random.default_rng(13)
    m = r.integers(-N // 2, N // 2, size=(len(scales), 11, 2))
    vox = np.asarray(c["center"])[None, None, :] + m * (scales[:, None, None] * c["pitch"])
    got = O.srsd_points(c["P"], xy, c["center"], c["pitch"], N, c["depths"], scales, c["omega"], vox)
    want = np.stack([V[z, m[z, :, 1] + N // 2, m[z, :, 0] + N // 2] for z in range(len(scales))])
    assert rel(got, want) < 1e-12


def test_srsd_points_with_unit_scale_are_the_nursd2_output():
    # s = 1 everywhere: the scaled lattice is the ordinary one and the off-lattice voxels give the
    # NURSD-2 output (Eqs. NURSD2-3).
    c = _lattice_case()
    N, M = c["N"], 2 * c["N"]
    xy = c["xy"] + np.random.default_rng(14).uniform(-0.4, 0.4, c["xy"].shape) * c["pitch"]
    r = np.random.default_rng(15)
    vox = np.asarray(c["center"]) + r.uniform(-0.5, 0.5, size=(len(c["depths"]), 9, 2)) * N * c["pitch"]
    got = O.srsd_points(c["P"], xy, c["center"], c["pitch"], N, c["depths"], np.ones(len(c["depths"])),
                        c["omega"], vox)
    U = O.nudft_type1(c["P"], O.relay_theta(xy, c["center"], c["pitch"], M), M)
    theta = np.stack([O.relay_theta(vox[z], c["center"], c["pitch"], M) for z in range(len(c["depths"]))])
    want = O.propagate_points(U, O.transfer_functions(c["depths"], c["omega"], M, c["pitch"]), theta)
    assert rel(got, want) < 1e-12


# -------------------------------------------------------------- a10-a11 ----

def test_adjoint_identity():
    c = _lattice_case()
    xy = c["xy"] + np.random.default_rng(2).uniform(-0.5, 0.5, c["xy"].shape) * c["pitch"]
    P = c["P"]
    r = np.random.default_rng(3)
    V = r.standard_normal((2, c["N"], c["N"])) + 1j * r.standard_normal((2, c["N"], c["N"]))
    AP = O.nursd_forward(P, xy, c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    AhV = O.nursd_adjoint(V, xy, c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    lhs, rhs = np.vdot(V, AP), np.vdot(AhV, P)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gradients_match_central_differences():
    c = _lattice_case(N=6, L=10, F=2, Z=2)
    r = np.random.default_rng(4)
    xy = c["xy"] + r.uniform(-0.5, 0.5, c["xy"].shape) * c["pitch"]
    args = (c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    Vt = r.standard_normal((2, 6, 6)) + 1j * r.standard_normal((2, 6, 6))
    gP, gx = O.nursd_gradients(c["P"], xy, *args, Vt)
    h = 1e-6
    for (l, f) in [(0, 0), (3, 1), (9, 0)]:
        for part, unit in (("re", 1.0), ("im", 1j)):
            Pp = c["P"].copy(); Pp[l, f] += h * unit
            Pm = c["P"].copy(); Pm[l, f] -= h * unit
            fd = (O.nursd_loss(Pp, xy, *args, Vt) - O.nursd_loss(Pm, xy, *args, Vt)) / (2 * h)
            an = gP[l, f].real if part == "re" else gP[l, f].imag
            assert abs(fd - an) < 1e-6 * (1 + abs(an)), (l, f, part, fd, an)
    hx = 1e-7
    for l in (1, 5, 8):
        for a in (0, 1):
            xp = xy.copy(); xp[l, a] += hx
            xm = xy.copy(); xm[l, a] -= hx
            fd = (O.nursd_loss(c["P"], xp, *args, Vt) - O.nursd_loss(c["P"], xm, *args, Vt)) / (2 * hx)
            assert abs(fd - gx[l, a]) < 1e-5 * (1 + abs(gx[l, a])), (l, a, fd, gx[l, a])


# ------------------------------------------------------- printed values ----

def test_frustum_worked_example_from_the_paper():
    g = _golden("frustum_example.txt")
    a, z = g["alpha"], g["z"]
    VF = O.frustum_volume(z, a, z)
    VC = z ** 3
    dV = O.frustum_extra_volume(a, z)
    assert abs(VC - g["V_C"]) < 0.5
    assert abs(VF - g["V_F"]) < 0.5
    assert abs(dV - g["dV"]) < 0.5
    assert abs(100 * dV / VC - g["percent"]) < 0.5
    assert abs((VF - VC) - dV) < 1e-9


def test_data_savings_example_from_the_paper():
    g = _golden("data_savings.txt")
    T = 1000
    F = int(T / g["T_over_F"])
    assert abs(O.data_compression(250, T, int(g["D"]), F) - g["compression"]) < 1e-9


# ----------------------------------------------- the pins catch mistakes ----

def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible oracle mistake, planted on the CPU, breaks a pin."""
    base = pin_on_lattice_equals_direct_backprojection()
    assert base < 1e-12
    orig_kernel, orig_prop, orig_theta = O.rsd_kernel, O.propagate, O.relay_theta
    import oracle.nursd_oracle as mod

    def flipped_kernel(M, pitch, z, k):  # wrong sign of the propagation phase
        return orig_kernel(M, pitch, z, -k)

    def no_norm(U, G, N):  # dropped M^-2
        return orig_prop(U, G, N) * (U.shape[-1] ** 2)

    def swapped_theta(xy, center, pitch, M):  # transposed operand (x <-> y)
        return orig_theta(xy, center, pitch, M)[:, ::-1]

    for name, bad in (("rsd_kernel", flipped_kernel), ("propagate", no_norm), ("relay_theta", swapped_theta)):
        monkeypatch.setattr(mod, name, bad)
        assert pin_on_lattice_equals_direct_backprojection() > 1e-3, name
        monkeypatch.setattr(mod, name, {"rsd_kernel": orig_kernel, "propagate": orig_prop,
                                        "relay_theta": orig_theta}[name])
    assert pin_on_lattice_equals_direct_backprojection() < 1e-12


def test_depthwise_adjoint_spectrum_and_gradients_from_w_agree_with_the_full_forms():
    c = _lattice_case(N=6, L=10, F=2, Z=2)
    r = np.random.default_rng(8)
    xy = c["xy"] + r.uniform(-0.5, 0.5, c["xy"].shape) * c["pitch"]
    M = 2 * c["N"]
    Gh = O.transfer_functions(c["depths"], c["omega"], M, c["pitch"])
    V = r.standard_normal((2, 6, 6)) + 1j * r.standard_normal((2, 6, 6))
    R = O.adjoint_spectrum(V, Gh)
    assert rel(O.adjoint_spectrum_depthwise(V, c["depths"], c["omega"], c["pitch"]), R) < 1e-13
    # with w = 2 (A P - V_t), gradients_from_w reproduces nursd_gradients
    Vt = r.standard_normal((2, 6, 6)) + 1j * r.standard_normal((2, 6, 6))
    args = (c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    gP, gx = O.nursd_gradients(c["P"], xy, *args, Vt)
    w = 2 * (O.nursd_forward(c["P"], xy, *args) - Vt)
    th = O.relay_theta(xy, c["center"], c["pitch"], M)
    gP2, gx2 = O.gradients_from_w(O.adjoint_spectrum(w, Gh), c["P"], th, c["pitch"])
    assert rel(gP2, gP) < 1e-12 and rel(gx2, gx) < 1e-12


def test_lattice_type1_equals_the_general_sum():
    M, L, F = 12, 30, 2
    r = np.random.default_rng(9)
    n = np.stack([r.integers(-M // 2, M // 2, L), r.integers(-M // 2, M // 2, L)], axis=1)
    P = r.standard_normal((L, F)) + 1j * r.standard_normal((L, F))
    assert rel(O.nudft_type1_lattice(P, n, M), O.nudft_type1(P, 2 * math.pi * n / M, M)) < 1e-13


# ------------------------------------------- the depth-streamed propagation ----

def pin_depth_streamed_equals_direct_backprojection(prop=None, case=None):
    """max relative error of a depth-streamed propagation (default O.propagate_depth) of the exact
    type-1 spectrum of on-lattice samples against direct back-projection at that depth's lattice."""
    prop = prop or O.propagate_depth
    c = case or _lattice_case(N=8, L=30, F=3, Z=2, seed=11)
    M = 2 * c["N"]
    U = O.nudft_type1(c["P"], O.relay_theta(c["xy"], c["center"], c["pitch"], M), M)
    m = O.index_set(c["N"]) * c["pitch"]
    X, Y = np.meshgrid(m + c["center"][0], m + c["center"][1], indexing="xy")
    err = 0.0
    for z in c["depths"]:
        vox = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
        d = O.fbp_direct(c["P"], c["xy"], c["omega"], vox).reshape(X.shape)
        err = max(err, rel(prop(U, z, c["omega"], c["pitch"], c["N"]), d))
    return err


def test_propagate_depth_equals_direct_backprojection_on_the_lattice():
    # the same physical special case that pins the full operator: samples on the lattice,
    # M = 2N (no wrap), so each plane is exactly the direct back-projection sum at that depth
    assert pin_depth_streamed_equals_direct_backprojection() < 1e-12


def test_propagate_depth_equals_each_plane_of_propagate():
    c = _lattice_case(N=6, L=12, F=3, Z=2, seed=12)
    r = np.random.default_rng(13)
    xy = c["xy"] + r.uniform(-0.5, 0.5, c["xy"].shape) * c["pitch"]
    M = 2 * c["N"]
    U = O.nudft_type1(c["P"], O.relay_theta(xy, c["center"], c["pitch"], M), M)
    V = O.propagate(U, O.transfer_functions(c["depths"], c["omega"], M, c["pitch"]), c["N"])
    for iz, z in enumerate(c["depths"]):
        assert rel(O.propagate_depth(U, z, c["omega"], c["pitch"], c["N"]), V[iz]) < 1e-13


def test_planted_mistakes_in_the_depth_streamed_propagation_are_caught():
    def no_norm(U, z, omega, pitch, N):  # dropped M^-2
        return O.propagate_depth(U, z, omega, pitch, N) * U.shape[-1] ** 2

    def wrong_pitch(U, z, omega, pitch, N):  # transfer function sampled at the wrong pitch
        return O.propagate_depth(U, z, omega, 1.01 * pitch, N)

    def wrong_depth(U, z, omega, pitch, N):  # another plane's kernel
        return O.propagate_depth(U, 1.05 * z, omega, pitch, N)

    for bad in (no_norm, wrong_pitch, wrong_depth):
        assert pin_depth_streamed_equals_direct_backprojection(bad) > 1e-3, bad.__name__


def test_single_sample_loss_differences_equal_brute_force_central_differences():
    # the full-size gradient check differences one sample's forward term at a time; on a small case
    # that must reproduce the central difference of the whole loss (up to the O(h^2) terms it drops)
    c = _lattice_case(N=6, L=10, F=2, Z=2)
    r = np.random.default_rng(14)
    xy = c["xy"] + r.uniform(-0.5, 0.5, c["xy"].shape) * c["pitch"]
    args = (c["center"], c["pitch"], c["N"], c["depths"], c["omega"])
    Vt = r.standard_normal((2, 6, 6)) + 1j * r.standard_normal((2, 6, 6))
    resid = O.nursd_forward(c["P"], xy, *args) - Vt
    rows, axes, h = np.array([0, 3, 3, 9]), np.array([0, 0, 1, 1]), 1e-5
    got = O.position_loss_differences(resid, c["P"][rows], xy[rows], axes, h, *args)
    want = []
    for l, a in zip(rows, axes):
        xp = xy.copy(); xp[l, a] += h
        xm = xy.copy(); xm[l, a] -= h
        want.append((O.nursd_loss(c["P"], xp, *args, Vt) - O.nursd_loss(c["P"], xm, *args, Vt)) / (2 * h))
    want = np.array(want)
    assert np.max(np.abs(got - want)) < 1e-6 * np.max(np.abs(want)), (got, want)
    # and the analytic gradient, which the differences must approach as h -> 0
    _, gx = O.nursd_gradients(c["P"], xy, *args, Vt)
    assert np.max(np.abs(got - gx[rows, axes])) < 1e-5 * np.max(np.abs(want))


# ------------------------------- subsampled acquisition (Methods: Sampling Criteria) ----

def test_nearest_upsampling_by_brute_force():
    r = np.random.default_rng(21)
    for N, D in ((7, 2), (9, 3), (10, 4), (5, 1)):
        P = r.standard_normal((N, N, 2)) + 1j * r.standard_normal((N, N, 2))
        Pc = O.subsample_grid(P, D)
        got = O.upsample_nearest(Pc, N, D)
        kept = np.arange(0, N, D)
        for y in range(N):
            for x in range(N):
                iy = int(np.argmin(np.abs(kept - y)))  # first minimum: the lower of two equidistant samples
                ix = int(np.argmin(np.abs(kept - x)))
                assert np.array_equal(got[y, x], P[kept[iy], kept[ix]])


def test_linear_upsampling_equals_scipy_and_holds_past_the_last_sample():
    from scipy.interpolate import RegularGridInterpolator

    r = np.random.default_rng(22)
    N, D = 13, 4  # kept samples 0, 4, 8, 12: the grid ends on a kept sample
    P = r.standard_normal((N, N, 3)) + 1j * r.standard_normal((N, N, 3))
    Pc = O.subsample_grid(P, D)
    got = O.upsample_linear(Pc, N, D)
    kept = np.arange(0, N, D).astype(float)
    yy, xx = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    pts = np.stack([yy.ravel(), xx.ravel()], axis=1)
    for f in range(3):
        want = (RegularGridInterpolator((kept, kept), Pc[..., f].real)(pts)
                + 1j * RegularGridInterpolator((kept, kept), Pc[..., f].imag)(pts)).reshape(N, N)
        assert np.max(np.abs(got[..., f] - want)) < 1e-13
    # N = 11, D = 4: samples 9 and 10 lie past the last kept sample (8) and hold its value
    P2 = P[:11, :11]
    got2 = O.upsample_linear(O.subsample_grid(P2, 4), 11, 4)
    assert np.array_equal(got2[9:, 9:], np.broadcast_to(P2[8, 8], got2[9:, 9:].shape))
    # affine data is reproduced exactly wherever it is interpolated, and D = 1 is the identity
    lin = (2.0 + 0.5 * yy - 1.5j * xx)[..., None]
    assert np.max(np.abs(O.upsample_linear(O.subsample_grid(lin, D), N, D) - lin)) < 1e-12
    assert np.array_equal(O.upsample_linear(P, N, 1), P) and np.array_equal(O.upsample_nearest(P, N, 1), P)


def test_subsampled_point_source_still_focuses_within_the_bound_of_eq_upsample2():
    # analytic phasors P = e^{-i k d} / d of a point source 1.2 m from a 32 x 32 relay lattice at
    # 1.5 cm pitch (half-width 0.24 m): Eq. upsample2 allows D < 2 * 1.2 / 0.24 = 10 over the whole
    # aperture.  Keeping every 2nd or 4th sample, nearest-neighbour or linear re-gridding, the
    # reconstruction still peaks within one voxel of the source and keeps most of its focus.
    N, pitch, z0 = 32, 0.015, 1.2
    assert O.downsampling_bound(N * pitch / 2, z0) > 9.9
    lat = relay_lattice(N, pitch, (0.0, 0.0), dtype=np.float64)
    om = 2 * math.pi * np.array([4.6e9, 5.0e9, 5.4e9])
    xs = np.array([0.0, 0.0, z0])
    d = np.sqrt(np.sum((lat - xs[None, :2]) ** 2, axis=1) + z0 * z0)
    P = np.exp(-1j * np.outer(d, om) / O.C) / d[:, None]  # [L][F], lattice order: row y, column x
    grid = P.reshape(N, N, -1)
    depths = np.array([1.0, 1.2, 1.4])
    full = np.abs(O.nursd_forward(P, lat, (0.0, 0.0), pitch, N, depths, om))
    peak = full.max()
    for D in (2, 4):
        for up in (O.upsample_nearest, O.upsample_linear):
            Pg = up(O.subsample_grid(grid, D), N, D).reshape(N * N, -1)
            V = np.abs(O.nursd_forward(Pg, lat, (0.0, 0.0), pitch, N, depths, om))
            iz, iy, ix = np.unravel_index(np.argmax(V), V.shape)
            # nearest-neighbour re-gridding displaces the field by up to half a kept interval, so the
            # peak may move by one voxel; it stays at the source's depth
            assert iz == 1 and abs(iy - N // 2) <= 1 and abs(ix - N // 2) <= 1, (D, up.__name__, (iz, iy, ix))
            assert V.max() > 0.5 * peak, (D, up.__name__, V.max() / peak)


# ------------------------------------------ NU-SFFT (SRSD on non-uniform acquisition) ----

def test_nu_sfft_brute_force_tiny():
    r = np.random.default_rng(31)
    N, L, F, pitch, center = 4, 3, 2, 0.05, (0.01, -0.02)
    M = 2 * N
    xy = center + r.uniform(-0.09, 0.09, (L, 2))
    P = r.standard_normal((L, F)) + 1j * r.standard_normal((L, F))
    depths, scales, om = np.array([0.4, 0.7]), np.array([1.3, 2.2]), 2 * math.pi * np.array([4e9, 5e9])
    Y = O.nu_sfft_spectra(P, xy, center, pitch, N, depths, scales, om)
    for iz in range(2):
        s = scales[iz]
        for iy, ky in enumerate(range(-M // 2, M // 2)):
            for ix, kx in enumerate(range(-M // 2, M // 2)):
                acc = 0j
                for f in range(F):
                    ph = sum(P[l, f] * cmath.exp(-1j * (kx * 2 * math.pi * (xy[l, 0] - center[0]) / (M * pitch)
                                                         + ky * 2 * math.pi * (xy[l, 1] - center[1]) / (M * pitch)) / s)
                             for l in range(L))
                    g = O.transfer_function(O.rsd_kernel(M, s * pitch, depths[iz], om[f] / O.C))[iy, ix]
                    acc += ph * g
                assert abs(Y[iz, iy, ix] - acc) < 1e-12 * (1 + abs(acc))


def test_nu_sfft_on_the_lattice_equals_srsd_and_at_unit_scale_equals_nursd():
    c = _lattice_case(N=8, L=30, F=3, Z=2, seed=32)
    args = (c["center"], c["pitch"], c["N"], c["depths"])
    scales = np.array([1.4, 2.9])
    # samples on the input lattice: the gridded input of SRSD is exactly the samples
    got = O.nu_sfft_forward(c["P"], c["xy"], *args, scales, c["omega"])
    assert rel(got, O.srsd_forward(c["P"], c["xy"], *args, scales, c["omega"])) < 1e-12
    # off the lattice at unit scale: the scaled DFT at integer modes is NURSD-1's type-1 sum
    xy = c["xy"] + np.random.default_rng(33).uniform(-0.5, 0.5, c["xy"].shape) * c["pitch"]
    got1 = O.nu_sfft_forward(c["P"], xy, *args, np.ones(2), c["omega"])
    assert rel(got1, O.nursd_forward(c["P"], xy, *args, c["omega"])) < 1e-12
    # and off the lattice at s > 1 it differs from SRSD's gridded input (the reason to fuse)
    assert rel(O.nu_sfft_forward(c["P"], xy, *args, scales, c["omega"]),
               O.srsd_forward(c["P"], xy, *args, scales, c["omega"])) > 1e-3


# ---------------------------------------------------- 3D NURSD (non-planar relays) ----

def _relay3d_case(on_grid, seed=41):
    r = np.random.default_rng(seed)
    N, pitch, dz, Mz, z0 = 6, 0.02, 0.015, 8, 0.1
    L, F = 14, 2
    if on_grid:
        n = r.integers(-N // 2, N // 2, (L, 2))
        nz = r.integers(-Mz // 4, Mz // 4, L)
        xyz = np.column_stack([n * pitch, z0 + nz * dz])
    else:
        xyz = np.column_stack([r.uniform(-0.055, 0.055, (L, 2)), z0 + r.uniform(-0.028, 0.028, L)])
    P = r.standard_normal((L, F)) + 1j * r.standard_normal((L, F))
    om = 2 * math.pi * np.array([4e9, 5.5e9])
    return P, xyz, (0.0, 0.0), pitch, N, z0, dz, Mz, om


def test_3d_stage1_on_the_3d_grid_is_the_direct_sum_to_the_plane():
    # samples on the lattice and on the z grid: the trigonometric interpolation is exact there, so the
    # plane z0 holds sum_l P_l G(m delta - x_l, z0 - z_l) (G = 0 at the zero offset)
    P, xyz, c, pitch, N, z0, dz, Mz, om = _relay3d_case(True)
    W = O.nursd3d_plane(P, xyz, c, pitch, N, z0, dz, Mz, om)
    m = O.index_set(N) * pitch
    for f, w in enumerate(om):
        k = w / O.C
        want = np.zeros((N, N), complex)
        for l in range(len(P)):
            r = np.sqrt((m[None, :] - xyz[l, 0]) ** 2 + (m[:, None] - xyz[l, 1]) ** 2 + (z0 - xyz[l, 2]) ** 2)
            with np.errstate(divide="ignore", invalid="ignore"):
                g = np.where(r > 0, np.exp(1j * k * r) / r, 0.0)
            want += P[l, f] * g
        assert rel(W[f], want) < 1e-12


def test_3d_stage1_brute_force_tiny():
    r = np.random.default_rng(42)
    N, pitch, dz, Mz, z0 = 2, 0.03, 0.02, 4, 0.0
    M = 2 * N
    xyz = np.array([[0.004, -0.011, 0.013], [-0.017, 0.009, -0.006]])
    P = (r.standard_normal((2, 1)) + 1j * r.standard_normal((2, 1)))
    om = np.array([2 * math.pi * 5e9])
    W = O.nursd3d_plane(P, xyz, (0.0, 0.0), pitch, N, z0, dz, Mz, om)[0]
    k = om[0] / O.C
    idx = list(range(-M // 2, M // 2))
    idz = list(range(-Mz // 2, Mz // 2))

    def g(jx, jy, jz):
        rr = math.sqrt((jx * pitch) ** 2 + (jy * pitch) ** 2 + (jz * dz) ** 2)
        return cmath.exp(1j * k * rr) / rr if rr > 0 else 0.0

    for iy, my in enumerate(range(-N // 2, N // 2)):
        for ix, mx in enumerate(range(-N // 2, N // 2)):
            acc = 0j
            for kz in idz:
                for ky in idx:
                    for kx in idx:
                        U = sum(P[l, 0] * cmath.exp(-1j * (kx * 2 * math.pi * xyz[l, 0] / (M * pitch)
                                                            + ky * 2 * math.pi * xyz[l, 1] / (M * pitch)
                                                            + kz * 2 * math.pi * (xyz[l, 2] - z0) / (Mz * dz)))
                                for l in range(2))
                        G = sum(g(jx, jy, jz) * cmath.exp(-2j * math.pi * (kx * jx / M + ky * jy / M + kz * jz / Mz))
                                for jz in idz for jy in idx for jx in idx)
                        acc += U * G * cmath.exp(2j * math.pi * (kx * mx + ky * my) / M)
            assert abs(W[iy, ix] - acc / (M * M * Mz)) < 1e-11 * (1 + abs(acc) / (M * M * Mz))


def test_3d_nursd_stage2_is_the_direct_back_projection_of_the_plane():
    P, xyz, c, pitch, N, z0, dz, Mz, om = _relay3d_case(False)
    depths = np.array([0.5, 0.8])
    V = O.nursd3d_forward(P, xyz, c, pitch, N, z0, dz, Mz, depths, om)
    W = O.nursd3d_plane(P, xyz, c, pitch, N, z0, dz, Mz, om)
    lat = O.voxel_lattice(c, pitch, N, [0.0])[0, :, :, :2].reshape(-1, 2)
    for iz, z in enumerate(depths):
        vox = np.column_stack([lat, np.full(len(lat), z - z0)])
        d = O.fbp_direct(W.reshape(len(om), -1).T, lat, om, vox).reshape(N, N)
        assert rel(V[iz], d) < 1e-12
