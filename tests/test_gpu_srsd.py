"""GPU parity of the scaled RSD (a9) against the FP64 oracle (explicit scaled-DFT
matrices, no chirp-z, no FFT of the data), through the C ABI.  Gate: 1e-4
relative L2 on the complex output."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import BASE_SEED, random_phasors, relay_lattice, srsd_depths_c3b, srsd_pitches_c3b

pytestmark = pytest.mark.gpu
TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    nursd.build()


def case(N, L, F, Z, seed, pitch=0.02, center=(0.01, -0.03), smax=4.1):
    r = np.random.default_rng(seed)
    half = N * pitch / 2
    xy = (r.uniform(-half, half, (L, 2)) * 0.999 + np.asarray(center)).astype(np.float32)
    P = random_phasors(L, F, seed=seed + 1)
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    depths = np.linspace(0.3, 0.9, Z)
    scales = np.linspace(1.0, smax, Z)
    return xy, P, om, depths, scales * pitch, pitch, center


@pytest.mark.parametrize("N,L,F,Z,seed", [(16, 300, 6, 5, 1), (32, 1200, 16, 7, 2), (8, 20, 2, 2, 3)])
def test_srsd_matches_oracle(N, L, F, Z, seed):
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, seed)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(xy).cuda())
    V = plan.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    ref = O.srsd_forward(P, xy, center, pitch, N, depths, out_pitch / pitch, om)
    assert rel(V, ref) < TOL


def test_srsd_pitch_given_at_the_call():
    # the interface statement's form srsd_forward(plan, pitch_per_depth, in, out): on a plan created
    # without SRSD tables, then with other pitches (scales below and above 1), then the first ones again
    N, L, F, Z = 32, 1200, 16, 6
    xy, P, om, depths, pitch_a, pitch, center = case(N, L, F, Z, 31)
    pitch_b = np.linspace(0.7, 2.5, Z) * pitch
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L)
    plan.set_points(torch.from_numpy(xy).cuda())
    Pg = torch.from_numpy(P).cuda()
    Va = plan.srsd_forward(Pg, pitch=pitch_a).cpu().numpy()
    assert rel(Va, O.srsd_forward(P, xy, center, pitch, N, depths, pitch_a / pitch, om)) < TOL
    Vb = plan.srsd_forward(Pg, pitch=pitch_b).cpu().numpy()
    assert rel(Vb, O.srsd_forward(P, xy, center, pitch, N, depths, pitch_b / pitch, om)) < TOL
    assert np.array_equal(plan.srsd_forward(Pg, pitch=pitch_a).cpu().numpy(), Va)
    assert np.array_equal(plan.srsd_forward(Pg).cpu().numpy(), Va)  # the last pitches stay in the plan
    with pytest.raises(nursd.NursdError):
        plan.srsd_forward(Pg, pitch=np.full(Z, -1.0))
    assert plan.sync_status() == 0


def test_srsd_with_unit_scale_equals_nursd_on_gpu():
    xy, P, om, depths, _, pitch, center = case(32, 900, 8, 4, 5)
    plan = nursd.Plan(32, pitch, center, depths, om, max_points=900, srsd_pitch=np.full(4, pitch))
    plan.set_points(torch.from_numpy(xy).cuda())
    Pg = torch.from_numpy(P).cuda()
    assert rel(plan.srsd_forward(Pg).cpu().numpy(), plan.forward_phasor(Pg).cpu().numpy()) < 1e-5


def test_srsd_magnitude_output():
    xy, P, om, depths, out_pitch, pitch, center = case(16, 200, 4, 3, 6)
    pc = nursd.Plan(16, pitch, center, depths, om, max_points=200, srsd_pitch=out_pitch)
    pm = nursd.Plan(16, pitch, center, depths, om, max_points=200, srsd_pitch=out_pitch, magnitude=True)
    for p in (pc, pm):
        p.set_points(torch.from_numpy(xy).cuda())
    Vc = pc.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    Vm = pm.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    assert np.allclose(Vm, np.abs(Vc), rtol=1e-5, atol=1e-6 * np.abs(Vc).max())


def test_srsd_at_the_65k_sample_size_sampled_planes():
    # 65,536 samples on the 256^2 lattice, 128 planes over 1-4 m, output pitch 8 mm -> 32 mm
    # (scales 1.024 -> 4.096); the oracle evaluates planes 0 and 127 with explicit scaled DFTs.
    N, pitch, F = 256, 2.0 / 256, 128
    depths = srsd_depths_c3b()
    out_pitch = srsd_pitches_c3b(depths)
    lat = relay_lattice(N, pitch)
    om, _ = O.phasor_frequencies(0.06, 4e-12, 8192, F)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=len(lat), srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(lat).cuda())
    P = random_phasors(len(lat), F, seed=BASE_SEED + 80)
    V = plan.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    M = 2 * N
    n_xy = np.rint(lat.astype(np.float64) / pitch).astype(int)
    u = O.idft_grid(O.nudft_type1_lattice(P, n_xy, M))
    for z in (0, len(depths) - 1):
        ref = O.srsd_from_grid(u, depths[z:z + 1], out_pitch[z:z + 1] / pitch, om, pitch, N)[0]
        assert rel(V[z], ref) < TOL


# ------------------------------------------------- SRSD + NURSD-2 (Eq. NURSD2_SRSD) ---

def scaled_voxels(N, pitch, center, scales, K, seed):
    # K voxels per plane, uniform over plane z's scaled aperture |x - c| <= N s_z delta / 2
    r = np.random.default_rng(seed)
    half = 0.5 * N * pitch * np.asarray(scales)[:, None, None]
    return (r.uniform(-1.0, 1.0, (len(scales), K, 2)) * 0.999 * half + np.asarray(center)).astype(np.float32)


@pytest.mark.parametrize("N,L,F,Z,seed", [(16, 300, 6, 5, 1), (32, 1200, 16, 7, 2)])
def test_srsd_points_match_oracle(N, L, F, Z, seed):
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, seed)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(xy).cuda())
    vox = scaled_voxels(N, pitch, center, out_pitch / pitch, 333, seed + 50)  # ragged K
    V = plan.srsd_forward_points(torch.from_numpy(P).cuda(), torch.from_numpy(vox).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.srsd_points(P, xy, center, pitch, N, depths, out_pitch / pitch, om, vox.astype(np.float64))
    assert rel(V, ref) < TOL


def test_srsd_points_on_each_scaled_lattice_equal_srsd_forward():
    N, L, F, Z = 32, 1200, 16, 7
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, 6)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(xy).cuda())
    Pg = torch.from_numpy(P).cuda()
    V = plan.srsd_forward(Pg).cpu().numpy()
    r = np.random.default_rng(7)
    # interior lattice points: m = -N/2 lies on the aperture edge, where float32 may round it out
    m = r.integers(-N // 2 + 1, N // 2, size=(Z, 64, 2))
    vox = (np.asarray(center)[None, None, :] + m * out_pitch[:, None, None]).astype(np.float32)
    Vp = plan.srsd_forward_points(Pg, torch.from_numpy(vox).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    want = np.stack([V[z, m[z, :, 1] + N // 2, m[z, :, 0] + N // 2] for z in range(Z)])
    assert rel(Vp, want) < TOL


def test_srsd_points_with_no_voxels():
    N, L, F, Z = 16, 300, 6, 5
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, 8)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(xy).cuda())
    out = plan.srsd_forward_points(torch.from_numpy(P).cuda(), torch.zeros((Z, 0, 2), dtype=torch.float32, device="cuda"))
    assert tuple(out.shape) == (Z, 0)
    assert plan.sync_status() == 0


def test_srsd_scales_below_and_above_one():
    # depths with s < 1 take Bluestein's chirp-z, the others the interpolated scaled DFT
    N, L, F, Z = 32, 1200, 16, 6
    xy, P, om, depths, _, pitch, center = case(N, L, F, Z, 9)
    scales = np.linspace(0.6, 1.8, Z)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=scales * pitch)
    plan.set_points(torch.from_numpy(xy).cuda())
    V = plan.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.srsd_forward(P, xy, center, pitch, N, depths, scales, om)
    for z in range(Z):
        assert rel(V[z], ref[z]) < TOL, (z, scales[z])


@pytest.mark.parametrize("F", [48, 200])
def test_srsd_channel_counts_beyond_64(F):
    # channel counts that are not a multiple of the kernel's channel chunk, above 64 and above 128
    N, L, Z = 16, 300, 4
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, 10 + F)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(xy).cuda())
    V = plan.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.srsd_forward(P, xy, center, pitch, N, depths, out_pitch / pitch, om)
    assert rel(V, ref) < TOL


@pytest.mark.parametrize("width,tol", [(4, 1e-2), (5, 2e-3), (7, 5e-5), (8, 5e-5)])
def test_srsd_at_every_kernel_width(width, tol):
    # both the spatial NUFFT and the scaled DFT's interpolation use the plan's ES width; the error
    # bounds are those of the type-2 output at the same widths
    N, L, F, Z = 32, 1200, 8, 5
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, 20 + width)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch, kernel_width=width)
    plan.set_points(torch.from_numpy(xy).cuda())
    V = plan.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.srsd_forward(P, xy, center, pitch, N, depths, out_pitch / pitch, om)
    assert rel(V, ref) < tol


def test_srsd_with_more_depths_than_one_tile_wave():
    # many depths (thousands of tiles) through the single persistent launch, scales 1 .. 4
    N, L, F, Z = 64, 2000, 4, 40
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, 30)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(xy).cuda())
    V = plan.srsd_forward(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.srsd_forward(P, xy, center, pitch, N, depths, out_pitch / pitch, om)
    assert rel(V, ref) < TOL


# --------------------------------------------- NU-SFFT (SRSD on non-uniform acquisition) ---

@pytest.mark.parametrize("N,L,F,Z,seed,width", [(16, 300, 6, 5, 41, 6), (32, 1500, 16, 7, 42, 6), (32, 900, 70, 3, 43, 7)])
def test_nu_sfft_matches_oracle(N, L, F, Z, seed, width):
    xy, P, om, depths, out_pitch, pitch, center = case(N, L, F, Z, seed)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=L, srsd_pitch=out_pitch, kernel_width=width)
    plan.set_points(torch.from_numpy(xy).cuda())
    V = plan.srsd_forward_nonuniform(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    ref = O.nu_sfft_forward(P, xy, center, pitch, N, depths, out_pitch / pitch, om)
    assert rel(V, ref) < TOL


def test_nu_sfft_on_the_lattice_equals_srsd_and_needs_scales_of_at_least_one():
    N, F, Z, pitch, center = 32, 8, 4, 0.02, (0.01, -0.03)
    lat = relay_lattice(N, pitch, center)
    P = torch.from_numpy(random_phasors(len(lat), F, seed=44)).cuda()
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    depths = np.linspace(0.3, 0.9, Z)
    plan = nursd.Plan(N, pitch, center, depths, om, max_points=len(lat), srsd_pitch=np.linspace(1.0, 3.0, Z) * pitch)
    plan.set_points(torch.from_numpy(lat).cuda())
    assert rel(plan.srsd_forward_nonuniform(P).cpu().numpy(), plan.srsd_forward(P).cpu().numpy()) < TOL
    low = nursd.Plan(N, pitch, center, depths, om, max_points=len(lat), srsd_pitch=np.linspace(0.7, 2.0, Z) * pitch)
    low.set_points(torch.from_numpy(lat).cuda())
    with pytest.raises(nursd.NursdError) as err:
        low.srsd_forward_nonuniform(P)
    assert err.value.status == nursd.nursd.NURSD_ERR_UNSUPPORTED


def test_nu_sfft_at_the_65k_sample_size_sampled_planes():
    # 65,536 samples on the 256^2 lattice, 128 planes over 1-4 m, pitch 8 -> 32 mm: on the lattice the
    # NU-SFFT is the SRSD of the gridded samples, evaluated by the oracle on planes 0 and 127
    N, pitch, F = 256, 2.0 / 256, 128
    depths = srsd_depths_c3b()
    out_pitch = srsd_pitches_c3b(depths)
    lat = relay_lattice(N, pitch)
    om, _ = O.phasor_frequencies(0.06, 4e-12, 8192, F)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=len(lat), srsd_pitch=out_pitch)
    plan.set_points(torch.from_numpy(lat).cuda())
    P = random_phasors(len(lat), F, seed=BASE_SEED + 81)
    V = plan.srsd_forward_nonuniform(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    M = 2 * N
    n_xy = np.rint(lat.astype(np.float64) / pitch).astype(int)
    u = O.idft_grid(O.nudft_type1_lattice(P, n_xy, M))
    for z in (0, len(depths) - 1):
        ref = O.srsd_from_grid(u, depths[z:z + 1], out_pitch[z:z + 1] / pitch, om, pitch, N)[0]
        assert rel(V[z], ref) < TOL
