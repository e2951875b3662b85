"""GPU parity of the per-frequency forms: the single-illumination volume (Eq. PF_RSD_Defn with the
illumination phase mask) and transient frames (Eq. Video_Voxel_Freq_Offset).

Gate: relative L2 error <= 1e-4 against the FP64 oracle (exact non-uniform DFT, explicit
per-frequency inverse DFTs) at the tiny and mid sizes, both for equispaced frequencies (the mask
advanced by rotation) and irregular ones (every phase reduced in FP64).  At the 65,536-sample
size: frames at t = 0 equal the ordinary forward (a property at any size), and on the lattice
variant sampled voxels of the illuminated volume equal the direct back-projection sum with the
mask.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import BASE_SEED, random_phasors, workload_c1, workload_c2_lattice, workload_mid

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
    nursd.load_library()


def make_plan(g, L, omega=None, weight=None):
    if omega is None:
        omega, weight = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    return nursd.Plan(g.N, g.pitch, g.center, g.depths, omega, weight, max_points=L)


ILLUM = (0.13, -0.21, 0.0)


@pytest.mark.parametrize("wlf", [workload_c1, workload_mid])
def test_illuminated_matches_oracle(wlf):
    wl = wlf()
    g = wl.geom
    plan = make_plan(g, len(wl.xy))
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    P = random_phasors(len(wl.xy), g.F, seed=BASE_SEED + 120)
    V = plan.forward_illuminated(torch.from_numpy(P).cuda(), ILLUM).cpu().numpy()
    assert plan.sync_status() == 0
    om, _ = O.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    ref = O.nursd_forward_illuminated(P, wl.xy, g.center, g.pitch, g.N, g.depths, om, ILLUM)
    assert rel(V, ref) < TOL


@pytest.mark.parametrize("wlf", [workload_c1, workload_mid])
def test_transient_frames_match_oracle(wlf):
    wl = wlf()
    g = wl.geom
    plan = make_plan(g, len(wl.xy))
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    P = random_phasors(len(wl.xy), g.F, seed=BASE_SEED + 121)
    times = g.t0 + np.array([0.0, 0.7e-9, 1.9e-9, 3.3e-9, 4.1e-9, 5.0e-9, 6.2e-9, 7.7e-9, 9.0e-9])  # 9: a ragged chunk
    Vt = plan.transient_frames(torch.from_numpy(P).cuda(), times).cpu().numpy()
    assert plan.sync_status() == 0
    om, _ = O.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    ref = O.nursd_transient_frames(P, wl.xy, g.center, g.pitch, g.N, g.depths, om, times)
    assert Vt.shape == ref.shape
    for t in range(len(times)):
        assert rel(Vt[t], ref[t]) < TOL, t


def test_irregular_frequencies_take_the_fp64_mask_path():
    wl = workload_c1()
    g = wl.geom
    om = 2 * math.pi * np.array([4.1e9, 4.5e9, 4.6e9, 5.0e9, 5.35e9, 5.9e9])
    plan = make_plan(g, len(wl.xy), omega=om, weight=np.ones(len(om)))
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    P = random_phasors(len(wl.xy), len(om), seed=BASE_SEED + 122)
    V = plan.forward_illuminated(torch.from_numpy(P).cuda(), ILLUM).cpu().numpy()
    ref = O.nursd_forward_illuminated(P, wl.xy, g.center, g.pitch, g.N, g.depths, om, ILLUM)
    assert rel(V, ref) < TOL
    Vt = plan.transient_frames(torch.from_numpy(P).cuda(), [1.3e-9, 2.2e-9]).cpu().numpy()
    ref_t = O.nursd_transient_frames(P, wl.xy, g.center, g.pitch, g.N, g.depths, om, [1.3e-9, 2.2e-9])
    assert rel(Vt, ref_t) < TOL


def test_invalid_per_frequency_calls_raise():
    wl = workload_c1()
    g = wl.geom
    plan = make_plan(g, len(wl.xy))
    P = torch.from_numpy(random_phasors(len(wl.xy), g.F, seed=BASE_SEED + 123)).cuda()
    with pytest.raises(RuntimeError):
        plan.forward_illuminated(P, ILLUM)  # no relay samples yet
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    with pytest.raises(nursd.NursdError):
        plan.forward_illuminated(P, (0.0, float("nan"), 0.0))
    with pytest.raises(nursd.NursdError):
        plan.transient_frames(P, [0.0, float("inf")])
    assert plan.sync_status() == 0


# ------------------------------------------------------------ spad-65k size ---

def test_spad_frame_at_time_zero_equals_forward():
    wl = workload_c2_lattice()
    g = wl.geom
    plan = make_plan(g, len(wl.xy))
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    P = torch.from_numpy(random_phasors(len(wl.xy), g.F, seed=BASE_SEED + 124)).cuda()
    V0 = plan.transient_frames(P, [0.0])[0].cpu().numpy()
    V = plan.forward_phasor(P).cpu().numpy()
    assert plan.sync_status() == 0
    assert rel(V0, V) < 1e-5


def test_spad_lattice_illuminated_equals_direct_sum_with_mask():
    # 256^2 samples on the lattice: each frequency's reconstruction is the direct sum, so sampled
    # voxels of the illuminated volume are exactly the mask-weighted direct sums.
    wl = workload_c2_lattice()
    g = wl.geom
    plan = make_plan(g, len(wl.xy))
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    om, wt = O.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    P = O.temporal_dft(wl.hist, g.t0, g.dt, om, wt)
    xp = (0.4, -0.3, 0.0)
    V = plan.forward_illuminated(torch.from_numpy(P.astype(np.complex64)).cuda(), xp).cpu().numpy()
    assert plan.sync_status() == 0
    r = np.random.default_rng(4)
    vz = r.integers(0, g.Z, 24)
    m = r.integers(0, g.N, size=(24, 2))
    vox = np.stack([(m[:, 0] - g.N // 2) * g.pitch, (m[:, 1] - g.N // 2) * g.pitch, g.depths[vz]], axis=1)
    R = O.fbp_direct_per_frequency(P, wl.xy.astype(np.float64), om, vox)  # [V][F]
    A = O.illumination_mask(xp, vox, om)  # [F][V]
    ref = np.einsum("fv,vf->v", A, R)
    assert rel(V[vz, m[:, 1], m[:, 0]], ref) < TOL


def test_several_depth_groups_with_a_ragged_last_one():
    # F = 128 puts 4 depths in a group (512 channels), so Z = 6 runs a group of 4 and one of 2
    wl = workload_c1()
    g = wl.geom
    om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, 8192, 128)  # 128 bins of a longer DFT stay positive
    depths = np.linspace(0.55, 1.45, 6)
    plan = nursd.Plan(g.N, g.pitch, g.center, depths, om, wt, max_points=len(wl.xy))
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    P = random_phasors(len(wl.xy), len(om), seed=BASE_SEED + 125)
    Pg = torch.from_numpy(P).cuda()
    V = plan.forward_illuminated(Pg, ILLUM).cpu().numpy()
    times = g.t0 + np.array([0.4e-9, 2.5e-9, 5.1e-9])
    Vt = plan.transient_frames(Pg, times).cpu().numpy()
    assert plan.sync_status() == 0
    om_o, _ = O.phasor_frequencies(g.lambda_c, g.dt, 8192, 128)
    M = 2 * g.N
    U = O.nudft_type1(P, O.relay_theta(wl.xy, g.center, g.pitch, M), M)
    G = O.transfer_functions(depths, om_o, M, g.pitch)
    assert rel(V, O.propagate_illuminated(U, G, g.N, ILLUM, g.center, g.pitch, depths, om_o)) < TOL
    assert rel(Vt, O.transient_frames(U, G, g.N, times, om_o)) < TOL


def test_empty_point_set_gives_zero_volume_and_frames():
    wl = workload_c1()
    g = wl.geom
    plan = make_plan(g, 8)
    plan.set_points(torch.zeros((0, 2), dtype=torch.float32, device="cuda"))
    P = torch.zeros((0, g.F), dtype=torch.complex64, device="cuda")
    assert float(plan.forward_illuminated(P, ILLUM).abs().max()) == 0.0
    assert float(plan.transient_frames(P, [0.0, 1e-9]).abs().max()) == 0.0
    assert plan.sync_status() == 0


@pytest.mark.parametrize("F,equispaced", [(8, True), (6, False)])
def test_products_formed_in_the_first_inverse_pass_match_oracle(F, equispaced):
    # M = 512 with Z % 4 == 0 and F even: the kx pass stages U and the table rows and forms the
    # products itself (channels 4 f + zz), the second pass writes channel-last volumes and the
    # masked sum runs a warp per voxel (fewer channels than lanes at F = 6; irregular frequencies
    # take the FP64 mask of every frequency); full outputs against the oracle
    N, pitch = 256, 2.0 / 256
    r = np.random.default_rng(BASE_SEED + 126)
    xy = r.uniform(-0.999, 0.999, (500, 2)).astype(np.float32)
    om = 2 * math.pi * (np.linspace(4.2e9, 5.8e9, F) if equispaced
                        else np.array([4.2e9, 4.4e9, 4.9e9, 5.05e9, 5.5e9, 5.8e9]))
    depths = np.array([0.6, 1.1, 1.7, 2.4])
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=len(xy))
    plan.set_points(torch.from_numpy(xy).cuda())
    P = random_phasors(len(xy), F, seed=BASE_SEED + 127)
    Pg = torch.from_numpy(P).cuda()
    xp = (0.35, -0.6, 0.0)
    V = plan.forward_illuminated(Pg, xp).cpu().numpy()
    times = np.array([3.0e-9, 6.5e-9])
    Vt = plan.transient_frames(Pg, times).cpu().numpy()
    assert plan.sync_status() == 0
    M = 2 * N
    U = O.nudft_type1(P, O.relay_theta(xy, (0.0, 0.0), pitch, M), M)
    G = O.transfer_functions(depths, om, M, pitch)
    assert rel(V, O.propagate_illuminated(U, G, N, xp, (0.0, 0.0), pitch, depths, om)) < TOL
    assert rel(Vt, O.transient_frames(U, G, N, times, om)) < TOL
