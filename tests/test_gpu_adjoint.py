"""GPU parity of the adjoint (a10), the gradients (a11) and the NURSD-2/3 type-2
output at arbitrary voxels (a8), against the FP64 oracle, through the C ABI.

Tolerances: 1e-4 relative L2 for complex outputs (the parity gate); the
adjoint identity <A P, V> = <P, A^H V> on the GPU to 1e-5 relative (the
NUFFT type-2 is the exact adjoint of the implemented type-1, so only FP32
rounding remains).  Position gradients are the spectral derivative (type 2 of
i kx R and i ky R), as accurate as a type-2 value, and are gated per coordinate
against FP64 central differences: |g - fd| <= 1e-3 max(|fd|, 1e-2 rms(fd)) (a
coordinate whose gradient is a hundred times below the typical one has no
meaningful relative error, so its denominator is floored there), and to 1e-4
relative L2 against the oracle's analytic gradient.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import (BASE_SEED, random_phasors, random_plane_points, relay_keystone, relay_lattice,
                       workload_c1, workload_mid)

pytestmark = pytest.mark.gpu
TOL = 1e-4
GRAD_TOL = 1e-4
FD_REL = 1e-3


def fd_gate(g, fd):
    """Per-coordinate relative errors |g - fd| / max(|fd|, 1e-2 rms(fd))."""
    g, fd = np.asarray(g, np.float64), np.asarray(fd, np.float64)
    floor = 1e-2 * np.sqrt(np.mean(fd ** 2))
    return np.abs(g - fd) / np.maximum(np.abs(fd), floor)


def rel(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cvec(shape, seed):
    r = np.random.default_rng(seed)
    return ((r.standard_normal(shape) + 1j * r.standard_normal(shape)) / math.sqrt(2)).astype(np.complex64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    nursd.build()


def small_case(N=16, L=300, F=6, Z=5, seed=1, pitch=0.02, center=(0.01, -0.03)):
    r = np.random.default_rng(seed)
    half = N * pitch / 2
    xy = (r.uniform(-half, half, (L, 2)) * 0.999 + np.asarray(center)).astype(np.float32)
    P = random_phasors(L, F, seed=seed + 1)
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    depths = np.linspace(0.3, 0.9, Z)
    return dict(N=N, pitch=pitch, center=center, xy=xy, P=P, om=om, depths=depths)


def plan_for(c, **kw):
    p = nursd.Plan(c["N"], c["pitch"], c["center"], c["depths"], c["om"], max_points=len(c["xy"]), adjoint=True, **kw)
    p.set_points(torch.from_numpy(c["xy"]).cuda())
    return p


def oracle_args(c):
    return (c["center"], c["pitch"], c["N"], c["depths"], c["om"])


# ----------------------------------------------------------------- a10 ---

@pytest.mark.parametrize("seed,N,L,F,Z", [(1, 16, 300, 6, 5), (2, 32, 1500, 16, 9), (3, 8, 1, 1, 1), (4, 16, 777, 33, 70)])
def test_adjoint_matches_oracle(seed, N, L, F, Z):
    c = small_case(N, L, F, Z, seed)
    plan = plan_for(c)
    V = cvec((Z, N, N), seed + 10)
    got = plan.adjoint(torch.from_numpy(V).cuda()).cpu().numpy()
    ref = O.nursd_adjoint(V, c["xy"], *oracle_args(c))
    assert rel(got, ref) < TOL


def test_adjoint_identity_on_gpu():
    c = small_case(32, 2000, 16, 12, seed=5)
    plan = plan_for(c)
    P = torch.from_numpy(c["P"]).cuda()
    V = torch.from_numpy(cvec((12, 32, 32), 6)).cuda()
    AP = plan.forward_phasor(P)
    AhV = plan.adjoint(V)
    lhs = torch.vdot(V.flatten().to(torch.complex128), AP.flatten().to(torch.complex128))
    rhs = torch.vdot(AhV.flatten().to(torch.complex128), P.flatten().to(torch.complex128))
    assert abs(complex(lhs - rhs)) < 1e-5 * abs(complex(lhs))


@pytest.mark.parametrize("width", [4, 5, 7, 8])
def test_adjoint_identity_at_every_kernel_width(width):
    # the type-2 interpolation (adjoint of the spread) is compiled per width; at any width it is the
    # exact adjoint of the implemented type 1, so the identity holds to FP32 rounding
    c = small_case(32, 1500, 8, 6, seed=20 + width)
    plan = plan_for(c, kernel_width=width)
    P = torch.from_numpy(c["P"]).cuda()
    V = torch.from_numpy(cvec((6, 32, 32), 30 + width)).cuda()
    AP = plan.forward_phasor(P)
    AhV = plan.adjoint(V)
    assert plan.sync_status() == 0
    lhs = torch.vdot(V.flatten().to(torch.complex128), AP.flatten().to(torch.complex128))
    rhs = torch.vdot(AhV.flatten().to(torch.complex128), P.flatten().to(torch.complex128))
    assert abs(complex(lhs - rhs)) < 1e-5 * abs(complex(lhs))


def test_adjoint_on_the_tiny_workload():
    wl = workload_c1()
    g = wl.geom
    om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, max_points=len(wl.xy), adjoint=True)
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    V = cvec((g.Z, g.N, g.N), 7)
    got = plan.adjoint(torch.from_numpy(V).cuda()).cpu().numpy()
    ref = O.nursd_adjoint(V, wl.xy, g.center, g.pitch, g.N, g.depths, om)
    assert rel(got, ref) < TOL


# ----------------------------------------------------------------- a11 ---

def test_gradients_match_oracle_and_finite_differences():
    c = small_case(16, 200, 6, 4, seed=11)
    plan = plan_for(c)
    Vt = cvec((4, 16, 16), 12)
    P = torch.from_numpy(c["P"]).cuda()
    V = plan.forward_phasor(P)
    w = 2 * (V - torch.from_numpy(Vt).cuda())
    gP, gx = plan.grad_points(w, P)
    gP_ref, gx_ref = O.nursd_gradients(c["P"], c["xy"], *oracle_args(c), Vt)
    assert rel(gP.cpu().numpy(), gP_ref) < TOL
    assert np.linalg.norm(gx.cpu().numpy() - gx_ref) / np.linalg.norm(gx_ref) < GRAD_TOL
    # FP64 central differences of the oracle loss on random coordinates, each gated on its own
    r = np.random.default_rng(13)
    args = oracle_args(c)
    gxc = gx.cpu().numpy()
    got, fds = [], []
    for l in r.choice(len(c["xy"]), 24, replace=False):
        a = int(r.integers(0, 2))
        h = 1e-6
        xp = c["xy"].astype(np.float64).copy()
        xm = xp.copy()
        xp[l, a] += h
        xm[l, a] -= h
        fds.append((O.nursd_loss(c["P"], xp, *args, Vt) - O.nursd_loss(c["P"], xm, *args, Vt)) / (2 * h))
        got.append(gxc[l, a])
    err = fd_gate(got, fds)
    assert err.max() < FD_REL, (err.max(), np.median(err))


def test_autograd_function_matches_oracle():
    from paper_2501_05244_gb300.autograd import nursd_apply

    c = small_case(16, 150, 4, 3, seed=21)
    plan = plan_for(c)
    Vt = torch.from_numpy(cvec((3, 16, 16), 22)).cuda()
    P = torch.from_numpy(c["P"]).cuda().requires_grad_(True)
    xy = torch.from_numpy(c["xy"]).cuda().requires_grad_(True)
    V = nursd_apply(plan, P, xy)
    loss = (V - Vt).abs().pow(2).sum()
    loss.backward()
    gP_ref, gx_ref = O.nursd_gradients(c["P"], c["xy"], *oracle_args(c), Vt.cpu().numpy())
    assert rel(P.grad.cpu().numpy(), gP_ref) < TOL
    assert np.linalg.norm(xy.grad.cpu().numpy() - gx_ref) / np.linalg.norm(gx_ref) < GRAD_TOL


def test_gradient_operator_at_the_65k_sample_grid128_size():
    # 65,536 keystone samples, F = 128, 128^2 x 64: a seeded w feeds both sides; the oracle
    # evaluates the adjoint spectrum plane by plane and the gradients at 64 sampled samples.
    N, pitch, F, Z = 128, 2.0 / 128, 128, 64
    xy = relay_keystone(seed=BASE_SEED + 60)
    om, _ = O.phasor_frequencies(0.06, 4e-12, 8192, F)
    depths = np.linspace(0.5, 3.0, Z)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=len(xy), adjoint=True)
    plan.set_points(torch.from_numpy(xy).cuda())
    P = random_phasors(len(xy), F, seed=BASE_SEED + 61)
    W = cvec((Z, N, N), BASE_SEED + 62)
    gP, gx = plan.grad_points(torch.from_numpy(W).cuda(), torch.from_numpy(P).cuda())
    R = O.adjoint_spectrum_depthwise(W, depths, om, pitch)
    idx = np.random.default_rng(63).choice(len(xy), 64, replace=False)
    th = O.relay_theta(xy[idx], (0.0, 0.0), pitch, 2 * N)
    gP_ref, gx_ref = O.gradients_from_w(R, P[idx], th, pitch)
    assert rel(gP.cpu().numpy()[idx], gP_ref) < TOL
    assert np.linalg.norm(gx.cpu().numpy()[idx] - gx_ref) / np.linalg.norm(gx_ref) < GRAD_TOL


def test_position_gradient_against_fp64_differences_at_the_65k_gradient_workload():
    # The gradient workload: 65,536 keystone samples x_true, relay positions x = x_true + N(0, 2 mm),
    # phasors of the simulated scene, target V_t = A(P, x_true), 128^2 x 64 voxels, F = 128.  The
    # residual r = A(P, x) - V_t of the GPU forward is promoted to FP64 and shared by both sides:
    # the GPU gradient from w = 2 r, and for 64 random coordinates the exact FP64 change of the loss
    # when that one sample moves by +-1 um (its single-sample forward term, contracted and cropped).
    from workloads import workload_c5
    wl = workload_c5()
    g = wl.geom
    om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    rng = np.random.default_rng(BASE_SEED + 64)
    half = g.N * g.pitch / 2
    x_true = wl.xy
    x_rel = np.clip(x_true + rng.normal(0.0, 2e-3, x_true.shape), -0.9999 * half, 0.9999 * half).astype(np.float32)
    plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=len(x_true),
                      adjoint=True)
    P = plan.temporal_dft(torch.from_numpy(wl.hist).cuda())
    plan.set_points(torch.from_numpy(x_true).cuda())
    Vt = plan.forward_phasor(P).clone()
    plan.set_points(torch.from_numpy(x_rel).cuda())
    resid = plan.forward_phasor(P) - Vt
    _, gx = plan.grad_points(2 * resid, P, want_phasor=False)
    assert plan.sync_status() == 0
    rows = rng.choice(len(x_rel), 64, replace=False)
    axes = rng.integers(0, 2, 64)
    P_rows = P.cpu().numpy()[rows].astype(np.complex128)
    fd = O.position_loss_differences(resid.cpu().numpy().astype(np.complex128), P_rows,
                                     x_rel[rows].astype(np.float64), axes, 1e-6, g.center, g.pitch, g.N, g.depths,
                                     om)
    err = fd_gate(gx.cpu().numpy()[rows, axes], fd)
    assert err.max() < FD_REL, (err.max(), np.median(err))


# ------------------------------------------------------------------ a8 ---

@pytest.mark.parametrize("seed,N,L,F,Z,K", [(31, 16, 300, 6, 5, 257), (32, 32, 1500, 16, 9, 1000), (33, 8, 3, 2, 1, 5)])
def test_type2_voxels_match_oracle(seed, N, L, F, Z, K):
    c = small_case(N, L, F, Z, seed)
    plan = plan_for(c)
    half = N * c["pitch"] / 2 * 0.999
    vox = random_plane_points(Z, K, half, c["center"], seed=seed + 5)
    got = plan.forward_points(torch.from_numpy(c["P"]).cuda(), torch.from_numpy(vox).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    M = 2 * N
    U = O.nudft_type1(c["P"], O.relay_theta(c["xy"], c["center"], c["pitch"], M), M)
    Gh = O.transfer_functions(c["depths"], c["om"], M, c["pitch"])
    th = np.stack([O.relay_theta(vox[z], c["center"], c["pitch"], M) for z in range(Z)])
    ref = O.propagate_points(U, Gh, th)
    assert rel(got, ref) < TOL


@pytest.mark.parametrize("width,tol", [(4, 1e-2), (5, 2e-3), (7, 5e-5), (8, 5e-5)])
def test_type2_voxels_at_every_kernel_width(width, tol):
    # the plane interpolation is compiled per width; ES accuracy at upsampling 2 bounds the error
    c = small_case(32, 1500, 8, 4, seed=60 + width)
    plan = plan_for(c, kernel_width=width)
    half = 32 * c["pitch"] / 2 * 0.999
    vox = random_plane_points(4, 500, half, c["center"], seed=70 + width)
    got = plan.forward_points(torch.from_numpy(c["P"]).cuda(), torch.from_numpy(vox).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    M = 64
    U = O.nudft_type1(c["P"], O.relay_theta(c["xy"], c["center"], c["pitch"], M), M)
    Gh = O.transfer_functions(c["depths"], c["om"], M, c["pitch"])
    th = np.stack([O.relay_theta(vox[z], c["center"], c["pitch"], M) for z in range(4)])
    assert rel(got, O.propagate_points(U, Gh, th)) < tol


def test_type2_at_lattice_voxels_equals_the_lattice_forward():
    # dyadic pitch and centre: every lattice voxel, including the row and column at
    # exactly -N delta / 2, is representable in float32 and inside the aperture
    c = small_case(32, 900, 8, 6, seed=41, pitch=2.0 ** -6, center=(0.25, -0.125))
    plan = plan_for(c)
    P = torch.from_numpy(c["P"]).cuda()
    lat = relay_lattice(32, c["pitch"], c["center"])
    vox = torch.from_numpy(np.broadcast_to(lat[None], (6,) + lat.shape).copy()).cuda()
    Vp = plan.forward_points(P, vox).cpu().numpy()
    V = plan.forward_phasor(P).cpu().numpy().reshape(6, -1)
    assert rel(Vp, V) < 1e-5


def test_type2_out_of_aperture_voxel_is_flagged():
    c = small_case(16, 100, 4, 2, seed=51)
    plan = plan_for(c)
    vox = random_plane_points(2, 10, 0.1, c["center"], seed=52)
    vox[1, 3, 1] = c["center"][1] + 16 * c["pitch"]
    out = plan.forward_points(torch.from_numpy(c["P"]).cuda(), torch.from_numpy(vox).cuda())
    assert plan.sync_status() == nursd.nursd.NURSD_ERR_POINT_OUT_OF_RANGE
    assert complex(out[1, 3]) == 0


def test_type2_voxels_at_the_spad_size_sampled_planes():
    # 65,536 samples on the 256^2 lattice (so the exact type-1 spectrum is an FFT), 128 planes x
    # 16,384 random voxels (2,097,152 in all); the oracle checks 3 planes x 64 voxels.
    N, pitch, F, Z, K = 256, 2.0 / 256, 128, 128, 16384
    lat = relay_lattice(N, pitch)
    om, _ = O.phasor_frequencies(0.06, 4e-12, 8192, F)
    depths = np.linspace(0.5, 3.0, Z)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=len(lat))
    plan.set_points(torch.from_numpy(lat).cuda())
    P = random_phasors(len(lat), F, seed=BASE_SEED + 70)
    vox = random_plane_points(Z, K, 0.999, seed=BASE_SEED + 71)
    got = plan.forward_points(torch.from_numpy(P).cuda(), torch.from_numpy(vox).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    M = 2 * N
    n_xy = np.rint(lat.astype(np.float64) / pitch).astype(int)
    U = O.nudft_type1_lattice(P, n_xy, M)
    r = np.random.default_rng(72)
    for z in (0, 70, Z - 1):
        Y = np.zeros((M, M), complex)
        for f in range(F):
            Y += U[f] * O.transfer_function(O.rsd_kernel(M, pitch, depths[z], om[f] / O.C))
        v = r.choice(K, 64, replace=False)
        th = O.relay_theta(vox[z, v], (0.0, 0.0), pitch, M)
        ref = O.nudft_type2(Y[None], th)[:, 0] / (M * M)
        assert rel(got[z, v], ref) < TOL
