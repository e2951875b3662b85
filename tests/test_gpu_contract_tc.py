"""The tensor-core contraction of a single reconstruction (table as the A operand, tf32 head and
tail products) against the FP64 oracle and against the FP32 bulk-copy kernel, forward (Eq.
RSD_conv summed over frequency) and adjoint.

Gates: FP64 oracle, relative L2 <= 1e-4 (the plan's FP32 gate).  Beyond it, the tensor form is held
to tc_bound(inner) above the FP32 kernel's own error: the tensor cores round each instruction's
accumulation toward zero (about 2^-23 of the running sum, always in the same direction), and a
K = 2 inner sum of three tf32 products takes 3 (2 inner / 8) such instructions; the head/tail split
itself loses about 2^-22 of each term (the tail x tail product and the tails' own rounding).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import BASE_SEED, random_phasors, random_spectrum, relay_uniform, workload_c2

pytestmark = pytest.mark.gpu
TOL = 1e-4


def tc_bound(inner):
    """Relative error the tensor form may add to an FP32 sum over `inner` complex terms."""
    return 3 * (2 * inner / 8) * 2.0 ** -23


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
    nursd.load_library()


def lattice_plan(N, F, Z, L=0, adjoint=True, seed=0, pitch=0.02):
    # adjoint plans keep the [class][z][f] table copy that the forward tensor form reads
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    depths = np.linspace(0.3, 1.5, Z)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=max(L, 1), adjoint=adjoint)
    xy = None
    if L:
        xy = relay_uniform(L, N * pitch / 2 * 0.999, seed=seed)
        plan.set_points(torch.from_numpy(xy).cuda())
    return plan, om, depths, xy


def both_kernels(plan, fn):
    plan.tune("contract_tc", 1)
    a = fn()
    plan.tune("contract_tc", 0)
    b = fn()
    return a, b


def test_forward_tensor_form_needs_an_adjoint_plan():
    # without the transposed table the forward keeps the FP32 kernel: identical results
    plan, *_ = lattice_plan(8, 16, 128, adjoint=False)
    Sd = torch.from_numpy(random_spectrum(16, 16, seed=BASE_SEED + 77)).cuda()
    tc, simt = both_kernels(plan, lambda: plan.propagate(Sd).cpu().numpy())
    assert np.array_equal(tc, simt)


def test_tunable_defaults_off_and_takes_only_0_or_1():
    plan, *_ = lattice_plan(8, 16, 128)
    assert plan.tuning()["contract_tc"] == 0
    plan.tune("contract_tc", 1)
    assert plan.tuning()["contract_tc"] == 1
    with pytest.raises(RuntimeError):
        plan.tune("contract_tc", 2)


# M = 16 (45 classes: one per CTA), 64 and 32; inner lengths of 1, 3 and 13 chunks (13 x 16 = 208,
# the longest the shared memory holds)
@pytest.mark.parametrize("N,F", [(8, 16), (32, 48), (16, 208)])
def test_forward_matches_oracle_and_the_fp32_kernel(N, F):
    Z = 128
    plan, om, depths, _ = lattice_plan(N, F, Z)
    M = 2 * N
    S = random_spectrum(M, F, seed=BASE_SEED + 70 + N)
    Sd = torch.from_numpy(S).cuda()
    tc, simt = both_kernels(plan, lambda: plan.propagate(Sd).cpu().numpy())
    assert rel(tc, simt) < tc_bound(F)
    U = np.transpose(S, (2, 0, 1)).astype(np.complex128)
    for iz in (0, 61, Z - 1):
        ref = O.propagate_depth(U, depths[iz], om, 0.02, N)
        e_tc, e_simt = rel(tc[iz], ref), rel(simt[iz], ref)
        assert e_tc < TOL and e_tc < e_simt + tc_bound(F)


@pytest.mark.parametrize("F,Z", [(8, 128), (32, 64), (24, 128)])
def test_shapes_outside_the_tensor_form_take_the_fp32_kernel(F, Z):
    # F = 8 and 24 are not multiples of 16, Z = 64 is not 128 rows: both settings run the same kernel
    plan, *_ = lattice_plan(16, F, Z)
    Sd = torch.from_numpy(random_spectrum(32, F, seed=BASE_SEED + 71)).cuda()
    tc, simt = both_kernels(plan, lambda: plan.propagate(Sd).cpu().numpy())
    assert np.array_equal(tc, simt)


# adjoint rows are the F = 128 frequencies; inner lengths Z = 16 and 48 (1 and 3 chunks)
@pytest.mark.parametrize("N,Z,L", [(8, 16, 200), (16, 48, 400)])
def test_adjoint_matches_oracle_and_the_fp32_kernel(N, Z, L):
    F = 128
    plan, om, depths, xy = lattice_plan(N, F, Z, L=L, adjoint=True, seed=BASE_SEED + 72 + N)
    V = cvec((Z, N, N), BASE_SEED + 73 + N)
    Vd = torch.from_numpy(V).cuda()
    tc, simt = both_kernels(plan, lambda: plan.adjoint(Vd).cpu().numpy())
    assert rel(tc, simt) < tc_bound(Z)
    ref = O.nursd_adjoint(V, xy, (0.0, 0.0), 0.02, N, depths, om)
    assert rel(tc, ref) < TOL and rel(tc, ref) < rel(simt, ref) + tc_bound(Z)


# ------------------------------------------- 65k-sample SPAD-array size ---

@pytest.fixture(scope="module")
def c2():
    wl = workload_c2()
    g = wl.geom
    om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=len(wl.xy),
                      adjoint=True)
    plan.set_points(torch.from_numpy(wl.xy).cuda())
    return wl, plan


def test_spad_forward_tensor_form_equals_the_fp32_kernel(c2):
    wl, plan = c2
    h = torch.from_numpy(wl.hist).cuda()
    tc, simt = both_kernels(plan, lambda: plan.forward(h).cpu().numpy())
    assert rel(tc, simt) < tc_bound(wl.geom.F)
    S = torch.from_numpy(random_spectrum(wl.geom.M, wl.geom.F, seed=BASE_SEED + 74)).cuda()
    tc, simt = both_kernels(plan, lambda: plan.propagate(S).cpu().numpy())
    assert rel(tc, simt) < tc_bound(wl.geom.F)


def test_spad_adjoint_identity_and_fp32_kernel(c2):
    wl, plan = c2
    g = wl.geom
    P = torch.from_numpy(random_phasors(len(wl.xy), g.F, seed=BASE_SEED + 75)).cuda()
    V = torch.from_numpy(cvec((g.Z, g.N, g.N), BASE_SEED + 76)).cuda()
    AP = plan.forward_phasor(P)
    AhV, AhV_simt = both_kernels(plan, lambda: plan.adjoint(V))
    assert rel(AhV.cpu().numpy(), AhV_simt.cpu().numpy()) < tc_bound(g.Z)
    lhs = torch.vdot(V.flatten().to(torch.complex128), AP.flatten().to(torch.complex128))
    rhs = torch.vdot(AhV.flatten().to(torch.complex128), P.flatten().to(torch.complex128))
    assert abs(complex(lhs - rhs)) < 1e-5 * abs(complex(lhs))
    assert plan.sync_status() == 0
