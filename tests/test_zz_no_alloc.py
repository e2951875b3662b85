"""nursd_nufft1_noalloc: the NUFFT type 1 for callers that cannot allocate device memory.

Callers that run inside an engine owning all device memory through a fixed
pool cannot call cudaMalloc, so they cannot create a plan.  This entry point
computes the same spectrum as nursd_set_points + nursd_nufft1 using only a
fixed scratch array inside libnursd.  Here it is called through the C ABI
several times in a row, with different geometries, and each result is
compared with the plan-based entry point on the same inputs.  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2501_05244_gb300 as nursd
from paper_2501_05244_gb300 import nursd as binding
from oracle import nursd_oracle as O
from workloads import BASE_SEED, random_phasors, workload_c1, workload_mid

pytestmark = pytest.mark.gpu
TOL = 1e-4  # the parity tolerance used by every GPU test


def rel(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    nursd.build()
    return nursd.load_library()


def case(wl, seed):
    g = wl.geom
    xy = torch.from_numpy(wl.xy).cuda()
    P = torch.from_numpy(random_phasors(len(wl.xy), g.F, seed=seed)).cuda()
    return g, xy, P


def with_plan(g, xy, P):
    plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, np.linspace(2e10, 4e10, g.F), max_points=xy.shape[0])
    plan.set_points(xy)
    U = plan.nufft1(P)
    torch.cuda.synchronize()
    out = U.cpu().numpy()
    plan.close()
    return out


def no_alloc(lib, g, xy, P):
    M = 2 * g.N
    out = torch.empty((M, M, g.F), dtype=torch.complex64, device="cuda")
    rc = lib.nursd_nufft1_noalloc(g.N, g.pitch, g.center[0], g.center[1], 6, xy.shape[0],
                                  ctypes.c_void_p(xy.data_ptr()), g.F, ctypes.c_void_p(P.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, nursd.status_string(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_no_alloc_matches_the_plan_entry_point_on_consecutive_calls(lib):
    a = case(workload_mid(), BASE_SEED + 90)   # N = 64, 4,096 samples, F = 16
    b = case(workload_c1(), BASE_SEED + 91)    # N = 32, 1,024 samples, F = 16
    ref_a = with_plan(*a)
    ref_b = with_plan(*b)
    # two calls in a row with different sizes, then the first again: the shared
    # scratch keeps the previous call's contents, which must not leak into the next
    assert rel(no_alloc(lib, *a), ref_a) < TOL
    assert rel(no_alloc(lib, *b), ref_b) < TOL
    assert rel(no_alloc(lib, *a), ref_a) < TOL


def test_no_alloc_matches_the_exact_nonuniform_dft(lib):
    # against the FP64 oracle's explicit sum, not only against the plan path: its own deconvolution
    # and quadrature tables are checked on their own
    g, xy, P = case(workload_c1(), BASE_SEED + 92)  # N = 32, 1,024 samples, F = 16
    U = no_alloc(lib, g, xy, P)
    M = 2 * g.N
    ref = O.nudft_type1(P.cpu().numpy().astype(np.complex128), O.relay_theta(xy.cpu().numpy(), g.center, g.pitch, M), M)
    assert rel(np.transpose(U, (2, 0, 1)), ref) < TOL


def test_no_alloc_rejects_sizes_beyond_its_scratch(lib):
    g = workload_c1().geom
    out = torch.empty((1024, 1024, 256), dtype=torch.complex64, device="cuda")
    xy = torch.zeros((8, 2), dtype=torch.float32, device="cuda")
    P = torch.zeros((8, 256), dtype=torch.complex64, device="cuda")
    rc = lib.nursd_nufft1_noalloc(512, g.pitch, 0.0, 0.0, 6, 8, ctypes.c_void_p(xy.data_ptr()), 256,
                                  ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == binding.NURSD_ERR_UNSUPPORTED
