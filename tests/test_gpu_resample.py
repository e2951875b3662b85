"""GPU parity of the subsampled acquisition (Methods: Sampling Criteria for NLOS): keeping every D-th
relay sample and re-gridding by nearest neighbour (a copy: bit-exact against the oracle) or linear
interpolation (FP32 weights: 1e-6 relative), through the C ABI, and the reconstruction of the
re-gridded lattice against the oracle's (1e-4)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import BASE_SEED, random_phasors, relay_lattice

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    nursd.build()


@pytest.mark.parametrize("N,F,D", [(32, 16, 2), (33, 5, 4), (30, 7, 4), (16, 3, 1), (13, 2, 13), (256, 128, 5)])
def test_subsample_and_upsample_match_the_oracle(N, F, D):
    grid = random_phasors(N * N, F, seed=BASE_SEED + 300 + N + D).reshape(N, N, F)
    g = torch.from_numpy(grid).cuda()
    kept = nursd.subsample(g, D)
    ref_kept = O.subsample_grid(grid, D)
    assert np.array_equal(kept.cpu().numpy(), ref_kept)
    near = nursd.upsample(kept, N, D).cpu().numpy()
    assert np.array_equal(near, O.upsample_nearest(ref_kept, N, D))
    lin = nursd.upsample(kept, N, D, linear=True).cpu().numpy()
    assert rel(lin, O.upsample_linear(ref_kept, N, D)) < 1e-6


def test_arguments_are_checked_before_any_launch():
    g = torch.zeros((8, 8, 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(nursd.NursdError):
        nursd.subsample(g, 9)  # D > N
    lib = nursd.load_library()
    assert lib.nursd_upsample(8, 2, 2, 7, g.data_ptr(), g.data_ptr(), None) == nursd.nursd.NURSD_ERR_INVALID_ARG


def test_reconstruction_of_a_regridded_lattice_matches_the_oracle():
    # compression then re-gridding on the GPU, the lattice reconstruction (NURSD-1 at lattice samples)
    # on the GPU, against the oracle's forward of the oracle's re-gridded phasors
    N, F, D, pitch = 32, 6, 4, 0.02
    lat = relay_lattice(N, pitch, (0.0, 0.0))
    P = random_phasors(N * N, F, seed=BASE_SEED + 310)
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    depths = np.linspace(0.4, 1.0, 5)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=N * N)
    plan.set_points(torch.from_numpy(lat).cuda())
    for linear, up in ((False, O.upsample_nearest), (True, O.upsample_linear)):
        kept = nursd.subsample(torch.from_numpy(P.reshape(N, N, F)).cuda(), D)
        Pg = nursd.upsample(kept, N, D, linear=linear).reshape(N * N, F)
        V = plan.forward_phasor(Pg).cpu().numpy()
        Pr = up(O.subsample_grid(P.reshape(N, N, F), D), N, D).reshape(N * N, F)
        ref = O.nursd_forward(Pr, lat, (0.0, 0.0), pitch, N, depths, om)
        assert rel(V, ref) < 1e-4
    assert plan.sync_status() == 0
