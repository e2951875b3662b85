"""GPU parity of 3D NURSD for non-planar relays (Eq. 3D_NURSD) against the FP64 oracle, through the C
ABI: relay heights within the z range, off the grid in all three axes; samples on the 3D grid (where
stage 1 is a direct sum); ragged sizes; a height beyond the range flagged.  Gate: 1e-4 relative L2."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import random_phasors

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


def case(N, L, F, Z, Mz, seed, on_grid=False, pitch=0.02, dz=0.015):
    r = np.random.default_rng(seed)
    half = N * pitch / 2 * 0.999
    hz = Mz * dz / 4 * 0.999
    if on_grid:
        n = r.integers(-N // 2, N // 2, (L, 2))
        xy = (n * pitch).astype(np.float32)
        h = (r.integers(-Mz // 4 + 1, Mz // 4, L) * dz).astype(np.float32)
    else:
        xy = r.uniform(-half, half, (L, 2)).astype(np.float32)
        h = r.uniform(-hz, hz, L).astype(np.float32)
    P = random_phasors(L, F, seed=seed + 1)
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    dist = np.linspace(0.3, 0.8, Z)  # plane distances from the reference plane z0 = 0
    return xy, h, P, om, dist, pitch, dz


@pytest.mark.parametrize("N,L,F,Z,Mz,seed,on_grid", [(16, 300, 4, 3, 8, 1, False), (16, 200, 3, 2, 16, 2, True),
                                                      (32, 777, 6, 5, 16, 3, False), (8, 1, 1, 1, 8, 4, False)])
def test_3d_nursd_matches_the_oracle(N, L, F, Z, Mz, seed, on_grid):
    xy, h, P, om, dist, pitch, dz = case(N, L, F, Z, Mz, seed, on_grid)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), dist, om, max_points=L)
    plan.enable_3d(dz, Mz)
    plan.set_points_3d(torch.from_numpy(xy).cuda(), torch.from_numpy(h).cuda())
    V = plan.forward_3d(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    xyz = np.column_stack([xy.astype(np.float64), h.astype(np.float64)])
    ref = O.nursd3d_forward(P, xyz, (0.0, 0.0), pitch, N, 0.0, dz, Mz, dist, om)
    assert rel(V, ref) < TOL


def test_3d_arguments_and_out_of_range_heights():
    xy, h, P, om, dist, pitch, dz = case(16, 50, 2, 2, 8, 5)
    plan = nursd.Plan(16, pitch, (0.0, 0.0), dist, om, max_points=50)
    Pg = torch.from_numpy(P).cuda()
    with pytest.raises(nursd.NursdError):  # not enabled
        plan.set_points_3d(torch.from_numpy(xy).cuda(), torch.from_numpy(h).cuda())
    with pytest.raises(nursd.NursdError) as err:  # the z window would not fit the fine grid
        plan.enable_3d(dz, 4)
    assert err.value.status == nursd.nursd.NURSD_ERR_UNSUPPORTED
    plan.enable_3d(dz, 8)
    plan.set_points(torch.from_numpy(xy).cuda())
    with pytest.raises(nursd.NursdError):  # the current points carry no heights
        plan.forward_3d(Pg)
    h2 = h.copy()
    h2[7] = 8 * dz  # beyond Mz dz / 4
    plan.set_points_3d(torch.from_numpy(xy).cuda(), torch.from_numpy(h2).cuda())
    plan.forward_3d(Pg)
    assert plan.sync_status() == nursd.nursd.NURSD_ERR_POINT_OUT_OF_RANGE


def test_3d_nursd_at_a_lattice_of_128():
    # M = 256: the z pass and the table's z transform run over 65,536 lateral modes (more than one grid
    # dimension holds), a few samples keep the oracle short
    xy, h, P, om, dist, pitch, dz = case(128, 20, 1, 2, 8, 6, pitch=0.015)
    plan = nursd.Plan(128, pitch, (0.0, 0.0), dist, om, max_points=20)
    plan.enable_3d(dz, 8)
    plan.set_points_3d(torch.from_numpy(xy).cuda(), torch.from_numpy(h).cuda())
    V = plan.forward_3d(torch.from_numpy(P).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    xyz = np.column_stack([xy.astype(np.float64), h.astype(np.float64)])
    ref = O.nursd3d_forward(P, xyz, (0.0, 0.0), pitch, 128, 0.0, dz, 8, dist, om)
    assert rel(V, ref) < TOL
