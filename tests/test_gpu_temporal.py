"""GPU parity of the temporal transform (Eq. PF_Response with Eq. PFPacket) on both tensor-core forms.

The tcgen05 form runs for T % 32 == 0 and 2F in {32, 64, 128, 256}; every other shape
takes the mma.sync form.  Both split each operand into an fp16 head and tail, and a
K-block of integer photon counts below 2048 skips the histogram-tail product, so the
cases cover integer counts (tail skipped) and fractional values (tail used), ragged L
(a partial last 128-row tile), L below one tile, and shapes on either side of the
dispatch.  Bar: relative L2 error <= 1e-5 against the FP64 oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import BASE_SEED

pytestmark = pytest.mark.gpu
C_LIGHT = 299792458.0


def rel(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    nursd.build()
    nursd.load_library()


def run_case(L, T, F, kind, seed):
    N, pitch, dt, t_pad, lam = 32, 1.0 / 32, 8e-12, 8192, 0.06  # band of F bins stays positive
    t0 = 0.5 / C_LIGHT
    rng = np.random.default_rng(seed)
    if kind == "counts":
        hist = rng.poisson(3.0, size=(L, T)).astype(np.float32)
    else:
        hist = rng.uniform(0.0, 50.0, size=(L, T)).astype(np.float32)
    om, wt = nursd.phasor_frequencies(lam, dt, t_pad, F)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), np.linspace(0.5, 1.5, 4), om, wt, T=T, t0=t0, dt=dt, max_points=L)
    P = plan.temporal_dft(torch.from_numpy(hist).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    om_o, wt_o = O.phasor_frequencies(lam, dt, t_pad, F)
    P_ref = O.temporal_dft(hist, t0, dt, om_o, wt_o)
    plan.close()
    return rel(P, P_ref)


@pytest.mark.parametrize("F", [16, 32, 64, 128])
@pytest.mark.parametrize("kind", ["counts", "fractional"])
def test_temporal_tcgen05_shapes(F, kind):
    # 1,000 rows: seven full 128-row tiles and a partial one
    assert run_case(1000, 256, F, kind, BASE_SEED + 60 + F) < 1e-5


@pytest.mark.parametrize("L", [1, 127, 129])
def test_temporal_short_inputs(L):
    assert run_case(L, 128, 128, "fractional", BASE_SEED + 70 + L) < 1e-5


@pytest.mark.parametrize("T", [32, 96])
def test_temporal_odd_k_block_counts(T):
    # one K-block, and an odd number of K-blocks (the producers stage K-blocks in pairs)
    assert run_case(700, T, 64, "fractional", BASE_SEED + 75 + T) < 1e-5


@pytest.mark.parametrize("T,F", [(200, 16), (256, 24), (64, 256)])
def test_temporal_other_shapes(T, F):
    # T not a multiple of 64, 2F outside the tcgen05 set, and F = 256 (2F = 512): the mma.sync form
    assert run_case(300, T, F, "fractional", BASE_SEED + 80 + T + F) < 1e-5
