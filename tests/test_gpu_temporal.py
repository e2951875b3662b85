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


# ------------------------------------------------------------------ FP32 input range
# Eq. PF_Response places no limit on the histogram values.  The fp16 head/tail split carries
# ~22 bits of every value of a row whose max lies in [2^-3, 65504); rows outside that window
# are recomputed scaled by a power of two, and the band-pass weight multiplies the accumulator
# instead of being rounded into the fp16 twiddles.  Each row (and each column, for the weights)
# is checked on its own, so a small row cannot hide behind a large one.

RANGE_SHAPES = [(256, 64), (200, 64)]  # tcgen05 form; mma.sync form (T % 32 != 0)


def per_row_err(P, P_ref):
    P = np.asarray(P, np.complex128)
    return float(np.max(np.linalg.norm(P - P_ref, axis=1) / np.linalg.norm(P_ref, axis=1)))


def temporal_pair(hist, F, weight=None):
    L, T = hist.shape
    dt, t_pad, lam = 8e-12, 8192, 0.06
    t0 = 0.5 / C_LIGHT
    om, wt = nursd.phasor_frequencies(lam, dt, t_pad, F)
    if weight is not None:
        wt = np.asarray(weight, np.float64)
    plan = nursd.Plan(32, 1.0 / 32, (0.0, 0.0), np.linspace(0.5, 1.5, 4), om, wt, T=T, t0=t0, dt=dt, max_points=L)
    P = plan.temporal_dft(torch.from_numpy(hist).cuda()).cpu().numpy()
    assert plan.sync_status() == 0
    plan.close()
    return P, O.temporal_dft(hist, t0, dt, om, wt)


def range_hist(kind, L, T, rng):
    if kind == "counts_to_1e7":  # row means log-uniform over 1 .. 1e7 photons per bin
        mean = 10.0 ** rng.uniform(0.0, 7.0, size=(L, 1))
        return rng.poisson(mean * rng.uniform(0.2, 1.0, size=(L, T))).astype(np.float32)
    if kind == "normalised_1e-6":
        return rng.uniform(0.0, 2e-6, size=(L, T)).astype(np.float32)
    if kind == "one_huge_bin":  # small background with a single bin of 1e7 in every other row
        h = rng.uniform(0.0, 1.0, size=(L, T)).astype(np.float32)
        rows = np.arange(0, L, 2)
        h[rows, rng.integers(0, T, size=rows.size)] = 1e7
        return h
    if kind == "exponents_pm120":  # row scales 2^-120 .. 2^120, signed values
        scale = np.exp2(rng.uniform(-120.0, 120.0, size=(L, 1)))
        return (rng.uniform(-1.0, 1.0, size=(L, T)) * scale).astype(np.float32)
    raise ValueError(kind)


@pytest.mark.parametrize("T,F", RANGE_SHAPES)
@pytest.mark.parametrize("kind", ["counts_to_1e7", "normalised_1e-6", "one_huge_bin", "exponents_pm120"])
def test_temporal_full_fp32_range(T, F, kind):
    rng = np.random.default_rng(BASE_SEED + 90 + T + len(kind))
    hist = range_hist(kind, 700, T, rng)
    P, P_ref = temporal_pair(hist, F)
    assert np.all(np.isfinite(P))
    assert per_row_err(P, P_ref) < 1e-5


@pytest.mark.parametrize("T,F", RANGE_SHAPES)
def test_temporal_weights_down_to_1e_8(T, F):
    # a caller weight per frequency spanning 1e-8 .. 1: every column to 1e-5 of its own norm
    rng = np.random.default_rng(BASE_SEED + 95 + T)
    hist = rng.uniform(0.0, 50.0, size=(500, T)).astype(np.float32)
    weight = np.logspace(-8.0, 0.0, F)
    P, P_ref = temporal_pair(hist, F, weight)
    col = np.linalg.norm(np.asarray(P, np.complex128) - P_ref, axis=0) / np.linalg.norm(P_ref, axis=0)
    assert float(col.max()) < 1e-5


def test_temporal_all_rows_in_range_and_out_of_range_in_one_call():
    # rows of every kind interleaved, in a call longer than the tcgen05 grid (several tiles per CTA)
    T, F = 256, 128
    rng = np.random.default_rng(BASE_SEED + 97)
    parts = [range_hist(k, 4000, T, rng) for k in ("counts_to_1e7", "normalised_1e-6", "one_huge_bin")]
    parts.append(rng.poisson(3.0, size=(4000, T)).astype(np.float32))
    hist = np.stack(parts, axis=1).reshape(-1, T)
    P, P_ref = temporal_pair(hist, F)
    assert per_row_err(P, P_ref) < 1e-5


def test_forward_and_batched_with_counts_above_fp16_range():
    # the full forward (phasors written in the spread's slot order) and the batched form
    # (mma.sync temporal over a ragged batch) on histograms scaled far above 65504; 2F = 32 and
    # T = 64 put the single forward on the tcgen05 form
    N, F, Z, T = 16, 16, 4, 64
    pitch, center = 0.02, (0.0, 0.0)
    r = np.random.default_rng(BASE_SEED + 98)
    from workloads import relay_uniform
    sizes = [300, 1, 900]
    xys = [relay_uniform(L, N * pitch / 2 * 0.999, seed=BASE_SEED + 99 + i) for i, L in enumerate(sizes)]
    hists = [(r.poisson(5.0, size=(L, T)) * 4096.0 * (1 + b)).astype(np.float32) for b, L in enumerate(sizes)]
    om = 2 * np.pi * np.linspace(3e9, 6e9, F)
    t0, dt, depths = 1e-9, 16e-12, np.linspace(0.3, 0.9, Z)
    plan = nursd.Plan(N, pitch, center, depths, om, T=T, t0=t0, dt=dt, max_points=max(sizes), max_batch=3)
    dx = [torch.from_numpy(x).cuda() for x in xys]
    dh = [torch.from_numpy(h).cuda() for h in hists]
    outs = plan.forward_batched(dx, dh)
    P = O.temporal_dft(hists[2], t0, dt, om, np.ones(F))
    ref = O.nursd_forward(P, xys[2], center, pitch, N, depths, om)
    plan.set_points(dx[2])
    single = plan.forward(dh[2]).cpu().numpy()
    assert plan.sync_status() == 0
    assert rel(single, ref) < 1e-4
    assert rel(outs[2].cpu().numpy(), ref) < 1e-4
    plan.close()
