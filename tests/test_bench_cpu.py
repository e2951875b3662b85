"""CPU checks of bench.py's host-side comparison rows (no GPU).

The secondary CPU baseline runs the fast algorithm (ES spread as a sparse matrix, oversampled FFT,
deconvolution, transfer-function multiply with the frequency sum, inverse FFT with crop) in FP64;
on the tiny workload, over all frequencies, it must reproduce the FP64 oracle's NURSD-1 volume to
the ES kernel's accuracy (width 6, upsampling 2: ~1e-5), so that the row times the same operator.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle as O  # noqa: E402
from workloads import workload_c1  # noqa: E402


def test_cpu_fast_algorithm_equals_the_oracle_on_the_tiny_workload():
    wl = workload_c1()
    g = wl.geom
    om, wt = O.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    P = O.temporal_dft(wl.hist, g.t0, g.dt, om, wt)
    plan = bench.CpuFastPlan(wl.xy, g.N, g.pitch, g.center, g.depths, om, range(g.F))
    V, stages = plan.forward(P, workers=2)
    ref = O.nursd_forward(P, wl.xy, g.center, g.pitch, g.N, g.depths, om)
    assert np.linalg.norm(V - ref) / np.linalg.norm(ref) < 1e-4
    assert set(stages) == {"spread", "fft", "deconv", "contract", "ifft"}


def test_cpu_fast_rate_row_on_the_tiny_workload():
    row = bench.cpu_fast_rate(workload_c1(), n_freq=2)
    assert row["value"] > 0 and row["cores"] == (os.cpu_count() or 1)
    assert row["stages_s"]["temporal"] >= 0.0
