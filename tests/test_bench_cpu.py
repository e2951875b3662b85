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


class _Tuned:
    def __init__(self, tc):
        self.tc = tc

    def tuning(self):
        return {"contract_tc": self.tc}


def test_roofline_traffic_is_reported_only_for_the_kernel_it_was_measured_on(tmp_path, monkeypatch):
    # which kernel a plan's contraction runs (the library's rule), and a traffic record that is used only
    # for the source it was measured on, and only while that source is unchanged
    assert bench.contract_kernel(_Tuned(0), 128, 128) == "fp32"
    assert bench.contract_kernel(_Tuned(1), 128, 128) == "fp32"  # no transposed table without the adjoint
    assert bench.contract_kernel(_Tuned(1), 128, 128, adjoint_plan=True) == "tc"
    assert bench.contract_kernel(_Tuned(1), 24, 128, adjoint_plan=True) == "fp32"  # F not a multiple of 16
    import hashlib
    import json
    src = tmp_path / "kernel.cu"
    src.write_text("// a kernel\n")
    (tmp_path / "profiles").mkdir()
    rec = {"source": "kernel.cu", "traffic_bytes_per_launch": 1234,
           "source_sha256_16": hashlib.sha256(src.read_bytes()).hexdigest()[:16]}
    (tmp_path / "profiles" / "contract_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("kernel.cu") == 1234
    assert bench.measured_traffic("other.cu") is None  # measured on another kernel
    src.write_text("// a kernel, edited\n")
    assert bench.measured_traffic("kernel.cu") is None  # the source changed since
