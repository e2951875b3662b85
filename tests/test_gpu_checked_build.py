"""The checked build (libnursd_checked.so, -DNURSD_CHECKED): every data-dependent index check compiled
in, a failed check reported as NURSD_ERR_CUDA through the status word with the access skipped.  The
same calls through it and through the normal library give the same results and a clean status."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import importlib

nbuild = importlib.import_module("paper_2501_05244_gb300.build")  # the module (the package exports its build())

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the calls, run in a process of its own with the library given on the command line
SCRIPT = r"""
import sys
import numpy as np, torch
from paper_2501_05244_gb300 import nursd as binding
binding.load_library(sys.argv[1])
import paper_2501_05244_gb300 as nursd
from workloads import BASE_SEED, workload_c1, random_phasors
wl = workload_c1(); g = wl.geom
om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=len(wl.xy),
                  max_batch=3, adjoint=True, srsd_pitch=np.linspace(1.0, 2.0, g.Z) * g.pitch)
xy = torch.from_numpy(wl.xy).cuda(); h = torch.from_numpy(wl.hist).cuda()
out = {"forward": plan.reconstruct(xy, h)}
outs = plan.forward_batched([xy, xy[:500], xy[:77]], [h, h[:500], h[:77]])
for b, o in enumerate(outs):
    out["batch%d" % b] = o
plan.set_points(xy)
P = torch.from_numpy(random_phasors(len(wl.xy), g.F, seed=BASE_SEED + 150)).cuda()
out["srsd"] = plan.srsd_forward(P)
out["adjoint"] = plan.adjoint(out["forward"])
assert plan.sync_status() == 0
np.savez(sys.argv[2], **{k: v.cpu().numpy() for k, v in out.items()})
"""


def run(lib, path):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", SCRIPT, lib, path], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(path)


def test_checked_build_gives_the_same_results_and_a_clean_status(tmp_path):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    normal = nbuild.build()
    checked = nbuild.build(checked=True)
    assert checked != normal and os.path.exists(checked)
    a = run(normal, str(tmp_path / "normal.npz"))
    b = run(checked, str(tmp_path / "checked.npz"))
    assert set(a.files) == set(b.files)
    for k in a.files:
        x, y = a[k].astype(np.complex128).ravel(), b[k].astype(np.complex128).ravel()
        assert np.linalg.norm(x - y) <= 1e-6 * max(np.linalg.norm(x), 1e-30), k
