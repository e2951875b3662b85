"""Failure paths on the GPU, made on the host or by a bounded wait that runs out; nothing here faults,
traps or hangs a GPU.

* A device allocation made to fail by the library's test hook: plan creation returns NURSD_ERR_OOM,
  releases everything it had allocated (device free memory returns to its level), and the next plan
  works.
* The bulk-copy contraction's data waits given a bound of zero polls by the test hook: they run out,
  each warp records the time-out, lets its own copies land (with the default bound) and returns;
  nursd_sync_status reports NURSD_ERR_TIMEOUT, and with the default bound restored the next call is
  correct again.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import random_phasors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    nursd.build()
    nursd.load_library()
    yield
    lib = nursd.load_library()
    lib.nursd_test_fail_allocation(0)
    lib.nursd_test_set_wait_limit(-1, None)
    torch.cuda.synchronize()


def big_plan_args():
    # about 0.7 GB of plan memory: a leaked table or workspace would show in the free-memory count
    N, F, Z = 256, 64, 32
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    return (N, 2.0 / N, (0.0, 0.0), np.linspace(0.5, 2.0, Z), om), dict(T=64, t0=1e-9, dt=8e-12, max_points=4096,
                                                                        adjoint=True)


def test_injected_allocation_failures_return_oom_and_leak_nothing():
    lib = nursd.load_library()
    args, kw = big_plan_args()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for after in (1, 2, 7, 20, 30):
        lib.nursd_test_fail_allocation(after)
        try:
            plan = nursd.Plan(*args, **kw)
        except nursd.NursdError as err:
            assert err.status == nursd.nursd.NURSD_ERR_OOM, after
        else:  # the plan needed fewer allocations than `after`: the hook stays armed, disarm it
            plan.close()
        lib.nursd_test_fail_allocation(0)
        torch.cuda.synchronize()
        assert abs(torch.cuda.mem_get_info()[0] - free0) < 32 << 20, after
    plan = nursd.Plan(*args, **kw)  # the context and the library still work
    assert plan.nbytes > 0
    plan.close()


def test_a_contraction_wait_that_runs_out_reports_timeout_and_the_next_call_recovers():
    lib = nursd.load_library()
    # F % 4 == 0 and Z == 64 select the bulk-copy form of the contraction
    N, L, F, Z, pitch = 32, 800, 16, 64, 0.02
    r = np.random.default_rng(9)
    xy = (r.uniform(-0.3, 0.3, (L, 2))).astype(np.float32)
    P = random_phasors(L, F, seed=10)
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    depths = np.linspace(0.3, 0.9, Z)
    plan = nursd.Plan(N, pitch, (0.0, 0.0), depths, om, max_points=L)
    plan.set_points(torch.from_numpy(xy).cuda())
    Pg = torch.from_numpy(P).cuda()
    good = plan.forward_phasor(Pg).cpu().numpy()
    assert plan.sync_status() == 0
    assert lib.nursd_test_set_wait_limit(0, None) == 0  # every data wait gives up at once
    plan.forward_phasor(Pg)
    assert plan.sync_status() == nursd.nursd.NURSD_ERR_TIMEOUT
    assert lib.nursd_test_set_wait_limit(-1, None) == 0
    again = plan.forward_phasor(Pg).cpu().numpy()
    assert plan.sync_status() == 0
    assert np.array_equal(again, good)
    ref = O.nursd_forward(P, xy, (0.0, 0.0), pitch, N, depths, om)
    assert np.linalg.norm(again - ref) / np.linalg.norm(ref) < 1e-4
