"""GPU tests of the batched form (a12): uneven reconstructions in one call equal
the single-reconstruction path (which the other GPU tests pin to the oracle) to
FP32 rounding of the spread's summation order,
one item is checked against the FP64 oracle directly, and the call replays
from a captured CUDA graph."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2501_05244_gb300 as nursd
from workloads import (BASE_SEED, batch_layouts_c4, batch_scenes_c4, batch_sizes_c4, device_histograms, geometry_c4,
                       relay_uniform)

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


def small_batch(sizes, N=16, F=6, Z=4, T=64, seed=3):
    pitch, center = 0.02, (0.0, 0.0)
    r = np.random.default_rng(seed)
    xys = [relay_uniform(L, N * pitch / 2 * 0.999, seed=seed + i) for i, L in enumerate(sizes)]
    hists = [r.poisson(5.0, size=(L, T)).astype(np.float32) for L in sizes]
    om = 2 * math.pi * np.linspace(3e9, 6e9, F)
    return dict(N=N, pitch=pitch, center=center, xys=xys, hists=hists, om=om, depths=np.linspace(0.3, 0.9, Z),
                T=T, t0=1e-9, dt=16e-12)


def make_plan(c, B):
    return nursd.Plan(c["N"], c["pitch"], c["center"], c["depths"], c["om"], T=c["T"], t0=c["t0"], dt=c["dt"],
                      max_points=max(max(len(x) for x in c["xys"]), 1), max_batch=B)


def test_batched_equals_single_reconstructions_and_the_oracle():
    sizes = [100, 1, 700, 0, 2049]
    c = small_batch(sizes)
    plan = make_plan(c, len(sizes))
    xys = [torch.from_numpy(x).cuda() for x in c["xys"]]
    hists = [torch.from_numpy(h).cuda() for h in c["hists"]]
    outs = plan.forward_batched(xys, hists)
    for b in range(len(sizes)):
        plan.set_points(xys[b])
        single = plan.forward(hists[b])
        if sizes[b]:
            assert rel(outs[b].cpu().numpy(), single.cpu().numpy()) < 1e-6, b
    assert float(outs[3].abs().max()) == 0.0
    P = O.temporal_dft(c["hists"][2], c["t0"], c["dt"], c["om"], np.ones(len(c["om"])))
    ref = O.nursd_forward(P, c["xys"][2], c["center"], c["pitch"], c["N"], c["depths"], c["om"])
    assert rel(outs[2].cpu().numpy(), ref) < TOL


def test_batched_call_replays_from_a_cuda_graph():
    sizes = [300, 50, 1200]
    c = small_batch(sizes, seed=9)
    plan = make_plan(c, 3)
    xys = [torch.from_numpy(x).cuda() for x in c["xys"]]
    hists = [torch.from_numpy(h).cuda() for h in c["hists"]]
    outs = [plan.empty_output() for _ in sizes]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.forward_batched(xys, hists, outs)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    ref = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.forward_batched(xys, hists, outs)
    graph.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert rel(o.cpu().numpy(), r.cpu().numpy()) < 1e-6


def test_grouped_batch_replays_from_a_cuda_graph_and_counts_launches_independent_of_b():
    sizes = [300, 50, 1200, 0, 900, 64]
    c = small_batch(sizes, seed=13)
    xys = [torch.from_numpy(x).cuda() for x in c["xys"]]
    hists = [torch.from_numpy(h).cuda() for h in c["hists"]]
    counts = []
    for B in (2, 6):
        plan = make_plan(c, 6)
        out = plan.empty_batch_output(B)
        n0 = plan.launch_count
        plan.forward_batched(xys[:B], hists[:B], list(out))
        counts.append(plan.launch_count - n0)
        torch.cuda.synchronize()
        ref = out.clone()
        out.zero_()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            plan.forward_batched(xys[:B], hists[:B], list(out))
        graph.replay()
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-6
        for b in range(B):
            plan.set_points(xys[b])
            if sizes[b]:
                assert rel(out[b].cpu().numpy(), plan.forward(hists[b]).cpu().numpy()) < 1e-6, b
    assert counts[0] == counts[1], counts


def test_batched_workload_of_64_uneven_reconstructions():
    # 64 reconstructions with L_b log-uniform in [4096, 65536], T = 512 @ 8 ps, F = 64,
    # 128^2 x 64 voxels; four items (smallest, largest, two others) against single calls.
    g = geometry_c4()
    sizes = batch_sizes_c4()
    layouts = batch_layouts_c4(sizes)
    scenes = batch_scenes_c4(len(sizes))
    om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt,
                      max_points=int(sizes.max()), max_batch=len(sizes))
    xys = [torch.from_numpy(x).cuda() for x in layouts]
    hists = [device_histograms(xys[b], *scenes[b], g.T, g.dt, g.t0, seed=BASE_SEED + 500 + b)
             for b in range(len(sizes))]
    outs = plan.forward_batched(xys, hists)
    # the batch's contraction runs on the tensor cores (tf32 head/tail products, about 2^-22 of each
    # product): 2e-6 against the FP32 single calls
    for b in {int(np.argmin(sizes)), int(np.argmax(sizes)), 7, 40}:
        plan.set_points(xys[b])
        assert rel(outs[b].cpu().numpy(), plan.forward(hists[b]).cpu().numpy()) < 2e-6, b


@pytest.mark.parametrize("grouped,group,streams,rows",
                         [(0, 6, 1, 8), (0, 6, 3, 4), (0, 6, 8, 16), (0, 6, 2, 16),
                          (1, 6, 4, 8), (1, 2, 4, 4), (1, 4, 4, 16), (1, 1, 4, 8)])
def test_batched_equals_single_calls_at_every_setting(grouped, group, streams, rows):
    # grouped: each stage one launch over `group` items at a time (outputs side by side); else the items
    # run round-robin on `streams` streams with their own workspaces; the spread's tile height changes
    # only the launch shape
    sizes = [700, 1, 0, 2049, 33, 400]
    c = small_batch(sizes, seed=11)
    plan = make_plan(c, len(sizes))
    plan.tune("batch_grouped", grouped)
    plan.tune("batch_group", group)
    plan.tune("batch_streams", streams)
    plan.tune("spread_rows", rows)
    assert plan.tuning() == {"spread_rows": rows, "batch_streams": streams, "batch_grouped": grouped,
                             "batch_group": group, "batch_tensor": 1, "contract_tc": 0}
    xys = [torch.from_numpy(x).cuda() for x in c["xys"]]
    hists = [torch.from_numpy(h).cuda() for h in c["hists"]]
    outs = plan.forward_batched(xys, hists)  # side by side
    single_plan = make_plan(c, 1)
    for b in range(len(sizes)):
        single_plan.set_points(xys[b])
        single = single_plan.forward(hists[b]).cpu().numpy()
        if sizes[b]:
            assert rel(outs[b].cpu().numpy(), single) < 1e-6, b
        else:
            assert float(outs[b].abs().max()) == 0.0
    # the plan keeps the last item's points, as a single call would
    assert rel(plan.forward(hists[-1]).cpu().numpy(), outs[-1].cpu().numpy()) < 1e-6
    assert plan.sync_status() == 0


@pytest.mark.parametrize("F,Z,B", [(8, 32, 19), (16, 64, 3), (24, 128, 17)])
def test_tensor_core_contraction_equals_the_fp32_kernel(F, Z, B):
    # the batched contraction as tf32 head/tail tensor-core products per symmetry class (16 items x 8
    # members per tile; B = 19 and 17 leave a partial item block) against the FP32 SIMT kernel, and one
    # item against the oracle
    sizes = [(37 * b) % 300 for b in range(B)]  # item 0 is empty
    c = small_batch(sizes, F=F, Z=Z, seed=20 + F)
    xys = [torch.from_numpy(x).cuda() for x in c["xys"]]
    hists = [torch.from_numpy(h).cuda() for h in c["hists"]]
    outs = {}
    for tensor in (1, 0):
        plan = make_plan(c, B)
        plan.tune("batch_tensor", tensor)
        outs[tensor] = plan.forward_batched(xys, hists)
        assert plan.sync_status() == 0
    for b in range(B):
        if sizes[b]:
            assert rel(outs[1][b].cpu().numpy(), outs[0][b].cpu().numpy()) < 2e-6, b
        else:
            assert float(outs[1][b].abs().max()) == 0.0
    k = B - 1  # a non-empty item
    P = O.temporal_dft(c["hists"][k], c["t0"], c["dt"], c["om"], np.ones(len(c["om"])))
    ref = O.nursd_forward(P, c["xys"][k], c["center"], c["pitch"], c["N"], c["depths"], c["om"])
    assert rel(outs[1][k].cpu().numpy(), ref) < TOL


def test_unsupported_tunable_values_are_refused():
    c = small_batch([10, 20])
    plan = make_plan(c, 2)
    for name, value in (("spread_rows", 6), ("batch_streams", 0), ("batch_streams", 17), ("batch_grouped", 2),
                        ("batch_group", 0), ("batch_group", 3), ("batch_tensor", 2)):
        with pytest.raises(nursd.NursdError) as err:
            plan.tune(name, value)
        assert err.value.status == nursd.nursd.NURSD_ERR_UNSUPPORTED


def test_autotuner_keeps_the_results_and_caches_its_choice(tmp_path):
    from paper_2501_05244_gb300.autotune import autotune

    sizes = [300, 50, 1200, 800]
    c = small_batch(sizes, seed=12)
    plan = make_plan(c, len(sizes))
    xys = [torch.from_numpy(x).cuda() for x in c["xys"]]
    hists = [torch.from_numpy(h).cuda() for h in c["hists"]]
    outs = [plan.empty_output() for _ in sizes]
    plan.forward_batched(xys, hists, outs)
    ref = [o.cpu().numpy() for o in outs]
    path = str(tmp_path / "tune.json")
    r = autotune(plan, lambda: plan.forward_batched(xys, hists, outs), workload="test", cache_path=path, reps=2)
    assert not r["cached"] and r["choice"]["spread_rows"] in (4, 8, 16) and 1 <= r["choice"]["batch_streams"] <= 16
    plan.forward_batched(xys, hists, outs)
    for o, want in zip(outs, ref):
        assert rel(o.cpu().numpy(), want) < 1e-6
    plan2 = make_plan(c, len(sizes))
    r2 = autotune(plan2, lambda: None, workload="test", cache_path=path)
    assert r2["cached"] and {k: plan2.tuning()[k] for k in r["choice"]} == r["choice"]
