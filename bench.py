#!/usr/bin/env python
"""Benchmark of the NURSD-1 forward on GB300 (one JSON line on stdout).

Workload (one step = one reconstruction): 65,536 keystone relay samples
(16x16 illumination spots x 16x16 SPAD pixels through a pinhole onto a
2 m x 2 m plane tilted 20 deg), 1,024-bin histograms at 4 ps, 128 phasor
frequencies, 256 x 256 x 128 voxels over 0.5-3 m.  A step is the whole path:
relay-sample preparation and sort, temporal transform, NUFFT type 1 (spread,
FFTs, deconvolution), transfer-function multiply with the frequency sum,
inverse FFT and crop.  Inputs are seeded synthetic data resident in HBM; the
histograms (268 MB) and the transfer-function table (4.35 GB) are larger than
L2, so no flush is needed between steps.

``--impl reference`` times the FP64 CPU oracle (direct back-projection) on the
host cores instead, each step a bounded voxel sample of the same workload.
"""
from __future__ import annotations

import argparse
import math
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NURSD voxel·freq/sec and recon/sec at 65k relay samples → 256²×128 voxels; fraction of HBM BW"
UNIT = "voxel*freq/s"
WORKLOAD = ("spad-65k: 65,536 keystone relay samples, T=1024 bins @ 4 ps, F=128 frequencies "
            "-> 256x256x128 voxels over 0.5-3 m (NUFFT sigma=2, ES width 6)")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--no-graph", action="store_true", help="time eager steps instead of a captured CUDA graph")
    ap.add_argument("--shard", choices=["replicas", "depth"], default="replicas",
                    help="replicas: one reconstruction per GPU (weak scaling); depth: one reconstruction whose "
                         "depth planes are split over the GPUs and gathered (strong scaling)")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the per-row measurements (type-2 voxels, SRSD, adjoint, gradients, batched)")
    ap.add_argument("--rows", default="",
                    help="comma-separated names of the rows to measure (default: every row); given, the rows run "
                         "with any --workload")
    ap.add_argument("--row-depths", type=int, default=128,
                    help="depth planes of the scaled-plane rows (SRSD, NU-SFFT, SRSD at voxels); 128 is the "
                         "measured workload, fewer make a small case for profiler captures")
    ap.add_argument("--row-items", type=int, default=64,
                    help="reconstructions of the batched row (the first of its 64 items); 64 is the measured "
                         "workload, fewer make a small case for profiler captures")
    ap.add_argument("--workload", choices=["spad", "grid128", "spad-z8", "spad-n128"], default="spad",
                    help="spad: the 65k-sample 256^2x128 workload (the metric); grid128: the same samples on "
                         "128^2x64 voxels; spad-z8: the spad workload with 8 of its 128 depth planes (same "
                         "spread and FFT launches, 1/16 of the table); spad-n128: the spad workload on "
                         "128^2x128 voxels (same contraction kernel, 1/4 of the table); the last three are "
                         "small cases for profiler captures")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, dist, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job rate: every rank processes `units_per_rank` in the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


CONTRACT_KERNELS = {
    "tc": ("contract_tc_kernel (tensor cores: tf32 head/tail products, table as the A operand by TMA)",
           "paper_2501_05244_gb300/csrc/contract_tc.cu"),
    "fp32": ("contract_tma_kernel (FP32 packed FMAs, bulk-copy rings)", "paper_2501_05244_gb300/csrc/contract.cu"),
}


def contract_kernel(plan, F, Z, adjoint_plan=False):
    """Key of CONTRACT_KERNELS for the kernel a plan's forward contraction runs (the library's rule:
    the tensor form when tuned on, on a plan with the adjoint enabled, Z = 128 rows and F a multiple
    of 16 up to 208)."""
    ok = plan.tuning()["contract_tc"] == 1 and adjoint_plan and Z == 128 and F % 16 == 0 and 16 <= F <= 208
    return "tc" if ok else "fp32"


def measured_traffic(source):
    """Per-launch DRAM traffic of the contraction from the recorded ncu counters
    (profiles/contract_traffic.json), or None when they were taken on another kernel or its source
    changed since."""
    import hashlib

    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "contract_traffic.json")))
        if rec["source"] != source:
            return None
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except (OSError, ValueError, KeyError):
        return None
    if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha256_16"):
        return None
    return int(rec["traffic_bytes_per_launch"])


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [l.strip().split(",") for l in self.tmp.read().splitlines() if l.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU side ---
# The FP64 oracle runs on every host core: a pool of single-threaded worker processes (spawned,
# so that no worker inherits a CUDA context), each back-projecting its own block of voxels.

_POOL_STATE = {}


def _oracle_worker_init(path_p, path_xy, path_om):
    import numpy as np

    _POOL_STATE["P"] = np.load(path_p)
    _POOL_STATE["xy"] = np.load(path_xy)
    _POOL_STATE["om"] = np.load(path_om)


def _oracle_worker_fbp(task):
    """Direct back-projection of one voxel block over frequency slice [f0, f1) (returns the count)."""
    import numpy as np

    import oracle as O

    vox, f0, f1 = task
    O.fbp_direct(_POOL_STATE["P"][:, f0:f1], _POOL_STATE["xy"], _POOL_STATE["om"][f0:f1], vox)
    return vox.shape[0] * (f1 - f0)


class OraclePool:
    """os.cpu_count() spawned single-threaded processes sharing the phasors through .npy files."""

    def __init__(self, P, xy, omega):
        import multiprocessing as mp
        import numpy as np

        self.dir = tempfile.mkdtemp(prefix="nursd_oracle_")
        paths = [os.path.join(self.dir, n) for n in ("P.npy", "xy.npy", "om.npy")]
        for path, arr in zip(paths, (P, xy, omega)):
            np.save(path, np.ascontiguousarray(arr))
        self.cores = os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init, initargs=paths)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.pool.map(_oracle_worker_fbp, [(np.zeros((1, 3)) + [0.0, 0.0, 1.0], 0, 1)] * self.cores)  # warm up

    def run(self, tasks):
        return sum(self.pool.map(_oracle_worker_fbp, tasks, chunksize=1))

    def close(self):
        import shutil

        self.pool.terminate()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def _random_voxels(g, n, rng):
    import numpy as np

    m = rng.integers(0, g.N, size=(n, 2))
    z = g.depths[rng.integers(0, g.Z, n)]
    return np.stack([(m[:, 0] - g.N // 2) * g.pitch, (m[:, 1] - g.N // 2) * g.pitch, z], axis=1)


def oracle_rate(wl, seconds: float, rng_seed: int = 7):
    """Time the FP64 oracle (direct back-projection) on a bounded voxel sample on all host cores.

    Returns (voxel*freq/s, description, cores).  The oracle's temporal transform of all histograms
    is timed too and charged pro rata to the sampled voxels' share of the full volume.
    """
    import numpy as np

    import oracle as O

    g = wl.geom
    om, wt = O.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    t0 = time.perf_counter()
    P = O.temporal_dft(wl.hist, g.t0, g.dt, om, wt)
    t_temporal = time.perf_counter() - t0
    rng = np.random.default_rng(rng_seed)
    pool = OraclePool(P, wl.xy, om)
    try:
        # cost of one voxel x all frequencies on one worker, then one voxel block per worker task
        t0 = time.perf_counter()
        pool.run([(_random_voxels(g, 1, rng), 0, g.F)])
        per_voxel = time.perf_counter() - t0
        per_task = max(1, int(2.0 / max(per_voxel, 1e-6)))
        ntask = max(pool.cores, int(seconds * pool.cores / max(per_voxel * per_task, 1e-6)))
        tasks = [(_random_voxels(g, per_task, rng), 0, g.F) for _ in range(ntask)]
        t0 = time.perf_counter()
        units = pool.run(tasks)
        t_fbp = time.perf_counter() - t0
    finally:
        pool.close()
    nvox = units // g.F
    full = g.Z * g.N * g.N
    t = t_fbp + t_temporal * nvox / full
    desc = (f"oracle.fbp_direct (FP64 NumPy direct back-projection) of {nvox} random voxels x {g.F} frequencies "
            f"over all {len(wl.xy)} relay samples on {pool.cores} single-threaded worker processes "
            f"({t_fbp:.1f} s) + oracle.temporal_dft of all histograms ({t_temporal:.1f} s, charged pro rata "
            f"{nvox}/{full})")
    return units / t, desc, pool.cores


# The same fast algorithm in FP64 on the host (a secondary, fairer CPU baseline than direct
# back-projection): ES spread as a sparse matrix, the oversampled 2D FFT (scipy.fft on every core),
# deconvolution and truncation, the transfer-function multiply with the frequency sum (z blocks on a
# thread pool), and one inverse FFT with crop per depth.  It is timed on a sample of the frequencies;
# the per-frequency stages are scaled to all F, the per-depth inverse FFTs are timed in full.

def _es_psi_hat(k, w: int, beta: float, nf: int, nodes: int = 200):
    """Fourier transform of the ES kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) spread over w
    fine cells, at integer frequencies k of an nf-point grid (Gauss-Legendre quadrature)."""
    import numpy as np

    z, wq = np.polynomial.legendre.leggauss(nodes)
    phi = np.exp(beta * (np.sqrt(1.0 - z * z) - 1.0))
    return (w / 2.0) * (np.cos(np.pi * np.outer(k, z) * w / nf) @ (wq * phi))


class CpuFastPlan:
    """Plan-time tables of the FP64 host run: spread matrix, deconvolution, transfer functions."""

    def __init__(self, xy, N, pitch, center, depths, omega, freqs, width=6):
        import numpy as np
        import scipy.sparse as sp

        self.N, self.M, self.nf, self.w = N, 2 * N, 4 * N, width
        self.depths, self.omega, self.freqs = np.asarray(depths, float), np.asarray(omega, float), list(freqs)
        M, nf, w = self.M, self.nf, width
        beta = 2.30 * w
        t0 = time.perf_counter()
        u = (np.asarray(xy, np.float64) - np.asarray(center, np.float64)[None, :]) * (2.0 / pitch)
        i0 = np.ceil(u - 0.5 * w).astype(np.int64)
        taps = np.arange(w)
        zz = 2.0 * (i0[:, :, None] + taps[None, None, :] - u[:, :, None]) / w  # [L][2][w]
        wt = np.where(np.abs(zz) < 1.0, np.exp(beta * (np.sqrt(np.maximum(1.0 - zz * zz, 0.0)) - 1.0)), 0.0)
        gx = (i0[:, 0, None] + taps[None, :]) % nf
        gy = (i0[:, 1, None] + taps[None, :]) % nf
        rows = (gy[:, :, None] * nf + gx[:, None, :]).reshape(len(u), -1)
        vals = (wt[:, 1, :, None] * wt[:, 0, None, :]).reshape(len(u), -1)
        cols = np.repeat(np.arange(len(u)), w * w)
        self.S = sp.csr_matrix((vals.ravel(), (rows.ravel(), cols)), shape=(nf * nf, len(u)))
        self.t_points = time.perf_counter() - t0
        k = np.fft.fftfreq(M, 1.0 / M)  # k in FFT order
        ph = _es_psi_hat(k, w, beta, nf)
        self.deconv = 1.0 / np.outer(ph, ph)
        self.kidx = np.asarray(k, np.int64) % nf  # fine-grid bins kept
        j = np.fft.fftfreq(M, 1.0 / M) * pitch  # offsets j delta in FFT order
        r2 = j[None, :] ** 2 + j[:, None] ** 2
        C = 299792458.0
        self.G = np.empty((len(self.depths), len(self.freqs), M, M), np.complex128)
        for iz, z in enumerate(self.depths):
            r = np.sqrt(r2 + z * z)
            for i, f in enumerate(self.freqs):
                self.G[iz, i] = np.fft.fft2(np.exp(1j * self.omega[f] / C * r) / r)

    def forward(self, P, workers):
        """V[z][my][mx] summed over the plan's frequencies, and the stage times (s)."""
        import concurrent.futures as cf

        import numpy as np
        import scipy.fft as sfft

        M, N, nf, Z = self.M, self.N, self.nf, len(self.depths)
        t = dict(spread=0.0, fft=0.0, deconv=0.0, contract=0.0, ifft=0.0)
        Y = np.zeros((Z, M, M), np.complex128)
        blocks = [slice(z0, min(Z, z0 + max(1, Z // workers))) for z0 in range(0, Z, max(1, Z // workers))]
        with cf.ThreadPoolExecutor(workers) as ex:
            for i, f in enumerate(self.freqs):
                t0 = time.perf_counter()
                fine = (self.S @ np.asarray(P[:, f], np.complex128)).reshape(nf, nf)
                t1 = time.perf_counter()
                bh = sfft.fft2(fine, workers=workers)
                t2 = time.perf_counter()
                U = bh[np.ix_(self.kidx, self.kidx)] * self.deconv
                t3 = time.perf_counter()

                def mac(b, U=U, i=i):
                    Y[b] += U[None] * self.G[b, i]

                list(ex.map(mac, blocks))
                t4 = time.perf_counter()
                t["spread"] += t1 - t0
                t["fft"] += t2 - t1
                t["deconv"] += t3 - t2
                t["contract"] += t4 - t3
        t0 = time.perf_counter()
        v = sfft.ifft2(Y, axes=(-2, -1), workers=workers)
        m = np.arange(-N // 2, N // 2) % M
        V = v[:, m][:, :, m]
        t["ifft"] = time.perf_counter() - t0
        return V, t


def cpu_fast_rate(wl, n_freq: int = 2):
    """FP64 host run of the fast algorithm on all cores, per reconstruction: the temporal transform
    and point preparation in full, the per-frequency stages on n_freq frequencies scaled to F, the
    per-depth inverse FFTs in full.  Returns a row dict."""
    import numpy as np

    g = wl.geom
    workers = os.cpu_count() or 1
    C = 299792458.0
    f_c = C / g.lambda_c
    f0 = math.floor(f_c * g.t_pad * g.dt + 0.5) - g.F // 2
    omega = 2 * math.pi * (f0 + np.arange(g.F)) / (g.t_pad * g.dt)
    wt = np.exp(-((omega - 2 * math.pi * f_c) ** 2) / (2 * (2 * math.pi * f_c / 5) ** 2))
    t0 = time.perf_counter()
    tn = g.t0 + g.dt * np.arange(g.T)
    P = (np.asarray(wl.hist, np.float64) @ np.exp(-1j * np.outer(tn, omega))) * wt[None, :]
    t_temporal = time.perf_counter() - t0
    freqs = list(np.linspace(0, g.F - 1, n_freq).round().astype(int))
    plan = CpuFastPlan(wl.xy, g.N, g.pitch, g.center, g.depths, omega, freqs)
    _, st = plan.forward(P, workers)
    per_f = st["spread"] + st["fft"] + st["deconv"] + st["contract"]
    t = t_temporal + plan.t_points + per_f * g.F / n_freq + st["ifft"]
    units = g.Z * g.N * g.N * g.F
    return {"value": units / t, "unit": UNIT, "cores": workers, "dtype": "f64", "s_per_reconstruction": t,
            "stages_s": {"temporal": t_temporal, "points": plan.t_points,
                         **{k: (v * g.F / n_freq if k != "ifft" else v) for k, v in st.items()}},
            "sample": f"NumPy/SciPy FP64 fast algorithm (sparse ES spread, scipy.fft with workers={workers}, "
                      f"contraction over a {workers}-thread pool); {n_freq} of {g.F} frequencies timed and "
                      f"scaled, temporal transform, point preparation and the {g.Z} inverse FFTs timed in full; "
                      f"transfer-function tables built outside the timing"}


# ---------------------------------------------------------------- GPU side ---

def _time(fn, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _stage_ms(plan, calls):
    """Per-call stage times (ms) over the `calls` calls made since profiling was enabled; a stage
    that runs as several launches per call (channel or depth groups) is summed over them."""
    return {k: v[0] / calls for k, v in plan.profile_read().items() if v[1]}


def fine_window(N: int, w: int = 6) -> int:
    """Width of the fine-grid window the spread writes (16-cell tiles covering every footprint)."""
    return (2 * N + w + 2 + 15) // 16 * 16


def n_classes(N: int) -> int:
    """8-fold symmetry classes of the transfer function on the M = 2N grid."""
    return (N + 1) * (N + 2) // 2


def bytes_type1(L: int, F: int, N: int) -> int:
    """Spread (phasors in, window out), FFT along x (window in, rows out), FFT along y with
    deconvolution (rows in, spectrum out): complex64 bytes."""
    M, W = 2 * N, fine_window(N)
    return 8 * (L * F + W * W * F + W * W * F + W * M * F + W * M * F + M * M * F)


def bytes_contract(F: int, Z: int, N: int) -> int:
    """Table once, spectrum in, depth spectra out."""
    M = 2 * N
    return 8 * (n_classes(N) * F * Z + M * M * F + M * M * Z)


def bytes_idft(Z: int, N: int, mag: bool = False) -> int:
    """Two pruned inverse passes: Y in, half inverse out and in, volume out."""
    M = 2 * N
    return 8 * (M * M * Z + 2 * M * N * Z) + (4 if mag else 8) * N * N * Z


def bytes_type2_fine(C: int, N: int) -> int:
    """Spectrum [M][M][C] in, rows [M][W][C] out and in, fine window [W][W][C] out."""
    M, W = 2 * N, fine_window(N)
    return 8 * (M * M * C + 2 * M * W * C + W * W * C)


def bytes_adjoint_spectrum(F: int, Z: int, N: int) -> int:
    """Volume in, half transform out and in, depth spectra out and in, table in, spectrum out."""
    M = 2 * N
    return 8 * (N * N * Z + 2 * N * M * Z + 2 * M * M * Z + n_classes(N) * Z * F + M * M * F)


def bytes_srsd(N: int, F: int, scales, w: int = 6) -> int:
    """SRSD spectra by interpolation of one oversampled spectrum: the gridded input (spectrum in, u
    out and back in), the shared oversampled spectrum (half-transformed rows written and read, the
    [2M][2M] spectrum written), and per depth the spectrum block its taps reach, its table and Y_z."""
    M = 2 * N
    Lg = 2 * M
    b = (3 * M * M + 2 * M * Lg + Lg * Lg) * F * 8
    for sc in scales:
        R = (math.ceil(2.0 * (M // 2 - 1) / sc - 0.5 * w) + w - 1) - math.ceil(2.0 * (-M // 2) / sc - 0.5 * w) + 1
        b += (R * R * F + n_classes(N) * F + M * M) * 8
    return b


def bytes_nusfft(L: int, N: int, F: int, scales, w: int = 6) -> int:
    """NU-SFFT spectra: spread (phasors in, window out), the window's rows transformed to 2M bins (in,
    out), the columns to the 2M x 2M spectrum (in, out), and per depth the spectrum block its taps
    reach (coordinates kappa / s on the 2M grid), its table and Y_z."""
    M, W = 2 * N, fine_window(N)
    Lg = 2 * M
    b = 8 * (L * F + W * W * F + W * W * F + W * Lg * F + W * Lg * F + Lg * Lg * F)
    for sc in scales:
        R = (math.ceil((M // 2 - 1) / sc - 0.5 * w) + w - 1) - math.ceil((-M // 2) / sc - 0.5 * w) + 1
        b += (R * R * F + n_classes(N) * F + M * M) * 8
    return b


def hbm_row(bytes_: int, ms: float, peak: float) -> dict:
    gbs = bytes_ / (ms / 1e3) / 1e9
    return {"algorithmic_bytes": int(bytes_), "achieved_gbs": gbs, "hbm_frac": gbs / peak}


def measure_rows(wl, peak, stages_ms=None, only=(), row_depths=128, row_items=64):
    """Per-row measurements of the other hot-path rows on the same GPU (one entry each)."""
    import numpy as np
    import torch

    import paper_2501_05244_gb300 as nursd
    from workloads import (BASE_SEED, batch_layouts_c4, batch_scenes_c4, batch_sizes_c4, device_histograms,
                           geometry_c4, random_phasors, random_plane_points, relay_keystone, srsd_depths_c3b,
                           srsd_pitches_c3b)

    stream = torch.cuda.current_stream()
    rows = {}
    g = wl.geom
    om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    L = len(wl.xy)
    d_xy = torch.from_numpy(wl.xy).cuda()
    d_hist = torch.from_numpy(wl.hist).cuda()

    def guarded(name, fn):
        if only and name not in only:
            return
        try:
            rows[name] = fn()
        except Exception as exc:  # a failing row is reported, not fatal to the headline line
            rows[name] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    def type2():
        plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=L)
        plan.set_points(d_xy)
        P = plan.temporal_dft(d_hist)
        K = 16384
        vox = torch.from_numpy(random_plane_points(g.Z, K, 0.999, seed=BASE_SEED + 30)).cuda()
        out = torch.empty((g.Z, K), dtype=torch.complex64, device="cuda")
        plan.profile(True)
        ms = _time(lambda: plan.forward_points(P, vox, out), 10, 2, stream)
        st = _stage_ms(plan, 12)
        assert plan.sync_status() == 0
        plan.close()
        units = g.Z * K * g.F
        W = fine_window(g.N)
        b = (bytes_type1(L, g.F, g.N) + bytes_contract(g.F, g.Z, g.N) + bytes_type2_fine(g.Z, g.N)
             + 8 * (W * W * g.Z + 2 * g.Z * K))  # plane windows in, voxel positions in, values out
        return {"workload": "65,536 keystone samples -> 128 planes x 16,384 random voxels (2,097,152), F=128",
                "ms": ms, "voxel_freq_per_s": units / (ms / 1e3), **hbm_row(b, ms, peak), "stages_ms": st}

    def srsd():
        depths = srsd_depths_c3b(row_depths)
        plan = nursd.Plan(g.N, g.pitch, g.center, depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=L,
                          srsd_pitch=srsd_pitches_c3b(depths))
        plan.set_points(d_xy)
        P = plan.temporal_dft(d_hist)
        out = plan.empty_output()
        plan.profile(True)
        ms = _time(lambda: plan.srsd_forward(P, out), 3, 1, stream)
        prof = plan.profile_read()  # 4 calls: the warm-up and the 3 timed
        plan.close()
        F, Z = g.F, len(depths)
        s_ms = prof["srsd"][0] / 4
        scales = srsd_pitches_c3b(depths) / g.pitch  # all >= 1: every depth is interpolated
        bytes_ = bytes_srsd(g.N, F, scales)
        call_bytes = bytes_type1(L, F, g.N) + bytes_ + bytes_idft(Z, g.N)
        units = Z * g.N * g.N * F
        return {"workload": f"65,536 keystone samples -> 256^2 x {Z} planes over 1-4 m, pitch 8 -> 32 mm, F=128",
                "ms": ms, "voxel_freq_per_s": units / (ms / 1e3), **hbm_row(call_bytes, ms, peak),
                "srsd_stage": {"ms": s_ms, "algorithmic_bytes": bytes_, "achieved_gbs": bytes_ / (s_ms / 1e3) / 1e9,
                               "hbm_frac": bytes_ / (s_ms / 1e3) / 1e9 / peak,
                               "method": "scaled DFT by ES interpolation of one oversampled spectrum"},
                "stages_ms": {k: v[0] / 4 for k, v in prof.items() if v[1]}}

    def adjoint():
        plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, max_points=L, adjoint=True)
        plan.set_points(d_xy)
        r = np.random.default_rng(5)
        V = torch.from_numpy((r.standard_normal((g.Z, g.N, g.N)) + 1j * r.standard_normal((g.Z, g.N, g.N)))
                             .astype(np.complex64)).cuda()
        out = torch.empty((L, g.F), dtype=torch.complex64, device="cuda")
        plan.profile(True)
        ms = _time(lambda: plan.adjoint(V, out), 10, 2, stream)
        st = _stage_ms(plan, 12)
        plan.close()
        units = g.Z * g.N * g.N * g.F
        W = fine_window(g.N)
        b = (bytes_adjoint_spectrum(g.F, g.Z, g.N) + bytes_type2_fine(g.F, g.N)
             + 8 * (W * W * g.F + L * g.F))  # window in, phasors out
        return {"workload": "spad-65k adjoint: 256^2 x 128 volume -> 65,536 x 128 phasors", "ms": ms,
                "voxel_freq_per_s": units / (ms / 1e3), **hbm_row(b, ms, peak), "stages_ms": st}

    def grad():
        N, Z, F = 128, 64, 128
        xy = relay_keystone(seed=BASE_SEED + 5)
        depths = np.linspace(0.5, 3.0, Z)
        plan = nursd.Plan(N, 2.0 / N, (0.0, 0.0), depths, om, wt, max_points=len(xy), adjoint=True)
        dxy = torch.from_numpy(xy).cuda()
        P = torch.from_numpy(random_phasors(len(xy), F, seed=BASE_SEED + 6)).cuda()
        Vt = torch.zeros((Z, N, N), dtype=torch.complex64, device="cuda")

        def step():  # loss = ||A(P, x) - V_t||^2: forward, then both gradients
            plan.set_points(dxy)
            V = plan.forward_phasor(P)
            plan.grad_points(2 * (V - Vt), P)

        plan.profile(True)
        ms = _time(step, 10, 2, stream)
        st = _stage_ms(plan, 12)
        plan.close()
        Lg, W = len(xy), fine_window(N)
        b = (bytes_type1(Lg, F, N) + bytes_contract(F, Z, N) + bytes_idft(Z, N)  # forward
             + bytes_adjoint_spectrum(F, Z, N) + 3 * bytes_type2_fine(F, N)  # R, kx R, ky R on the window
             + 8 * (3 * W * W * F + 2 * Lg * F + Lg))  # three windows and P in, grad P and grad x out
        return {"workload": "65,536 keystone samples, F=128, 128^2 x 64: forward + gradients w.r.t. phasors "
                            "and positions", "ms": ms, **hbm_row(b, ms, peak),
                "bytes_exclude": "the residual 2 (V - V_t) formed by torch between the two calls",
                "stages_ms": st}

    def illuminated():
        # next row 1: one illumination point's phase mask per voxel and frequency (Eq. PF_RSD_Defn),
        # and transient frames (Eq. Video_Voxel_Freq_Offset); both keep every frequency's volume
        plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=L)
        plan.set_points(d_xy)
        P = plan.temporal_dft(d_hist)
        out = torch.empty((g.Z, g.N, g.N), dtype=torch.complex64, device="cuda")
        xp = (0.0, 0.0, 0.0)  # the aperture centre
        plan.profile(True)
        ms = _time(lambda: plan.forward_illuminated(P, xp, out=out), 3, 1, stream)
        st = _stage_ms(plan, 4)
        plan.profile(False)
        nt = 16
        times = g.t0 + np.linspace(0.0, 4e-9, nt)
        frames = torch.empty((nt, g.Z, g.N, g.N), dtype=torch.complex64, device="cuda")
        ms_f = _time(lambda: plan.transient_frames(P, times, out=frames), 3, 1, stream)
        assert plan.sync_status() == 0
        M, F, Z, N = 2 * g.N, g.F, g.Z, g.N
        ncls = (M // 2 + 1) * (M // 2 + 2) // 2
        fused = Z % 4 == 0 and F % 2 == 0 and M in (512, 1024)  # products formed inside the kx pass
        zg = 4 if fused else min(Z, max(1, 512 // F))
        # per group of zg depths (C = zg F channels): spectrum + zg table values per class and f in,
        # the half inverse and per-frequency volumes (and, unfused, the products) each written and
        # read once, volume out
        per_group = lambda zn: (M * M * F + ncls * F * zn + (0 if fused else 2 * M * M * zn * F)
                                + 2 * M * N * zn * F + 2 * N * N * zn * F + N * N * zn) * 8
        groups = [min(zg, Z - z0) for z0 in range(0, Z, zg)]
        bytes_pf = sum(per_group(zn) for zn in groups)
        units = Z * N * N * F
        return {"workload": "65,536 keystone samples -> 256^2 x 128, F=128: single illumination at the aperture "
                            "centre; and 16 transient frames over 4 ns",
                "ms": ms, "voxel_freq_per_s": units / (ms / 1e3), "ms_16_frames": ms_f,
                "per_frequency_stages": {"algorithmic_bytes": bytes_pf,
                                         "ms": ms - st.get("spread", 0) - st.get("fft_x", 0) - st.get("fft_y", 0),
                                         "depth_group": zg, "products_in_kx_pass": fused},
                **hbm_row(bytes_type1(L, F, N) + bytes_pf, ms, peak), "stages_ms": st}

    def srsd_points():
        # next row 2: SRSD + NURSD-2 (Eq. NURSD2_SRSD), 16,384 random voxels in each plane's scaled aperture
        depths = srsd_depths_c3b(row_depths)
        pitches = srsd_pitches_c3b(depths)
        plan = nursd.Plan(g.N, g.pitch, g.center, depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=L,
                          srsd_pitch=pitches)
        plan.set_points(d_xy)
        P = plan.temporal_dft(d_hist)
        K = 16384
        unit = random_plane_points(len(depths), K, 0.999, seed=BASE_SEED + 31)  # [Z][K][2] in a unit half-extent
        vox = torch.from_numpy((unit * (0.5 * g.N * pitches)[:, None, None]).astype(np.float32)).cuda()
        out = torch.empty((len(depths), K), dtype=torch.complex64, device="cuda")
        ms = _time(lambda: plan.srsd_forward_points(P, vox, out=out), 3, 1, stream)
        assert plan.sync_status() == 0
        plan.close()
        Z, W = len(depths), fine_window(g.N)
        b = (bytes_type1(L, g.F, g.N) + bytes_srsd(g.N, g.F, pitches / g.pitch) + bytes_type2_fine(Z, g.N)
             + 8 * (W * W * Z + 2 * Z * K))
        return {"workload": f"65,536 keystone samples -> {Z} scaled planes over 1-4 m (pitch 8 -> 32 mm) x 16,384 "
                            "random voxels each, F=128",
                "ms": ms, "voxel_freq_per_s": len(depths) * K * g.F / (ms / 1e3), **hbm_row(b, ms, peak)}

    def batched():
        gb = geometry_c4()
        all_sizes = batch_sizes_c4()
        layouts = batch_layouts_c4(all_sizes)[:row_items]
        scenes = batch_scenes_c4(len(all_sizes))[:row_items]
        sizes = all_sizes[:row_items]
        omb, wtb = nursd.phasor_frequencies(gb.lambda_c, gb.dt, gb.t_pad, gb.F)
        plan = nursd.Plan(gb.N, gb.pitch, gb.center, gb.depths, omb, wtb, T=gb.T, t0=gb.t0, dt=gb.dt,
                          max_points=int(sizes.max()), max_batch=len(sizes))
        xys = [torch.from_numpy(x).cuda() for x in layouts]
        hists = [device_histograms(xys[b], *scenes[b], gb.T, gb.dt, gb.t0, seed=BASE_SEED + 500 + b)
                 for b in range(len(sizes))]
        outs = list(plan.empty_batch_output(len(sizes)))  # side by side: the grouped launches
        from paper_2501_05244_gb300.autotune import autotune

        tuned = autotune(plan, lambda: plan.forward_batched(xys, hists, outs), workload="64 items, L 4096-65536",
                         cache_path=os.path.join(tempfile.gettempdir(), f"nursd_tune_{os.getpid()}.json"),
                         use_cache=False, reps=3)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            plan.forward_batched(xys, hists, outs)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            plan.forward_batched(xys, hists, outs)
        ms_graph = _time(graph.replay, 5, 1, stream)

        def singles():
            for b in range(len(sizes)):
                plan.set_points(xys[b])
                plan.forward(hists[b], outs[b])

        ms_single = _time(singles, 3, 1, stream)
        plan.close()
        units = len(sizes) * gb.Z * gb.N * gb.N * gb.F
        M = 2 * gb.N
        b = 8 * n_classes(gb.N) * gb.F * gb.Z  # the shared table, read once
        for Lb in sizes:  # per item: temporal, type 1, its spectrum and depth spectra, inverse passes
            Lb = int(Lb)
            b += (Lb * gb.T * 4 + Lb * gb.F * 8 + bytes_type1(Lb, gb.F, gb.N) + 8 * (M * M * gb.F + M * M * gb.Z)
                  + bytes_idft(gb.Z, gb.N))
        return {"workload": "%d reconstructions, L log-uniform 4,096-65,536 (sum %d), T=512 @ 8 ps, F=64, "
                            "128^2 x 64 each" % (len(sizes), int(sizes.sum())),
                "ms_graph": ms_graph, "recon_per_s": len(sizes) / (ms_graph / 1e3),
                "voxel_freq_per_s": units / (ms_graph / 1e3), **hbm_row(b, ms_graph, peak),
                "ms_64_single_calls": ms_single, "speedup_vs_single_calls": ms_single / ms_graph,
                "autotuned": {"choice": tuned["choice"], "ms_by_setting": tuned["results"]}}

    def cufft():
        # comparison only (timed, not part of the path): cuFFT through torch.fft on the full
        # oversampled grid [F][4N][4N] and on the depth spectra [Z][2N][2N] with the crop, beside
        # this library's pruned channel-last panel passes of the same two stages
        M, nf, F, Z, N = 2 * g.N, 4 * g.N, g.F, g.Z, g.N
        x = torch.randn((F, nf, nf), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        ms_f = _time(lambda: torch.fft.fft2(x, out=y), 5, 2, stream)
        del x, y
        Yd = torch.randn((Z, M, M), dtype=torch.complex64, device="cuda")
        m = torch.arange(-(N // 2), N - N // 2, device="cuda") % M
        ms_i = _time(lambda: torch.fft.ifft2(Yd)[:, m][:, :, m], 5, 2, stream)
        del Yd
        st = stages_ms or {}
        ours_f = st.get("fft_x", 0.0) + st.get("fft_y", 0.0)
        ours_i = st.get("ifft_x", 0.0) + st.get("ifft_y", 0.0)
        return {"workload": "forward fine-grid FFT (a4-a5) and inverse FFT with crop (a7) at spad-65k",
                "cufft_forward_full_grid_ms": ms_f, "ours_forward_pruned_ms": ours_f,
                "cufft_inverse_with_crop_ms": ms_i, "ours_inverse_pruned_ms": ours_i,
                "note": "cuFFT transforms the whole 1024^2 oversampled grid of every frequency (plane-major) and "
                        "every 512^2 depth spectrum before the crop; the library's passes transform only the "
                        "spread window and keep only the retained bins, channel-last"}

    guarded("d_cufft_comparison", cufft)
    guarded("a8_type2_voxels", type2)
    guarded("a9_srsd", srsd)
    guarded("a10_adjoint", adjoint)
    guarded("a11_gradients", grad)
    guarded("a12_batched", batched)

    def batched_spad():
        # throughput form of the headline workload: 16 reconstructions of the 65k-sample keystone layout
        # (16 captures of different scenes through the same relay samples) in one call; the shared table
        # is then read once per call, and the contraction runs on the tensor cores
        B = 16
        scenes = batch_scenes_c4(B, seed=BASE_SEED + 60)
        plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=L,
                          max_batch=B)
        xys = [d_xy] * B
        hists = [device_histograms(d_xy, *scenes[b], g.T, g.dt, g.t0, seed=BASE_SEED + 600 + b) for b in range(B)]
        outs = list(plan.empty_batch_output(B))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            plan.forward_batched(xys, hists, outs)  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            plan.forward_batched(xys, hists, outs)
        ms_graph = _time(graph.replay, 5, 1, stream)
        plan.profile(True)
        plan.forward_batched(xys, hists, outs)
        st = {k: v[0] for k, v in plan.profile_read().items() if v[1]}
        plan.profile(False)

        def singles():
            for b in range(B):
                plan.set_points(xys[b])
                plan.forward(hists[b], outs[b])

        ms_single = _time(singles, 2, 1, stream)
        assert plan.sync_status() == 0
        plan.close()
        M = 2 * g.N
        b = 8 * n_classes(g.N) * g.F * g.Z + B * (L * g.T * 4 + L * g.F * 8 + bytes_type1(L, g.F, g.N)
                                                 + 8 * (M * M * g.F + M * M * g.Z) + bytes_idft(g.Z, g.N))
        units = B * g.Z * g.N * g.N * g.F
        return {"workload": "16 reconstructions of the 65,536-sample keystone layout (16 scenes), T=1024 @ 4 ps, "
                            "F=128 -> 256^2 x 128 each, in one batched call",
                "ms_graph": ms_graph, "recon_per_s": B / (ms_graph / 1e3), "voxel_freq_per_s": units / (ms_graph / 1e3),
                **hbm_row(b, ms_graph, peak), "ms_16_single_calls": ms_single,
                "speedup_vs_single_calls": ms_single / ms_graph, "stages_ms": st}

    guarded("a12_batched_spad", batched_spad)
    def nusfft():
        # next row 2, second half: SRSD taken directly at the 65,536 keystone samples (NU-SFFT)
        depths = srsd_depths_c3b(row_depths)
        pitches = srsd_pitches_c3b(depths)
        plan = nursd.Plan(g.N, g.pitch, g.center, depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=L,
                          srsd_pitch=pitches)
        plan.set_points(d_xy)
        P = plan.temporal_dft(d_hist)
        out = plan.empty_output()
        plan.srsd_forward_nonuniform(P, out)  # first call: tables and workspace
        ms = _time(lambda: plan.srsd_forward_nonuniform(P, out), 3, 1, stream)
        assert plan.sync_status() == 0
        plan.close()
        Z = len(depths)
        b = bytes_nusfft(L, g.N, g.F, pitches / g.pitch) + bytes_idft(Z, g.N)
        return {"workload": f"65,536 keystone samples -> 256^2 x {Z} planes over 1-4 m, pitch 8 -> 32 mm, F=128, "
                            "scaled DFT at the samples (NU-SFFT)",
                "ms": ms, "voxel_freq_per_s": Z * g.N * g.N * g.F / (ms / 1e3), **hbm_row(b, ms, peak)}

    def resample():
        # next row 4: keep every 5th relay sample of a 256 x 256 x 128 phasor grid, re-grid linearly
        N, F, D = g.N, g.F, 5
        grid = torch.from_numpy(random_phasors(N * N, F, seed=BASE_SEED + 32).reshape(N, N, F)).cuda()
        kept = nursd.subsample(grid, D)
        full = torch.empty_like(grid)
        ms_s = _time(lambda: nursd.subsample(grid, D, out=kept), 20, 3, stream)
        ms_u = _time(lambda: nursd.upsample(kept, N, D, linear=True, out=full), 20, 3, stream)
        nc = kept.shape[0]
        return {"workload": "256 x 256 x 128 phasor grid, every 5th sample kept (52 x 52), linear re-gridding",
                "subsample_ms": ms_s, "upsample_ms": ms_u,
                "subsample": hbm_row(8 * 2 * nc * nc * F, ms_s, peak),
                "upsample": hbm_row(8 * (nc * nc * F + N * N * F), ms_u, peak)}

    def nursd3d():
        # next row 3: 3D NURSD on a non-planar relay: the 65,536 keystone samples bent into a cylinder
        # (heights within +-5 cm of the reference plane), 128^2 x 64 planes 0.5-3 m beyond it, F = 64,
        # 16 z offsets of 1.5 cm
        N, F, Z, Mz, dz = 128, 64, 64, 16, 0.015
        xy = relay_keystone(seed=BASE_SEED + 7)
        h = (0.05 * ((xy[:, 0].astype(np.float64) / 0.985) ** 2 * 2.0 - 1.0)).astype(np.float32)
        om3, wt3 = om[::2].copy(), wt[::2].copy()
        plan = nursd.Plan(N, 2.0 / N, (0.0, 0.0), np.linspace(0.5, 3.0, Z), om3, wt3, max_points=len(xy))
        plan.enable_3d(dz, Mz)
        plan.set_points_3d(torch.from_numpy(xy).cuda(), torch.from_numpy(h).cuda())
        P = torch.from_numpy(random_phasors(len(xy), F, seed=BASE_SEED + 8)).cuda()
        out = plan.empty_output()
        plan.profile(True)
        ms = _time(lambda: plan.forward_3d(P, out), 5, 2, stream)
        st = _stage_ms(plan, 7)
        assert plan.sync_status() == 0
        plan.close()
        M, W = 2 * N, fine_window(N)
        Wz = min(2 * Mz, Mz + 6 + 2)
        b = (Wz * (8 * (len(xy) * F) + bytes_type1(len(xy), F, N))  # per z slice: phasors, spread, lateral passes
             + 8 * (Wz * M * M * F + M * M * Mz * F)  # the z pass
             + 8 * (2 * M * M * Mz * F + M * M * F)  # the kz sum with the 3D table
             + 8 * (M * M * F + 2 * M * N * F + N * N * F) + 8 * (N * N * F + 2 * N * M * F + M * M * F)  # crop, pad
             + bytes_contract(F, Z, N) + bytes_idft(Z, N))  # stage 2
        return {"workload": "65,536 keystone samples on a cylindrical relay (heights +-5 cm), F=64, 128^2 x 64 planes "
                            "0.5-3 m, Mz=16 offsets of 1.5 cm",
                "ms": ms, "voxel_freq_per_s": Z * N * N * F / (ms / 1e3), **hbm_row(b, ms, peak), "stages_ms": st}

    guarded("f3_nursd3d", nursd3d)
    guarded("f2_nu_sfft", nusfft)
    guarded("f4_subsample_regrid", resample)
    guarded("f1_single_illumination", illuminated)
    guarded("f2_srsd_points", srsd_points)
    return rows


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import paper_2501_05244_gb300 as nursd
    from workloads import BASE_SEED, workload_c2, workload_c5

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    nursd.build()
    if args.workload == "grid128":
        wl = workload_c5(seed=BASE_SEED + 5 + rank)
    else:
        wl = workload_c2(seed=BASE_SEED + 2 + rank)  # each rank reconstructs its own measurement
    if args.workload == "spad-z8":
        wl.geom = dataclasses.replace(wl.geom, depths=wl.geom.depths[::16].copy())
    if args.workload == "spad-n128":
        wl.geom = dataclasses.replace(wl.geom, N=128, pitch=2.0 * wl.geom.pitch)
    g = wl.geom
    L = len(wl.xy)
    om, wt = nursd.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    stream = torch.cuda.current_stream()
    plan = nursd.Plan(g.N, g.pitch, g.center, g.depths, om, wt, T=g.T, t0=g.t0, dt=g.dt, max_points=L)
    ckernel = CONTRACT_KERNELS[contract_kernel(plan, g.F, len(g.depths))]
    d_xy = torch.from_numpy(wl.xy).cuda()
    d_hist = torch.from_numpy(wl.hist).cuda()
    out = plan.empty_output()

    def step():  # positions + histograms -> volume (the point sort beside the temporal transform)
        plan.reconstruct(d_xy, d_hist, out=out)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if plan.sync_status() != 0:
        raise RuntimeError("device status error during warm-up")

    # The timed region replays one captured CUDA graph per step (same kernels and launches as the
    # eager call; the replay avoids per-launch host and scheduling gaps).  Each graph also holds the
    # two event-record nodes the plan places around the contraction, so the dominant kernel is timed
    # in every step of the timed region itself.  Eager steps if capture fails.
    launches0 = plan.launch_count
    step()
    launches_per_step = plan.launch_count - launches0
    plan.profile_stages(["contract"])
    for _ in range(args.steps):  # creates the event pairs the captures use
        step()
    torch.cuda.synchronize()
    plan.profile_read()
    graphs = None
    if not args.no_graph:
        try:
            cap = torch.cuda.Stream()
            cap.wait_stream(stream)
            with torch.cuda.stream(cap):
                step()
            stream.wait_stream(cap)
            torch.cuda.synchronize()
            plan.profile_read()
            graphs = []
            for _ in range(args.steps):
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr):
                    step()
                graphs.append(gr)
            torch.cuda.synchronize()
        except Exception:  # fall back to eager steps
            graphs = None
            torch.cuda.synchronize()
            plan.profile_read()

    # ---- timed region (device): K steps, events on the launching stream
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        if graphs is not None:
            graphs[i].replay()
        else:
            step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    if plan.sync_status() != 0:
        raise RuntimeError("device status error in the timed region")
    c_ms, c_n = plan.profile_read()["contract"]  # the contraction of each timed step
    plan.profile(False)
    graphs = None
    launches = launches_per_step * args.steps
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, dist, "cuda")

    # ---- per-stage times: CUDA events around each stage of eager steps (outside the timed region)
    plan.profile(True)
    n_prof = max(1, min(args.steps, 100))
    for _ in range(n_prof):
        step()
    torch.cuda.synchronize()
    stages = plan.profile_read()
    plan.profile(False)

    # ---- end to end through the public API with host buffers (pinned), copies inside the timed region.
    # Each step uploads its histograms and samples, reconstructs and downloads the volume.  The
    # upload of step k+1 and the download of step k-1 run on two copy streams (one per direction of
    # the host link) while step k computes (double-buffered device inputs and outputs); every copy is
    # inside the region.
    h_hist = torch.from_numpy(wl.hist).pin_memory()
    h_xy = torch.from_numpy(wl.xy).pin_memory()
    h_out = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    ke = max(1, min(args.e2e_steps, args.steps))
    copy = torch.cuda.Stream()
    copy_down = torch.cuda.Stream()
    dh = [d_hist, torch.empty_like(d_hist)]
    dx = [d_xy, torch.empty_like(d_xy)]
    do = [out, torch.empty_like(out)]
    up = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    down = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(k):
        with torch.cuda.stream(copy):
            copy.wait_event(done[k % 2])  # the buffers' previous reconstruction has finished
            dh[k % 2].copy_(h_hist, non_blocking=True)
            dx[k % 2].copy_(h_xy, non_blocking=True)
            up[k % 2].record(copy)

    # each step's reconstruction is an eager call here: a captured graph per buffer parity measured
    # slower end to end (graph launches interleaved with the copy stream's waits)
    recon = [lambda i=i: plan.reconstruct(dx[i], dh[i], out=do[i]) for i in range(2)]

    def e2e_run(steps):
        for e in done + down:
            e.record(stream)
        upload(0)
        for k in range(steps):
            if k + 1 < steps:
                upload(k + 1)
            stream.wait_event(up[k % 2])
            stream.wait_event(down[k % 2])  # this output buffer's previous download has finished
            recon[k % 2]()
            done[k % 2].record(stream)
            with torch.cuda.stream(copy_down):
                copy_down.wait_event(done[k % 2])
                h_out.copy_(do[k % 2], non_blocking=True)
                down[k % 2].record(copy_down)
        stream.wait_stream(copy)
        stream.wait_stream(copy_down)

    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    e2e_run(ke)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = reduce_max(f0.elapsed_time(f1) / ke, dist, "cuda")
    if plan.sync_status() != 0:
        raise RuntimeError("device status error in the timed region")

    units = g.Z * g.N * g.N * g.F  # voxel*freq per reconstruction
    value = job_throughput(units, world, ms)
    peak, peak_src = peaks()
    M, Z, F, N = plan.M, g.Z, g.F, g.N
    # algorithmic bytes of the contraction launch: table once, spectrum once, depth spectra once
    contract_bytes = plan.n_classes * F * Z * 8 + M * M * F * 8 + M * M * Z * 8
    c_avg = c_ms / max(c_n, 1)
    achieved = contract_bytes / (c_avg / 1e3) / 1e9
    W = (2 * N + 6 + 2 + 15) // 16 * 16
    step_bytes = (L * g.T * 4 + L * F * 8  # temporal: histograms in, phasors out
                  + L * F * 8 + W * W * F * 8  # spread: phasors in, fine window out
                  + W * W * F * 8 + W * M * F * 8  # FFT x
                  + W * M * F * 8 + M * M * F * 8  # FFT y
                  + contract_bytes  # contraction
                  + M * M * Z * 8 + M * N * Z * 8  # IFFT kx
                  + M * N * Z * 8 + Z * N * N * 8)  # IFFT ky
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic (seeded keystone layout, Poisson histograms of 5 point scatterers)",
        "config": {"workload": {"spad": WORKLOAD,
                                "grid128": "grid128: " + WORKLOAD.replace("256x256x128", "128x128x64"),
                                "spad-z8": "spad-z8: " + WORKLOAD.replace("256x256x128", "256x256x8"),
                                "spad-n128": "spad-n128: " + WORKLOAD.replace("256x256x128", "128x128x128")}[
                                    args.workload], "L": L, "T": g.T, "F": F, "N": N, "Z": Z, "M": M, "fine_n": plan.fine_n,
                   "parallelism": f"replicas x{world} (one reconstruction per GPU)",
                   "launch": (f"one captured CUDA graph of a nursd_reconstruct call ({launches_per_step} kernels) "
                              f"replayed per step" if c_n and not args.no_graph else "eager nursd_reconstruct calls"),
                   "roofline_timing": f"CUDA events around the contraction in each of the {c_n} timed steps "
                                      f"(event-record nodes of the replayed graphs, on the launching stream)",
                   "stage_times": "CUDA events around each stage of 100 eager steps after the timed region, per step "
                                  "(a stage run in channel or depth groups is summed over its launches)",
                   "l2": "inputs larger than L2 (histograms 268 MB, transfer table %.2f GB); no flush" %
                         (plan.n_classes * F * Z * 8 / 1e9)},
        "recon_per_s": world * 1e3 / ms,
        "roofline": {"bound": "hbm", "kernel": ckernel[0],
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_src} hbm_gbs",
                     "traffic": measured_traffic(ckernel[1]) if args.workload == "spad" else None,
                     "algorithmic_bytes": contract_bytes, "avg_launch_ms": c_avg},
        "step_hbm": {"algorithmic_bytes": step_bytes, "achieved_gbs": step_bytes / (ms / 1e3) / 1e9,
                     "frac": step_bytes / (ms / 1e3) / 1e9 / peak},
        "stages_ms": {k: v[0] / n_prof for k, v in stages.items() if v[1]},
        "gpu_launches": int(launches),
        "e2e": {"value": job_throughput(units, world, ms_e2e), "unit": UNIT, "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": int(h_hist.numel() * 4 + h_xy.numel() * 4),
                "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size())},
        "clocks": clk,
    }
    only = tuple(r for r in args.rows.split(",") if r)
    if rank == 0 and world == 1 and not args.no_rows and (args.workload == "spad" or only):
        plan.close()
        line["rows"] = measure_rows(wl, peak, line["stages_ms"], only, args.row_depths, args.row_items)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, desc, cores = oracle_rate(wl, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        try:
            line["cpu_fast_fp64"] = cpu_fast_rate(wl)
        except Exception as exc:  # a comparison row; its failure is reported, not fatal
            line["cpu_fast_fp64"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_sharded(args, rank, world, local):
    """One spad-65k reconstruction per step with its depth planes split over the ranks (each rank holds
    its slice of the transfer table) and gathered in depth order by an all_gather (NCCL): strong
    scaling, eager steps (the gather is a collective between the ranks' launches)."""
    import torch

    from paper_2501_05244_gb300.nursd import phasor_frequencies
    from paper_2501_05244_gb300.sharding import DepthShardedPlan, depth_slices
    from workloads import BASE_SEED, workload_c2
    import paper_2501_05244_gb300 as nursd

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    nursd.build()
    wl = workload_c2(seed=BASE_SEED + 2)  # the same measurement on every rank
    g = wl.geom
    L = len(wl.xy)
    om, wt = phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    sp = DepthShardedPlan(g.N, g.pitch, g.center, g.depths, om, wt, rank=rank, world=world, dist=dist, T=g.T,
                          t0=g.t0, dt=g.dt, max_points=L)
    d_xy = torch.from_numpy(wl.xy).cuda()
    d_hist = torch.from_numpy(wl.hist).cuda()
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        sp.reconstruct(d_xy, d_hist)
    torch.cuda.synchronize()
    launches0 = sp.plan.launch_count if sp.plan is not None else 0
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        vol = sp.reconstruct(d_xy, d_hist)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    launches = (sp.plan.launch_count if sp.plan is not None else 0) - launches0  # this rank's, the timed steps
    # end to end: pinned host inputs uploaded, the reconstruction, the gathered volume downloaded
    h_hist = torch.from_numpy(wl.hist).pin_memory()
    h_xy = torch.from_numpy(wl.xy).pin_memory()
    h_out = torch.empty(tuple(vol.shape), dtype=vol.dtype).pin_memory()
    ke = max(1, min(args.e2e_steps, args.steps))
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(ke):
        d_hist.copy_(h_hist, non_blocking=True)
        d_xy.copy_(h_xy, non_blocking=True)
        vol = sp.reconstruct(d_xy, d_hist)
        h_out.copy_(vol, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = reduce_max(f0.elapsed_time(f1) / ke, dist, "cuda")
    units = g.Z * g.N * g.N * g.F
    line = {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic (seeded keystone layout, Poisson histograms of 5 point scatterers)",
        "config": {"workload": WORKLOAD, "L": L, "T": g.T, "F": g.F, "N": g.N, "Z": g.Z,
                   "parallelism": f"depth-sharded x{world} ({[b - a for a, b in depth_slices(g.Z, world)]} planes "
                                  f"per rank, all_gather of the planes)",
                   "launch": "eager nursd_reconstruct calls on each rank's depth slice, then the gather",
                   "l2": "inputs larger than L2; no flush"},
        "recon_per_s": 1e3 / ms,
        "gpu_launches": int(launches),
        "e2e": {"value": units / (ms_e2e / 1e3), "unit": UNIT, "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": int(h_hist.numel() * 4 + h_xy.numel() * 4),
                "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size())},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    sp.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args, rank, world, local):
    """The FP64 oracle (direct back-projection) on all host cores: each step back-projects one random
    voxel x 16 frequencies per worker process over all relay samples."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    from workloads import BASE_SEED, workload_c2

    wl = workload_c2(seed=BASE_SEED + 2)
    g = wl.geom
    om, wt = O.phasor_frequencies(g.lambda_c, g.dt, g.t_pad, g.F)
    t0 = time.perf_counter()
    P = O.temporal_dft(wl.hist, g.t0, g.dt, om, wt)
    t_temporal = time.perf_counter() - t0
    rng = np.random.default_rng(11)
    nf = 16  # each task: one voxel x 16 frequencies (cycling through the band)
    pool = OraclePool(P, wl.xy, om)
    cores = pool.cores

    def one(i):
        tasks = []
        for c in range(cores):
            f0 = ((i * cores + c) * nf) % g.F
            tasks.append((_random_voxels(g, 1, rng), f0, f0 + nf))
        return pool.run(tasks)

    try:
        for i in range(args.warmup):
            one(i)
        t0 = time.perf_counter()
        units = 0
        for i in range(args.steps):
            units += one(args.warmup + i)
        t = time.perf_counter() - t0
    finally:
        pool.close()
    full = g.Z * g.N * g.N * g.F
    per_step = units / args.steps
    t_step = t / args.steps + t_temporal * per_step / full
    value = per_step / t_step
    desc = (f"each step: oracle.fbp_direct (FP64 NumPy direct back-projection) of one random voxel x {nf} "
            f"frequencies per worker on {cores} single-threaded worker processes, over all {len(wl.xy)} relay "
            f"samples, plus the oracle temporal transform of all histograms ({t_temporal:.1f} s) charged pro rata")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": len(wl.xy), "T": g.T, "F": g.F, "N": g.N, "Z": g.Z,
                       "M": 2 * g.N, "fine_n": 4 * g.N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    elif args.shard == "depth":
        run_sharded(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
