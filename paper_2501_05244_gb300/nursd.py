"""Thin Python binding of libnursd (ctypes): argument marshalling only.

Every computation runs in the CUDA library; this module checks tensor
devices / dtypes / shapes, passes ``data_ptr()`` and the current CUDA stream,
and turns non-zero status codes into exceptions.  There is no CPU fallback:
if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnursd.so")

NURSD_OK = 0
NURSD_ERR_INVALID_ARG = 1
NURSD_ERR_OOM = 2
NURSD_ERR_CUDA = 3
NURSD_ERR_TIMEOUT = 4
NURSD_ERR_UNSUPPORTED = 5
NURSD_ERR_POINT_OUT_OF_RANGE = 6
NURSD_OUTPUT_MAGNITUDE = 0x1
NURSD_ENABLE_ADJOINT = 0x2
NURSD_CONFOCAL = 0x4
NURSD_UPSAMPLE_NEAREST = 0
NURSD_UPSAMPLE_LINEAR = 1
#: plan tunables (nursd_plan_tune)
TUNABLES = {"spread_rows": 0, "batch_streams": 1, "batch_grouped": 2, "batch_group": 3, "batch_tensor": 4,
            "contract_tc": 5}

#: every entry point declared in include/nursd.h
EXPORTS = (
    "nursd_status_string", "nursd_phasor_frequencies", "nursd_plan_create", "nursd_plan_destroy",
    "nursd_plan_bytes", "nursd_plan_dims", "nursd_set_points", "nursd_temporal_dft", "nursd_nufft1",
    "nursd_propagate", "nursd_forward_phasor", "nursd_forward", "nursd_sync_status",
    "nursd_profile_enable", "nursd_profile_select", "nursd_profile_read", "nursd_launch_count",
    "nursd_nufft1_noalloc",
    "nursd_forward_points", "nursd_adjoint", "nursd_grad_points", "srsd_forward", "srsd_forward_at", "nursd_plan",
    "nursd_forward_batched",
    "nursd_reconstruct", "nursd_forward_illuminated", "nursd_transient_frames", "srsd_forward_points",
    "nursd_subsample", "nursd_upsample", "srsd_forward_nonuniform", "nursd_plan_tune", "nursd_plan_get_tune",
    "nursd_test_fail_allocation", "nursd_test_set_wait_limit", "nursd_enable_3d", "nursd_set_points_3d",
    "nursd_forward_3d",
)

#: stage names in nursd_stage order
STAGES = ("points", "temporal", "spread", "fft_x", "fft_y", "contract", "ifft_x", "ifft_y", "srsd",
          "per_frequency")


class NursdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class _Desc(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("pitch", ctypes.c_double), ("center_x", ctypes.c_double),
        ("center_y", ctypes.c_double), ("Z", ctypes.c_int32), ("h_depths", ctypes.POINTER(ctypes.c_double)),
        ("F", ctypes.c_int32), ("h_omega", ctypes.POINTER(ctypes.c_double)),
        ("h_weight", ctypes.POINTER(ctypes.c_double)), ("T", ctypes.c_int32), ("t0", ctypes.c_double),
        ("dt", ctypes.c_double), ("upsample", ctypes.c_int32), ("kernel_width", ctypes.c_int32),
        ("flags", ctypes.c_uint32), ("max_points", ctypes.c_int32),
        ("h_srsd_pitch", ctypes.POINTER(ctypes.c_double)), ("max_batch", ctypes.c_int32),
        ("lambda_c", ctypes.c_double),
    ]


class _BatchItem(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("d_xy", ctypes.c_void_p), ("d_hist", ctypes.c_void_p),
                ("d_out", ctypes.c_void_p)]


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libnursd and declare the C signatures (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libnursd is not built ({path} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "nursd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "nursd_phasor_frequencies": (ctypes.c_int, [dbl, dbl, i32, i32, dp, dp]),
        "nursd_plan_create": (ctypes.c_int, [ctypes.POINTER(_Desc), vp, ctypes.POINTER(vp)]),
        "nursd_plan_destroy": (ctypes.c_int, [vp]),
        "nursd_plan_bytes": (i64, [vp]),
        "nursd_plan_dims": (ctypes.c_int, [vp, ip, ip, ip]),
        "nursd_set_points": (ctypes.c_int, [vp, i32, vp, vp]),
        "nursd_temporal_dft": (ctypes.c_int, [vp, i32, vp, vp, vp]),
        "nursd_nufft1": (ctypes.c_int, [vp, vp, vp, vp]),
        "nursd_propagate": (ctypes.c_int, [vp, vp, vp, vp]),
        "nursd_forward_phasor": (ctypes.c_int, [vp, vp, vp, vp]),
        "nursd_forward": (ctypes.c_int, [vp, vp, vp, vp]),
        "nursd_sync_status": (ctypes.c_int, [vp, vp]),
        "nursd_profile_enable": (ctypes.c_int, [vp, ctypes.c_int]),
        "nursd_profile_select": (ctypes.c_int, [vp, ctypes.c_uint32]),
        "nursd_profile_read": (ctypes.c_int, [vp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int64)]),
        "nursd_launch_count": (i64, [vp]),
        "nursd_nufft1_noalloc": (ctypes.c_int, [i32, dbl, dbl, dbl, i32, i32, vp, i32, vp, vp, vp]),
        "nursd_forward_points": (ctypes.c_int, [vp, vp, i32, vp, vp, vp]),
        "nursd_adjoint": (ctypes.c_int, [vp, vp, vp, vp]),
        "nursd_grad_points": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
        "srsd_forward": (ctypes.c_int, [vp, vp, vp, vp]),
        "srsd_forward_at": (ctypes.c_int, [vp, dp, vp, vp, vp]),
        "nursd_plan": (ctypes.c_int, [ctypes.POINTER(_Desc), vp, ctypes.POINTER(vp)]),
        "nursd_forward_batched": (ctypes.c_int, [vp, i32, ctypes.POINTER(_BatchItem), vp]),
        "nursd_reconstruct": (ctypes.c_int, [vp, i32, vp, vp, vp, vp]),
        "nursd_forward_illuminated": (ctypes.c_int, [vp, dp, vp, vp, vp]),
        "nursd_transient_frames": (ctypes.c_int, [vp, i32, dp, vp, vp, vp]),
        "srsd_forward_points": (ctypes.c_int, [vp, vp, i32, vp, vp, vp]),
        "nursd_subsample": (ctypes.c_int, [i32, i32, i32, vp, vp, vp]),
        "srsd_forward_nonuniform": (ctypes.c_int, [vp, vp, vp, vp]),
        "nursd_plan_tune": (ctypes.c_int, [vp, i32, i32]),
        "nursd_test_fail_allocation": (ctypes.c_int, [i32]),
        "nursd_enable_3d": (ctypes.c_int, [vp, dbl, i32, vp]),
        "nursd_set_points_3d": (ctypes.c_int, [vp, i32, vp, vp, vp]),
        "nursd_forward_3d": (ctypes.c_int, [vp, vp, vp, vp]),
        "nursd_test_set_wait_limit": (ctypes.c_int, [i64, vp]),
        "nursd_plan_get_tune": (ctypes.c_int, [vp, i32, ip]),
        "nursd_upsample": (ctypes.c_int, [i32, i32, i32, i32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load_library().nursd_status_string(status).decode()
    except RuntimeError:
        return f"status {status}"


def _check(rc: int, where: str):
    if rc != NURSD_OK:
        raise NursdError(rc, where)


def phasor_frequencies(lambda_c: float, dt: float, t_pad: int, F: int):
    """Frequencies [rad/s] and weights of the phasor-field band-pass (computed by libnursd)."""
    lib = load_library()
    om = (ctypes.c_double * F)()
    wt = (ctypes.c_double * F)()
    _check(lib.nursd_phasor_frequencies(lambda_c, dt, t_pad, F, om, wt), "nursd_phasor_frequencies")
    return np.array(om[:], dtype=np.float64), np.array(wt[:], dtype=np.float64)


def subsample(grid, D: int, out=None, stream=None):
    """Keep every D-th relay sample of a channel-last grid [N][N][F] complex64 -> [Nc][Nc][F], Nc = ceil(N / D)."""
    torch = _torch()
    N, F = int(grid.shape[0]), int(grid.shape[2])
    g = _dev(grid, torch.complex64, (N, N, F), "grid")
    nc = -(-N // int(D))
    if out is None:
        out = torch.empty((nc, nc, F), dtype=torch.complex64, device=grid.device)
    o = _dev(out, torch.complex64, (nc, nc, F), "kept")
    _check(load_library().nursd_subsample(N, F, int(D), g, o, ctypes.c_void_p(_stream_ptr(stream))),
           "nursd_subsample")
    return out


def upsample(kept, N: int, D: int, linear: bool = False, out=None, stream=None):
    """Re-grid kept samples [Nc][Nc][F] to the full N x N grid by nearest-neighbour or linear interpolation."""
    torch = _torch()
    nc, F = int(kept.shape[0]), int(kept.shape[2])
    if nc != -(-int(N) // int(D)):
        raise ValueError(f"kept grid must be ceil(N / D) = {-(-int(N) // int(D))} wide, got {nc}")
    k = _dev(kept, torch.complex64, (nc, nc, F), "kept")
    if out is None:
        out = torch.empty((N, N, F), dtype=torch.complex64, device=kept.device)
    o = _dev(out, torch.complex64, (N, N, F), "grid")
    _check(load_library().nursd_upsample(int(N), F, int(D), NURSD_UPSAMPLE_LINEAR if linear else NURSD_UPSAMPLE_NEAREST,
                                         k, o, ctypes.c_void_p(_stream_ptr(stream))), "nursd_upsample")
    return out


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev(t, dtype, shape, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A NURSD plan: geometry, transfer-function table and workspace on the current GPU."""

    def __init__(self, N: int, pitch: float, center, depths, omega, weight=None, T: int = 0, t0: float = 0.0,
                 dt: float = 0.0, max_points: int = 0, kernel_width: int = 6, upsample: int = 2,
                 magnitude: bool = False, adjoint: bool = False, srsd_pitch=None, max_batch: int = 0,
                 confocal: bool = False, lambda_c: float = 0.0,
                 stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("libnursd needs a CUDA GPU; none is available")
        self._lib = load_library()
        self.depths = np.ascontiguousarray(depths, dtype=np.float64)
        self.omega = np.ascontiguousarray(omega, dtype=np.float64)
        self.weight = None if weight is None else np.ascontiguousarray(weight, dtype=np.float64)
        self.N, self.Z, self.F, self.T = int(N), len(self.depths), len(self.omega), int(T)
        self.magnitude = bool(magnitude)
        d = _Desc()
        d.N = self.N
        d.pitch = float(pitch)
        d.center_x, d.center_y = float(center[0]), float(center[1])
        d.Z = self.Z
        d.h_depths = self.depths.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.F = self.F
        d.h_omega = self.omega.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.h_weight = (self.weight.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if self.weight is not None
                      else ctypes.POINTER(ctypes.c_double)())
        d.T, d.t0, d.dt = self.T, float(t0), float(dt)
        d.upsample, d.kernel_width = int(upsample), int(kernel_width)
        d.flags = ((NURSD_OUTPUT_MAGNITUDE if magnitude else 0) | (NURSD_ENABLE_ADJOINT if adjoint else 0)
                   | (NURSD_CONFOCAL if confocal else 0))
        d.max_points = int(max_points)
        self.srsd_pitch = None if srsd_pitch is None else np.ascontiguousarray(srsd_pitch, dtype=np.float64)
        d.h_srsd_pitch = (self.srsd_pitch.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                          if self.srsd_pitch is not None else ctypes.POINTER(ctypes.c_double)())
        d.max_batch = int(max_batch)
        d.lambda_c = float(lambda_c)  # with weight None: the Gaussian band-pass of this central wavelength
        self._desc = d
        h = ctypes.c_void_p()
        _check(self._lib.nursd_plan_create(ctypes.byref(d), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)),
               "nursd_plan_create")
        self._h = h
        M, nf, nc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.nursd_plan_dims(h, ctypes.byref(M), ctypes.byref(nf), ctypes.byref(nc)), "nursd_plan_dims")
        self.M, self.fine_n, self.n_classes = M.value, nf.value, nc.value
        self.max_points = int(max_points)
        self.L = None

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.nursd_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbytes(self) -> int:
        return int(self._lib.nursd_plan_bytes(self._h))

    def out_shape(self):
        return (self.Z, self.N, self.N)

    def out_dtype(self):
        torch = _torch()
        return torch.float32 if self.magnitude else torch.complex64

    def empty_output(self):
        torch = _torch()
        return torch.empty(self.out_shape(), dtype=self.out_dtype(), device="cuda")

    def empty_batch_output(self, B: int):
        """[B][Z][N][N] outputs side by side: forward_batched runs such a batch with grouped launches."""
        torch = _torch()
        return torch.empty((B,) + self.out_shape(), dtype=self.out_dtype(), device="cuda")

    # -- entry points
    def set_points(self, xy, stream=None):
        torch = _torch()
        L = int(xy.shape[0])
        p = _dev(xy, torch.float32, (L, 2), "xy")
        _check(self._lib.nursd_set_points(self._h, L, p, ctypes.c_void_p(_stream_ptr(stream))), "nursd_set_points")
        self.L = L

    def temporal_dft(self, hist, out=None, stream=None):
        torch = _torch()
        L = int(hist.shape[0])
        h = _dev(hist, torch.float32, (L, self.T), "hist")
        if out is None:
            out = torch.empty((L, self.F), dtype=torch.complex64, device=hist.device)
        o = _dev(out, torch.complex64, (L, self.F), "phasor")
        _check(self._lib.nursd_temporal_dft(self._h, L, h, o, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_temporal_dft")
        return out

    def nufft1(self, phasor, out=None, stream=None):
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        if out is None:
            out = torch.empty((self.M, self.M, self.F), dtype=torch.complex64, device=phasor.device)
        o = _dev(out, torch.complex64, (self.M, self.M, self.F), "spectrum")
        _check(self._lib.nursd_nufft1(self._h, p, o, ctypes.c_void_p(_stream_ptr(stream))), "nursd_nufft1")
        return out

    def propagate(self, spectrum, out=None, stream=None):
        torch = _torch()
        s = _dev(spectrum, torch.complex64, (self.M, self.M, self.F), "spectrum")
        if out is None:
            out = self.empty_output()
        o = _dev(out, self.out_dtype(), self.out_shape(), "out")
        _check(self._lib.nursd_propagate(self._h, s, o, ctypes.c_void_p(_stream_ptr(stream))), "nursd_propagate")
        return out

    def forward_phasor(self, phasor, out=None, stream=None):
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        if out is None:
            out = self.empty_output()
        o = _dev(out, self.out_dtype(), self.out_shape(), "out")
        _check(self._lib.nursd_forward_phasor(self._h, p, o, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_forward_phasor")
        return out

    def forward(self, hist, out=None, stream=None):
        torch = _torch()
        self._need_points()
        h = _dev(hist, torch.float32, (self.L, self.T), "hist")
        if out is None:
            out = self.empty_output()
        o = _dev(out, self.out_dtype(), self.out_shape(), "out")
        _check(self._lib.nursd_forward(self._h, h, o, ctypes.c_void_p(_stream_ptr(stream))), "nursd_forward")
        return out

    def reconstruct(self, xy, hist, out=None, stream=None):
        """Points and histograms -> volume in one call (set_points + forward, the point sort
        overlapped with the temporal transform); the plan keeps the points."""
        torch = _torch()
        L = int(xy.shape[0])
        p = _dev(xy, torch.float32, (L, 2), "xy")
        h = _dev(hist, torch.float32, (L, self.T), "hist")
        if out is None:
            out = self.empty_output()
        o = _dev(out, self.out_dtype(), self.out_shape(), "out")
        _check(self._lib.nursd_reconstruct(self._h, L, p, h, o, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_reconstruct")
        self.L = L
        return out

    def forward_points(self, phasor, vox, out=None, stream=None):
        """NURSD-2/3: values at per-plane voxels vox [Z][K][2] (metres) -> [Z][K] complex64."""
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        K = int(vox.shape[1])
        v = _dev(vox, torch.float32, (self.Z, K, 2), "vox")
        if out is None:
            out = torch.empty((self.Z, K), dtype=torch.complex64, device=phasor.device)
        o = _dev(out, torch.complex64, (self.Z, K), "out")
        _check(self._lib.nursd_forward_points(self._h, p, K, v, o, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_forward_points")
        return out

    def forward_batched(self, xys, hists, outs=None, stream=None):
        """B reconstructions (lists of xy [L_b][2], hist [L_b][T]) in one call -> list of volumes."""
        torch = _torch()
        B = len(xys)
        if outs is None:
            outs = list(self.empty_batch_output(B))
        items = (_BatchItem * B)()
        for b in range(B):
            L = int(xys[b].shape[0])
            items[b].L = L
            items[b].d_xy = _dev(xys[b], torch.float32, (L, 2), "xy").value
            items[b].d_hist = _dev(hists[b], torch.float32, (L, self.T), "hist").value
            items[b].d_out = _dev(outs[b], self.out_dtype(), self.out_shape(), "out").value
        self._batch_items = items  # keep alive while the call is enqueued
        _check(self._lib.nursd_forward_batched(self._h, B, items, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_forward_batched")
        self.L = int(xys[-1].shape[0])
        return outs

    def srsd_forward(self, phasor, out=None, stream=None, pitch=None):
        """Scaled RSD: plane z on the lattice of pitch srsd_pitch[z] -> [Z][N][N].  With `pitch` ([Z] metres)
        the plane pitches are given at the call (the plan's SRSD tables are rebuilt when they change)."""
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        if out is None:
            out = self.empty_output()
        o = _dev(out, self.out_dtype(), self.out_shape(), "out")
        if pitch is None:
            _check(self._lib.srsd_forward(self._h, p, o, ctypes.c_void_p(_stream_ptr(stream))), "srsd_forward")
        else:
            hp = np.ascontiguousarray(pitch, dtype=np.float64)
            if hp.shape != (self.Z,):
                raise ValueError(f"pitch: expected {self.Z} values")
            _check(self._lib.srsd_forward_at(self._h, hp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p, o,
                                             ctypes.c_void_p(_stream_ptr(stream))), "srsd_forward_at")
            self.srsd_pitch = hp
        return out

    # -- 3D NURSD (non-planar relays)
    def enable_3d(self, dz: float, Mz: int, stream=None):
        """Build the 3D transfer table for heights sampled at dz over Mz offsets (|h| <= Mz dz / 4)."""
        _check(self._lib.nursd_enable_3d(self._h, float(dz), int(Mz), ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_enable_3d")

    def set_points_3d(self, xy, h, stream=None):
        """Relay samples xy [L][2] with heights h [L] (metres, relative to the reference plane)."""
        torch = _torch()
        L = int(xy.shape[0])
        p = _dev(xy, torch.float32, (L, 2), "xy")
        hh = _dev(h, torch.float32, (L,), "h")
        _check(self._lib.nursd_set_points_3d(self._h, L, p, hh, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_set_points_3d")
        self.L = L

    def forward_3d(self, phasor, out=None, stream=None):
        """3D NURSD: the field at the reference plane, then propagated to the plan's depths -> [Z][N][N]."""
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        if out is None:
            out = self.empty_output()
        o = _dev(out, self.out_dtype(), self.out_shape(), "out")
        _check(self._lib.nursd_forward_3d(self._h, p, o, ctypes.c_void_p(_stream_ptr(stream))), "nursd_forward_3d")
        return out

    def srsd_forward_nonuniform(self, phasor, out=None, stream=None):
        """NU-SFFT: the scaled DFT taken at the relay samples (every scale >= 1) -> [Z][N][N]."""
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        if out is None:
            out = self.empty_output()
        o = _dev(out, self.out_dtype(), self.out_shape(), "out")
        _check(self._lib.srsd_forward_nonuniform(self._h, p, o, ctypes.c_void_p(_stream_ptr(stream))),
               "srsd_forward_nonuniform")
        return out

    def forward_illuminated(self, phasor, illum, out=None, stream=None):
        """Single-illumination volume [Z][N][N] complex64: each frequency's reconstruction weighted
        by exp(+i k_f |x_p - x_v|) before the frequency sum; illum = (x, y, z) metres."""
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        if out is None:
            out = torch.empty((self.Z, self.N, self.N), dtype=torch.complex64, device=phasor.device)
        o = _dev(out, torch.complex64, (self.Z, self.N, self.N), "out")
        xp = (ctypes.c_double * 3)(*[float(v) for v in illum])
        _check(self._lib.nursd_forward_illuminated(self._h, xp, p, o, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_forward_illuminated")
        return out

    def transient_frames(self, phasor, times, out=None, stream=None):
        """Frames [T][Z][N][N] complex64 of the virtual wave at the given times (seconds, the
        measurement's clock): each frequency's reconstruction weighted by exp(+i w_f t)."""
        torch = _torch()
        self._need_points()
        times = np.ascontiguousarray(times, dtype=np.float64).ravel()
        T = int(times.shape[0])
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        if out is None:
            out = torch.empty((T, self.Z, self.N, self.N), dtype=torch.complex64, device=phasor.device)
        o = _dev(out, torch.complex64, (T, self.Z, self.N, self.N), "out")
        tp = times.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(self._lib.nursd_transient_frames(self._h, T, tp, p, o, ctypes.c_void_p(_stream_ptr(stream))),
               "nursd_transient_frames")
        return out

    def srsd_forward_points(self, phasor, vox, out=None, stream=None):
        """SRSD + NURSD-2: scaled reconstruction at per-plane voxels vox [Z][K][2] (metres) -> [Z][K]."""
        torch = _torch()
        self._need_points()
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        K = int(vox.shape[1])
        v = _dev(vox, torch.float32, (self.Z, K, 2), "vox")
        if out is None:
            out = torch.empty((self.Z, K), dtype=torch.complex64, device=phasor.device)
        o = _dev(out, torch.complex64, (self.Z, K), "out")
        _check(self._lib.srsd_forward_points(self._h, p, K, v, o, ctypes.c_void_p(_stream_ptr(stream))),
               "srsd_forward_points")
        return out

    def adjoint(self, vol, out=None, stream=None):
        """A^H: complex volume [Z][N][N] -> phasors [L][F] at the current relay samples."""
        torch = _torch()
        self._need_points()
        v = _dev(vol, torch.complex64, self.out_shape(), "vol")
        if out is None:
            out = torch.empty((self.L, self.F), dtype=torch.complex64, device=vol.device)
        o = _dev(out, torch.complex64, (self.L, self.F), "phasor")
        _check(self._lib.nursd_adjoint(self._h, v, o, ctypes.c_void_p(_stream_ptr(stream))), "nursd_adjoint")
        return out

    def grad_points(self, w, phasor, want_phasor=True, want_xy=True, stream=None):
        """(A^H w, Re sum_f P conj(d(A^H w)/dx)) for w = 2 dL/d conj(V)."""
        torch = _torch()
        self._need_points()
        wv = _dev(w, torch.complex64, self.out_shape(), "w")
        p = _dev(phasor, torch.complex64, (self.L, self.F), "phasor")
        gp = torch.empty((self.L, self.F), dtype=torch.complex64, device=w.device) if want_phasor else None
        gx = torch.empty((self.L, 2), dtype=torch.float32, device=w.device) if want_xy else None
        _check(self._lib.nursd_grad_points(self._h, wv, p, None if gp is None else ctypes.c_void_p(gp.data_ptr()),
                                           None if gx is None else ctypes.c_void_p(gx.data_ptr()),
                                           ctypes.c_void_p(_stream_ptr(stream))), "nursd_grad_points")
        return gp, gx

    def sync_status(self, stream=None) -> int:
        return int(self._lib.nursd_sync_status(self._h, ctypes.c_void_p(_stream_ptr(stream))))

    # -- tunables
    def tune(self, name: str, value: int):
        """Set a launch-shape tunable (see TUNABLES); results do not depend on it."""
        _check(self._lib.nursd_plan_tune(self._h, TUNABLES[name], int(value)), "nursd_plan_tune")

    def tuning(self) -> dict:
        out = {}
        for name, key in TUNABLES.items():
            v = ctypes.c_int32()
            _check(self._lib.nursd_plan_get_tune(self._h, key, ctypes.byref(v)), "nursd_plan_get_tune")
            out[name] = v.value
        return out

    # -- profiling
    def profile(self, enable: bool = True):
        _check(self._lib.nursd_profile_enable(self._h, 1 if enable else 0), "nursd_profile_enable")

    def profile_stages(self, names):
        """Time only the named stages (see STAGES); an empty list stops recording."""
        mask = 0
        for n in names:
            mask |= 1 << STAGES.index(n)
        _check(self._lib.nursd_profile_select(self._h, mask), "nursd_profile_select")

    def profile_read(self):
        """{stage: (total_ms, executions)} since profiling was enabled or last read."""
        out = {}
        for i, name in enumerate(STAGES):
            ms, n = ctypes.c_double(), ctypes.c_int64()
            _check(self._lib.nursd_profile_read(self._h, i, ctypes.byref(ms), ctypes.byref(n)), "nursd_profile_read")
            out[name] = (ms.value, n.value)
        return out

    @property
    def launch_count(self) -> int:
        return int(self._lib.nursd_launch_count(self._h))

    def _need_points(self):
        if self.L is None:
            raise RuntimeError("set_points() must be called first")
