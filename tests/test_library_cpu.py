"""CPU-side checks of libnursd: it builds, loads, exports every declared entry
point, and its host-only logic (status strings, frequency helper, descriptor
validation) behaves.  No GPU compute is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2501_05244_gb300 as nursd
from paper_2501_05244_gb300 import nursd as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nursd.build()
    return nursd.load_library()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\*]+\s+\**\s*(nursd_\w+|srsd_\w+)\s*\(", text, re.M))
    return names


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(binding.EXPORTS) | (names - set(binding.EXPORTS))
    assert set(binding.EXPORTS) <= names


def test_binding_tunables_and_stages_match_the_header():
    # the Python names of the plan tunables and profiling stages must carry the header's numbers
    text = open(os.path.join(ROOT, "include", "nursd.h")).read()
    tunes = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"#define NURSD_TUNE_(\w+) (\d+)", text)}
    assert tunes == binding.TUNABLES
    stages = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"NURSD_STAGE_(\w+) = (\d+)", text)}
    assert {name: i for i, name in enumerate(binding.STAGES)} == {k: v for k, v in stages.items() if k != "count"}


def test_status_strings(lib):
    assert nursd.status_string(0) == "ok"
    assert "aperture" in nursd.status_string(binding.NURSD_ERR_POINT_OUT_OF_RANGE)
    assert nursd.status_string(999) == "unknown status"


def test_library_frequency_helper_matches_oracle(lib):
    for args in ((0.06, 16e-12, 256, 16), (0.06, 4e-12, 8192, 128), (0.04, 8e-12, 2048, 64)):
        om, wt = nursd.phasor_frequencies(*args)
        om_o, wt_o = oracle.phasor_frequencies(*args)
        assert np.allclose(om, om_o, rtol=1e-14) and np.allclose(wt, wt_o, rtol=1e-12, atol=1e-15)
    with pytest.raises(nursd.NursdError):
        nursd.phasor_frequencies(-1.0, 1e-12, 256, 16)


def _desc(**kw):
    depths = np.linspace(0.5, 1.5, 4)
    omega = np.linspace(2e10, 4e10, 8)
    d = binding._Desc()
    d.N, d.pitch, d.center_x, d.center_y = 32, 1 / 32, 0.0, 0.0
    d.Z, d.F, d.T, d.t0, d.dt = 4, 8, 256, 1e-9, 16e-12
    d.upsample, d.kernel_width, d.flags, d.max_points = 2, 6, 0, 128
    keep = [depths, omega]
    d.h_depths = depths.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.h_omega = omega.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.h_weight = ctypes.POINTER(ctypes.c_double)()
    d.h_srsd_pitch = ctypes.POINTER(ctypes.c_double)()
    d.max_batch = 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("field,value,code", [
    ("N", 48, binding.NURSD_ERR_UNSUPPORTED),
    ("N", 4, binding.NURSD_ERR_UNSUPPORTED),
    ("N", 1024, binding.NURSD_ERR_UNSUPPORTED),
    ("pitch", 0.0, binding.NURSD_ERR_INVALID_ARG),
    ("pitch", float("nan"), binding.NURSD_ERR_INVALID_ARG),
    ("Z", 0, binding.NURSD_ERR_INVALID_ARG),
    ("F", 0, binding.NURSD_ERR_INVALID_ARG),
    ("F", 257, binding.NURSD_ERR_INVALID_ARG),
    ("T", 100, binding.NURSD_ERR_INVALID_ARG),
    ("dt", 0.0, binding.NURSD_ERR_INVALID_ARG),
    ("upsample", 3, binding.NURSD_ERR_UNSUPPORTED),
    ("kernel_width", 12, binding.NURSD_ERR_UNSUPPORTED),
    ("max_points", -1, binding.NURSD_ERR_INVALID_ARG),
    ("flags", 0x80, binding.NURSD_ERR_UNSUPPORTED),
    ("max_batch", 257, binding.NURSD_ERR_INVALID_ARG),
    ("max_batch", -1, binding.NURSD_ERR_INVALID_ARG),
])
def test_descriptor_validation_happens_on_the_host(lib, field, value, code):
    d, keep = _desc(**{field: value})
    h = ctypes.c_void_p()
    assert lib.nursd_plan_create(ctypes.byref(d), None, ctypes.byref(h)) == code
    assert not h.value


def test_null_arguments_are_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.nursd_plan_create(None, None, ctypes.byref(h)) == binding.NURSD_ERR_INVALID_ARG
    d, keep = _desc()
    d.h_depths = ctypes.POINTER(ctypes.c_double)()
    assert lib.nursd_plan_create(ctypes.byref(d), None, ctypes.byref(h)) == binding.NURSD_ERR_INVALID_ARG
    assert lib.nursd_set_points(None, 0, None, None) == binding.NURSD_ERR_INVALID_ARG
    assert lib.nursd_forward(None, None, None, None) == binding.NURSD_ERR_INVALID_ARG
    assert lib.nursd_plan_bytes(None) == -1
    assert lib.nursd_plan_destroy(None) == 0


def test_depths_must_be_positive(lib):
    d, keep = _desc()
    keep[0][2] = -0.1
    h = ctypes.c_void_p()
    assert lib.nursd_plan_create(ctypes.byref(d), None, ctypes.byref(h)) == binding.NURSD_ERR_INVALID_ARG
