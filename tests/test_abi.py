"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/*.h declares; host-side argument checks fail cleanly."""
import ctypes as ct
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(kc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for want in ("kc_gonzalez", "kc_radius", "kc_sync", "kc_last_error", "kc_release", "kc_version"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1604_03228_gb300 import build
    lib = ct.CDLL(build.build())
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version_and_host_argument_errors():
    import paper_1604_03228_gb300 as kc
    L = kc.load()
    assert b"sm_103a" in L.kc_version()
    pts = np.zeros((4, 2), dtype=np.float32)
    C = np.zeros(2, dtype=np.int64)
    ko = np.zeros(1, dtype=np.int32)
    r = np.zeros(1, dtype=np.float64)
    # invalid sizes are rejected before any CUDA call
    assert L.kc_gonzalez(pts.ctypes.data, 0, 2, 2, 0, C.ctypes.data, ko.ctypes.data, r.ctypes.data, None) == kc.KC_ERR_ARG
    assert b"n=0" in L.kc_last_error()
    assert L.kc_gonzalez(pts.ctypes.data, 4, 2, 0, 0, C.ctypes.data, ko.ctypes.data, r.ctypes.data, None) == kc.KC_ERR_ARG
    assert L.kc_gonzalez(pts.ctypes.data, 4, 2, 2, 4, C.ctypes.data, ko.ctypes.data, r.ctypes.data, None) == kc.KC_ERR_ARG
    assert L.kc_gonzalez(None, 4, 2, 2, 0, C.ctypes.data, ko.ctypes.data, r.ctypes.data, None) == kc.KC_ERR_ARG
    assert L.kc_radius(pts.ctypes.data, 4, 0, C.ctypes.data, 2, r.ctypes.data, None, None) == kc.KC_ERR_ARG


def test_binding_raises_typed_errors():
    import paper_1604_03228_gb300 as kc
    with pytest.raises(TypeError):
        kc.kc_gonzalez(np.zeros((4, 2), dtype=np.float64), 2)
    with pytest.raises(kc.KCError) as e:
        kc.kc_gonzalez(np.zeros((4, 2), dtype=np.float32), 2, first=9)
    assert e.value.status == kc.KC_ERR_ARG


def test_batch_plan_host_argument_errors():
    import paper_1604_03228_gb300 as kc
    L = kc.load()
    h = ct.c_void_p()
    n = np.array([10], dtype=np.int64)
    d = np.array([2], dtype=np.int32)
    k = np.array([2], dtype=np.int32)
    # rejected before any CUDA call
    assert L.kc_batch_plan_create(0, None, None, None, None, None, None, None, None, ct.byref(h)) == kc.KC_ERR_ARG
    assert L.kc_batch_plan_create(1, None, n.ctypes.data, d.ctypes.data, k.ctypes.data, None, None, None, None,
                                  None) == kc.KC_ERR_ARG
    assert L.kc_batch_plan_run(None, None) == kc.KC_ERR_ARG
    assert L.kc_batch_plan_wait(None) == kc.KC_ERR_ARG
    assert L.kc_batch_plan_destroy(None) == kc.KC_OK


def test_measurement_and_diagnostic_entry_points_check_arguments():
    import paper_1604_03228_gb300 as kc
    L = kc.load()
    sink = np.zeros(1, dtype=np.uint64)
    buf = np.zeros(64, dtype=np.float32)
    # rejected before any CUDA call: no buffer, no sink, no repetition, size not a multiple of 16
    assert L.kc_read_sweep(None, 256, 1, sink.ctypes.data, None) == kc.KC_ERR_ARG
    assert L.kc_read_sweep(buf.ctypes.data, 256, 1, None, None) == kc.KC_ERR_ARG
    assert L.kc_read_sweep(buf.ctypes.data, 256, 0, sink.ctypes.data, None) == kc.KC_ERR_ARG
    assert L.kc_read_sweep(buf.ctypes.data, 250, 1, sink.ctypes.data, None) == kc.KC_ERR_ARG
    assert L.kc_last_fp32_radius(None, None) == kc.KC_ERR_ARG


def test_checked_build_flags_are_declared():
    import paper_1604_03228_gb300 as kc
    src = open(os.path.join(ROOT, "include", "kcenter.h")).read()
    assert "KC_ERR_BOUNDS = 7" in src and "KC_TEST_BAD_INDEX 0x40000000u" in src
    assert kc.binding.KC_ERR_BOUNDS == 7 and kc.binding.KC_TEST_BAD_INDEX == 0x40000000
