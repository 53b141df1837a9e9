"""CPU checks of the C-ABI boundary: the library loads and exports every entry
point that include/dpvba.h declares, and host-checkable errors behave as the
header documents.  No kernel is launched here."""
import ctypes
import os
import re

import pytest

from paper_2408_01654_b300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "dpvba.h")).read()
    return sorted(set(re.findall(r"DPVBA_API\s+[\w\s\*]+?\b(ba_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return capi.lib()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("ba_create", "ba_set_graph", "ba_step", "ba_sync", "ba_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(L):
    for s in declared_symbols():
        assert hasattr(L, s), s
    assert sorted(declared_symbols()) == sorted(capi.EXPORTED)


def test_default_options_and_status_strings(L):
    o = capi.default_options()
    assert o.precision == capi.BA_FP32
    assert abs(o.lambda_pose - 1e-4) < 1e-9 and abs(o.lambda_depth - 1e-4) < 1e-9
    assert abs(o.z_min - 0.1) < 1e-7 and abs(o.d_min - 1e-3) < 1e-9
    assert L.ba_status_string(capi.BA_ERR_NOT_SPD) == b"BA_ERR_NOT_SPD"
    assert L.ba_status_string(99) == b"BA_ERR_UNKNOWN"


def test_null_arguments_rejected_without_gpu(L):
    assert L.ba_create(None, None) == capi.BA_ERR_INVALID_ARG
    assert L.ba_step(None, 1, 0) == capi.BA_ERR_INVALID_ARG
    assert L.ba_sync(None) == capi.BA_ERR_INVALID_ARG
    assert L.ba_destroy(None) == capi.BA_ERR_INVALID_ARG
    assert L.ba_default_options(None) == capi.BA_ERR_INVALID_ARG


def test_bad_options_rejected(L):
    h = ctypes.c_void_p()
    o = capi.default_options(patches_per_group=1000)
    assert L.ba_create(ctypes.byref(h), ctypes.byref(o)) == capi.BA_ERR_INVALID_ARG
    o = capi.default_options(precision=7)
    assert L.ba_create(ctypes.byref(h), ctypes.byref(o)) == capi.BA_ERR_INVALID_ARG
