"""The C ABI without a GPU: the library loads, exports every entry point that
include/*.h declares, and rejects bad arguments on the host before it would
touch a device (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, f)).read(), flags=re.S)
            names.update(re.findall(r"\b(mmlttb_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib(libpath):
    return ctypes.CDLL(libpath)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("mmlttb_minmax_preselect", "mmlttb_lttb", "mmlttb_minmaxlttb",
                     "mmlttb_workspace_bytes", "mmlttb_strerror", "mmlttb_raster",
                     "mmlttb_raster_intensity", "mmlttb_visual_counts"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version(lib):
    lib.mmlttb_strerror.restype = ctypes.c_char_p
    assert lib.mmlttb_strerror(0) == b"success"
    assert lib.mmlttb_strerror(-1) == b"invalid argument"
    assert lib.mmlttb_strerror(-2) == b"workspace too small"
    assert lib.mmlttb_strerror(12345) == b"unknown error"
    assert lib.mmlttb_version() >= 100


def _call_minmaxlttb(lib, y, ydt, x, xk, n, n_out, r_ps, binmode, out, cap):
    f = lib.mmlttb_minmaxlttb
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                  ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    return f(y, ydt, x, xk, n, n_out, r_ps, binmode, out, cap, None, None, 0, None)


@pytest.mark.parametrize("args,code", [
    # (y, ydt, x, xk, n, n_out, r_ps, binmode, out, cap)
    ((1, 0, None, 0, 100, 10, 1, 0, 1, 10), -1),     # r_ps < 2
    ((1, 0, None, 0, 100, 2, 4, 0, 1, 10), -1),      # n_out < 3
    ((1, 7, None, 0, 100, 10, 4, 0, 1, 10), -1),     # bad dtype
    ((1, 0, None, 9, 100, 10, 4, 0, 1, 10), -1),     # bad x kind
    ((1, 0, None, 0, 100, 10, 4, 5, 1, 10), -1),     # bad bin mode
    ((1, 0, None, 0, 100, 10, 4, 1, 1, 10), -1),     # x-width bins need int64 x
    ((1, 0, None, 1, 100, 10, 4, 0, 1, 10), -1),     # int64 x but NULL pointer
    ((None, 0, None, 0, 100, 10, 4, 0, 1, 10), -1),  # NULL y
    ((1, 0, None, 0, -5, 10, 4, 0, 1, 10), -1),      # negative n
    ((1, 0, None, 0, 100, 10, 4, 0, 1, 9), -6),      # output capacity too small
    ((1, 0, None, 0, 100, 10, 4, 0, None, 10), -1),  # NULL output
])
def test_host_side_validation(lib, args, code):
    assert _call_minmaxlttb(lib, *args) == code


def test_single_path_preference_is_validated_on_the_host(lib):
    f = lib.mmlttb_set_single_path
    f.argtypes = [ctypes.c_int]
    for bad in (-1, 4, 99):
        assert f(bad) == -1
    for good in (1, 2, 3, 0):  # ends on AUTO
        assert f(good) == 0


def _raster(lib, y=1, ydt=0, x=None, xk=0, n=10, idx=None, k=0, ext=(0.0, 1.0, 0.0, 1.0), w=8, h=8, mask=1):
    f = lib.mmlttb_raster
    f.restype = ctypes.c_int
    d = ctypes.c_double
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, d, d, d, d, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    return f(y, ydt, x, xk, n, idx, k, *ext, w, h, mask, None)


@pytest.mark.parametrize("kw", [
    dict(y=None), dict(mask=None), dict(ydt=3), dict(xk=5), dict(xk=1), dict(n=-1), dict(idx=1, k=-2),
    dict(ext=(0.0, float("inf"), 0.0, 1.0)), dict(ext=(0.0, 1.0, float("nan"), 1.0)), dict(w=0), dict(h=-3),
    dict(w=65537), dict(w=65536, h=8192),
])
def test_raster_validation(lib, kw):
    assert _raster(lib, **kw) == -1


def test_raster_with_fewer_than_two_points_enqueues_nothing(lib):
    # returns before any CUDA call: fake pointers are never touched
    assert _raster(lib, n=1) == 0
    assert _raster(lib, idx=1, k=1) == 0
    assert _raster(lib, n=0, ext=(5.0, -5.0, 2.0, 2.0)) == 0  # reversed / zero extents are valid


def test_visual_metric_validation(lib):
    f = lib.mmlttb_visual_counts
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                  ctypes.c_void_p, ctypes.c_void_p]
    assert f(None, 1, 4, 4, 20, 1, None) == -1
    assert f(1, 1, 0, 4, 20, 1, None) == -1
    assert f(1, 1, 4, 4, -1, 1, None) == -1
    assert f(1, 1, 4, 4, 20, None, None) == -1
    assert f(1, 1, 65536, 65536, 20, 1, None) == -1
    g = lib.mmlttb_raster_intensity
    g.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    assert g(None, 4, 1, None) == -1
    assert g(1, -1, 1, None) == -1
    assert g(1, 0, 1, None) == 0


def test_diag_probe_validation(lib):
    f = lib.mmlttb_diag_wait_timeout
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert f(7, 1, 256, None) == -1      # unknown barrier kind
    assert f(0, None, 256, None) == -1   # NULL workspace
    assert f(1, 1, 255, None) == -1      # smaller than the header


def test_check_series_validation(lib):
    f = lib.mmlttb_check_series
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p]
    assert f(None, 0, None, 0, 10, 1, None) == -1  # NULL y
    assert f(1, 0, None, 0, 10, None, None) == -1  # NULL flags
    assert f(1, 5, None, 0, 10, 1, None) == -1     # bad y type
    assert f(1, 0, None, 1, 10, 1, None) == -1     # int64 x but NULL
    assert f(1, 0, None, 0, -1, 1, None) == -1     # negative n
