"""CPU checks of the C ABI: the library builds, loads without a GPU and exports
every symbol include/pip.h declares; host-side argument checks reject bad
calls before any device work (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2007_15385_gb300 import binding as B
from paper_2007_15385_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pip.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pip_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_three_calls():
    syms = declared_symbols()
    for s in ("pip_prepare", "pip_test", "pip_margin", "pip_destroy", "pip_get_status"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s
        assert s in B.SIGNATURES, "binding lacks %s" % s


def test_status_strings(lib):
    for code in range(8):
        assert lib.pip_status_string(code)
    assert b"unknown" in lib.pip_status_string(99)


def test_host_argument_checks(lib):
    out = ctypes.c_void_p()
    # null pointers / bad sizes are refused before touching the device
    assert lib.pip_prepare(None, 0, None, 1, 8, 10, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG
    assert lib.pip_prepare(8, 0, 8, 0, 8, 10, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG
    assert lib.pip_prepare(8, 7, 8, 1, 8, 10, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG
    assert lib.pip_prepare(8, 0, 8, 1, 2, 10, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG
    assert lib.pip_prepare(8, 0, 8, 1, 65, 10, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG
    assert lib.pip_prepare(9, 0, 8, 1, 8, 10, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG  # misaligned
    assert lib.pip_prepare(8, 0, 8, 1, 8, -1, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG
    assert lib.pip_prepare(8, 0, 8, 1, 8, 1 << 33, None, ctypes.byref(out)) == B.PIP_E_INVALID_ARG
    assert lib.pip_prepare(8, 0, 8, 1, 8, 10, None, None) == B.PIP_E_INVALID_ARG
    # calls on a null table handle
    assert lib.pip_test(None, None, 0, 0, None, 1, None, None, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_margin(None, None, 0, 0, None, None, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_get_status(None, None, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_test_sign_of_offset(None, None, 0, None, None, None) == B.PIP_E_INVALID_ARG
    lib.pip_destroy(None)  # no-op
    assert lib.pip_num_polygons(None) == 0


def test_build_flags_target_sm103a():
    assert "arch=compute_103a,code=sm_103a" in build_mod.ARCH


def test_host_argument_checks_of_the_other_entry_points(lib):
    """Every entry point refuses a null table handle or a bad size on the host,
    before any device work; the size helpers compute their bytes on the host."""
    i32, f64 = ctypes.c_int32(0), ctypes.c_double(0.0)
    fms = ctypes.c_float(0.0)
    assert lib.pip_timing(None, 1) == B.PIP_E_INVALID_ARG
    assert lib.pip_timing_read(None, ctypes.byref(i32), ctypes.byref(f64), ctypes.byref(f64)) == B.PIP_E_INVALID_ARG
    assert lib.pip_get_polygon_status(None, None, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_export_tables(None, None, None, None, None, None, None, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_set_stream_variant(None, 0) == B.PIP_E_INVALID_ARG
    assert lib.pip_set_batch_variant(None, 0) == B.PIP_E_INVALID_ARG
    assert lib.pip_autotune_stream(None, None, 0, 1, None, 1, None, ctypes.byref(i32),
                                   ctypes.byref(fms)) == B.PIP_E_INVALID_ARG
    assert lib.pip_autotune_batch(None, None, 0, 1, None, None, 1, None, ctypes.byref(i32),
                                  ctypes.byref(fms)) == B.PIP_E_INVALID_ARG
    assert lib.pip_selftest_wait_timeout(None, None, 1000, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_rasterize(None, 8, 8, 0.0, 0.0, 1.0, 1.0, None, None, None, 0, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_stream_variant_count() >= 1 and lib.pip_batch_variant_count() >= 1
    # raster workspace: one bit per (tile, polygon), tiles of 64 x 48 pixels
    assert lib.pip_raster_workspace_bytes(0, 10, 10) == 0
    assert lib.pip_raster_workspace_bytes(1, 0, 10) == 0
    assert lib.pip_raster_workspace_bytes(33, 64, 48) == 2 * 4
    assert lib.pip_raster_workspace_bytes(32, 65, 49) == 4 * 4
    # penalty: bad sizes and null pointers are refused; the workspace size grows with the blocks
    assert lib.pip_penalty_workspace_bytes(0, 1, 1) == 0
    assert lib.pip_penalty_workspace_bytes(12, 4, 1 << 20) > lib.pip_penalty_workspace_bytes(12, 4, 1 << 10) > 0
    assert lib.pip_penalty_forward(None, 12, None, 4, None, 10, 0.05, None, 0, None, 0, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_penalty_backward(None, 12, None, 4, None, 10, 0.05, None, None, None, 0, None, 0,
                                    None) == B.PIP_E_INVALID_ARG
    # the tuning cache can be set and cleared without a GPU
    assert lib.pip_set_tuning_cache(None) == B.PIP_OK
    # the host-buffer call and the FMA calibration kernel refuse bad handles and sizes
    assert lib.pip_test_host(None, None, 0, 10, None, None, None, 8, None) == B.PIP_E_INVALID_ARG
    fm = ctypes.c_int64(0)
    assert lib.pip_fma_peak(0, 1, None, 0, None, ctypes.byref(fm)) == B.PIP_E_INVALID_ARG
    assert lib.pip_fma_peak(8, 0, None, 0, None, ctypes.byref(fm)) == B.PIP_E_INVALID_ARG
    # the allocation-free one-polygon call checks its arguments first
    assert lib.pip_test_single_noalloc(None, 0, 8, None, 0, 10, None, None, None) == B.PIP_E_INVALID_ARG
    assert lib.pip_test_single_noalloc(8, 5, 8, 8, 0, 10, 8, None, None) == B.PIP_E_INVALID_ARG  # bad dtype
    assert lib.pip_test_single_noalloc(8, 0, 2, 8, 0, 10, 8, None, None) == B.PIP_E_INVALID_ARG  # 2 vertices
