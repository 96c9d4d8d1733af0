"""The C-ABI library loads and exports every entry point include/vr.h declares; without a GPU the
calls fail with a status instead of falling back to the CPU.  CPU only (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "vr.h")).read()
    return re.findall(r"^\s*(?:vr_status|const char\s*\*)\s*(vr_\w+)\s*\(", src, re.M)


def test_header_declares_the_boundary_calls():
    names = set(declared())
    for n in ("vr_create", "vr_destroy", "vr_insert_slice", "vr_insert_block", "vr_set_transfer_functions",
              "vr_set_clip_planes", "vr_render", "vr_render_backward", "vr_read_level", "vr_stats", "vr_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1407_2074_b300 import vr

    lib = ctypes.CDLL(vr.LIB_PATH)
    for n in declared():
        assert hasattr(lib, n), n


def test_invalid_arguments_rejected_before_any_device_work():
    from paper_1407_2074_b300 import vr

    L = vr.lib()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(64, 64, 64)
    assert L.vr_create(dims, 5, 16, None, None, ctypes.byref(h)) == vr.VR_ERR_INVALID_ARG
    assert L.vr_create(dims, 3, 15, None, None, ctypes.byref(h)) == vr.VR_ERR_INVALID_ARG
    assert L.vr_create((ctypes.c_int64 * 3)(0, 4, 4), 3, 16, None, None, ctypes.byref(h)) == vr.VR_ERR_INVALID_ARG
    assert b"channels" in L.vr_last_error(None) or b"dims" in L.vr_last_error(None)
    assert L.vr_insert_slice(None, 0, None, 0, None) == vr.VR_ERR_INVALID_ARG
    assert L.vr_render(None, None, 0, None, 0, None) == vr.VR_ERR_INVALID_ARG


def test_no_device_means_an_error_not_a_fallback():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1407_2074_b300 import vr

    h = ctypes.c_void_p()
    rc = vr.lib().vr_create((ctypes.c_int64 * 3)(64, 64, 64), 3, 16, None, None, ctypes.byref(h))
    assert rc == vr.VR_ERR_CUDA and not h.value
