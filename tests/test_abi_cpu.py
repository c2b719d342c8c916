"""The C-ABI library loads and exports every entry point that include/hv.h
declares; error paths that need no GPU behave as documented."""
import ctypes
import os
import re

import pytest

from paper_2508_03911_gb300 import hv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hv_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = hv.lib()
    declared = header_functions()
    assert "hv_open" in declared and "hv_render" in declared
    for name in declared:
        assert hasattr(L, name), name


def test_version_and_null_handling():
    assert "sm_103a" in hv.hv_version()
    L = hv.lib()
    assert L.hv_close(None) == hv.HV_OK
    assert L.hv_push_frames(None, None, 1, 0) == hv.HV_ERR_ARG
    n = ctypes.c_uint32(7)
    assert L.hv_render(None, None, 0, 0, ctypes.byref(n)) == hv.HV_ERR_ARG
    assert L.hv_get_stats(None, None) == hv.HV_ERR_ARG
    assert L.hv_debug_inject(None, hv.HV_INJECT_FUSED_STALL) == hv.HV_ERR_ARG


def test_open_rejects_bad_descriptor_without_touching_a_device():
    d = hv.hv_open_desc(ctypes.sizeof(hv.hv_open_desc), 0, 256, 256, 12, 8, 0, 0, None)
    h = ctypes.c_void_p()
    assert hv.lib().hv_open(ctypes.byref(d), ctypes.byref(h)) == hv.HV_ERR_ARG
    assert "pixel_bits" in hv.hv_last_error(None)
    d = hv.hv_open_desc(ctypes.sizeof(hv.hv_open_desc), 0, 2048, 256, 16, 8, 0, 0, None)
    assert hv.lib().hv_open(ctypes.byref(d), ctypes.byref(h)) == hv.HV_ERR_ARG
    d = hv.hv_open_desc(12, 0, 256, 256, 16, 8, 0, 0, None)
    assert hv.lib().hv_open(ctypes.byref(d), ctypes.byref(h)) == hv.HV_ERR_ARG


def test_params_struct_layout():
    # offsets the C side relies on (natural alignment, doubles on 8 bytes)
    assert ctypes.sizeof(hv.hv_params) == 144
    assert hv.hv_params.z_m.offset == 24 and hv.hv_params.fs_hz.offset == 72
    assert hv.hv_params.highpass_cpp.offset == 128 and hv.hv_params.stft_kernel.offset == 136
    assert ctypes.sizeof(hv.hv_open_desc) == 40
