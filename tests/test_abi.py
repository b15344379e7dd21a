"""The C-ABI library builds, loads and exports every symbol include/heget.h
declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "heget.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(heget_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_hot_path_calls():
    syms = declared_symbols()
    for s in ["heget_phase_space", "heget_amp2", "heget_xsec"]:
        assert s in syms


def test_library_exports_every_declared_symbol(heget_lib):
    lib = heget_lib.load()
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert missing == []
    # the binding covers every declared call
    assert set(declared_symbols()) <= set(heget_lib.SIGNATURES)


def test_version_and_error_paths_without_gpu(heget_lib):
    lib = heget_lib.load()
    assert b"sm_103a" in lib.heget_version()
    # NULL context and bad n are rejected before any CUDA call
    assert lib.heget_amp2(None, 4, 10, None, None, 32, None, None) == heget_lib.HEGET_EINVAL
    assert b"context" in lib.heget_last_error()
    s = heget_lib.sampler_fixed(500.0)
    r = heget_lib.heget_xsec_result()
    assert lib.heget_xsec(None, 4, 10, 1, ctypes.byref(s), 32, ctypes.byref(r), None) == heget_lib.HEGET_EINVAL
    assert lib.heget_sum(None, None, 0, None, None) == heget_lib.HEGET_EINVAL


def test_create_reports_missing_device_cleanly(heget_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = heget_lib.load().heget_create(0, ctypes.byref(h))
    assert st in (heget_lib.HEGET_ECUDA, heget_lib.HEGET_EINVAL)
    assert not h.value


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_0908_4403_gb300 import heget
    saved = heget._lib
    heget._lib = None
    try:
        with pytest.raises(ImportError):
            heget.load(str(tmp_path / "missing.so"))
    finally:
        heget._lib = saved
