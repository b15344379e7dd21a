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


STRUCTS = ["heget_params", "heget_sampler", "heget_xsec_result", "heget_xsec_request", "heget_server_cfg",
           "heget_request", "heget_result"]


def test_binding_structs_match_the_c_layout(heget_lib, tmp_path):
    """Every ctypes struct of the binding has the size and field offsets the C
    compiler gives the header's struct."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "heget.h"', 'int main(void) {']
    for name in STRUCTS:
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in getattr(heget_lib, name)._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for name in STRUCTS:
        cls = getattr(heget_lib, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_server_calls_reject_null_arguments_without_gpu(heget_lib):
    lib = heget_lib.load()
    h = ctypes.c_void_p()
    assert lib.heget_server_start(None, None, ctypes.byref(h)) == heget_lib.HEGET_EINVAL
    q = heget_lib.heget_request(4, 32, 1, 0, 10, heget_lib.sampler_toy_pdf())
    t = ctypes.c_uint64()
    assert lib.heget_submit(None, ctypes.byref(q), ctypes.byref(t)) == heget_lib.HEGET_EINVAL
    r = heget_lib.heget_result()
    assert lib.heget_poll(None, 1, ctypes.byref(r)) == heget_lib.HEGET_EINVAL
    assert lib.heget_wait(None, 1, 0.01, ctypes.byref(r)) == heget_lib.HEGET_EINVAL
    assert lib.heget_server_stop(None) == heget_lib.HEGET_EINVAL


def test_distribution_and_sampling_calls_reject_null_context_without_gpu(heget_lib):
    """heget_hist and the helicity-sampling switch check their arguments on
    the host (no GPU needed for the refusals)."""
    H = heget_lib
    lib = H.load()
    spec = (H.heget_hist_spec * 1)(H.heget_hist_spec(H.HEGET_OBS_PT_MAX, 10, 0.0, 100.0))
    S = H.sampler_toy_pdf()
    assert lib.heget_hist(None, 4, 1, 0, 10, ctypes.byref(S), None, spec, 1, None, None) == H.HEGET_EINVAL
    assert b"context" in lib.heget_last_error()
    assert lib.heget_set_helicity_sampling(None, 1) == H.HEGET_EINVAL
    assert lib.heget_get_helicity_sampling(None) == -1
    assert H.hist_bins([(H.HEGET_OBS_PT, 10, 0.0, 1.0), (H.HEGET_OBS_DR, 4, 0.0, 4.0)]) == 2 * (12 + 6)
