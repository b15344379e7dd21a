"""The request server's first-fit device-arena allocator (heget_arena.h),
checked on the host against a byte-occupancy model (tests/arena_check.cpp):
aligned, disjoint, first-fit placements, merged free ranges, nothing lost."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_allocator(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "arena_check"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_0908_4403_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "arena checks: 0 failures" in r.stdout, r.stdout
