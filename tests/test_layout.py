"""Index tables and shared-memory layouts of the kernels, checked on the host
(tests/layout_check.cu, compiled with nvcc): tree index tables consistent and
ordered by set size, every attach of the walk inside the held step tables,
pair-column indices inside their table, and the shared memory of the tuned
launch shapes small enough for the blocks per SM they were tuned for."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_layout_checks(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / "layout_check"
    cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_0908_4403_gb300", "csrc"),
           os.path.join(ROOT, "tests", "layout_check.cu"), "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    assert "layout checks: 0 failures" in r.stdout
