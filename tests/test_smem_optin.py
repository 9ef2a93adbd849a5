"""The dynamic shared memory opt-in of the kernels is tracked per (kernel,
device) and is thread-safe: the bookkeeping header is compiled with the host
compiler into a small check program (no GPU involved) and run."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_smem_optin_tracks_each_device_apart(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "smem_optin_check")
    src = os.path.join(ROOT, "tests", "smem_optin_check.cpp")
    inc = os.path.join(ROOT, "paper_1406_4519_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I", inc, src, "-o", exe], check=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "ALL OK" in res.stdout
