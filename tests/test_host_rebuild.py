"""The regrid's incremental layout build against a build from scratch (host
code only: the C++ check in native/ is compiled against the library's host
sources with the system compiler and run)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1703_03116_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


def test_incremental_build_equals_full_build(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "rebuild_check"
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", CUDA_INC, os.path.join(HERE, "native", "rebuild_check.cpp"),
                    os.path.join(CSRC, "forest.cpp"), "-o", str(exe), "-lpthread"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 different" in out.stdout
