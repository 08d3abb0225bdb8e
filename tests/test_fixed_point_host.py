"""The fixed-point arithmetic of the complex128 passes (fixed_point.cuh)
compiled as host C++ and checked against long-double arithmetic: conversions
between doubles and the tile's 64-bit units (round trip within one unit,
headroom, correct rounding), the Q1.62 table-and-series rotation (error
below 1e-15 relative), its cosine and sine rounded to doubles (the adjoint
kernel's rotation factor, within 2e-16), quarter turns."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2206_11664_gb300", "csrc")


def test_fixed_point_host(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = "/usr/local/cuda/include"
    exe = str(tmp_path / "fx_host_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", cuda_inc,
                           os.path.join(HERE, "fx_host_check.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
