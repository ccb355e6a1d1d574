"""The two forms of the element routines agree: the Gauss-point form the FP64 kernels use and the
ScaleSums form of the FP32 and double-float kernels (the rows' constant factors applied to the 8
test sums), both instantiated in FP64 on the host from nc_element.cuh (tests/native/scale_sums_check.cpp):
residual, J v, J^T w with design derivatives and element-Jacobian columns on 100 random elements, to
1e-13 of the largest output. The GPU tests tie the FP64 form to the oracle at 1e-12, so this carries
that pin over to the other form."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_00182_gb300", "csrc")


def test_scale_sums_form_equals_gauss_point_form(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir("/usr/local/cuda/include"):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "scale_sums_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I/usr/local/cuda/include", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "native", "scale_sums_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ALL OK" in r.stdout
