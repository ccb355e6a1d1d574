"""The frozen-coefficient element operator in the modal basis of the Q1 element (the form the FP32
multigrid kernels apply) equals its Gauss-point form, which the GPU tests check against the oracle's
frozen-coefficient operator: both are instantiated in FP64 on the host from nc_element.cuh
(tests/native/picard_modal_check.cpp) and compared on 200 random elements (size, materials, velocity,
tau, buoyancy, nodal values), operator and transpose, to 1e-13 of the largest output. The two forms
share only the element constants, so a wrong modal mass, stiffness or coupling entry, a sign, a
dropped term or a transposed coupling fails here."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_00182_gb300", "csrc")


def test_modal_form_equals_gauss_point_form(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir("/usr/local/cuda/include"):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "picard_modal_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I/usr/local/cuda/include", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "native", "picard_modal_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ALL OK" in r.stdout
