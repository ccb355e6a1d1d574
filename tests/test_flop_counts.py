"""The algorithmic flop counts the library reports (nc_launch.h) are those of its element code.

The element arithmetic (nc_element.cuh) is compiled on the host with a counting number type
(tests/native/flop_count.cpp) and its additions and multiplications per element are compared with
the constants behind the ALU rooflines: FP32/FP64 kernels count adds + multiplies, double-float
kernels 11 FP32 flops per add and 10 per multiply.
"""

import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_00182_gb300", "csrc")


def _constants():
    src = open(os.path.join(CSRC, "nc_launch.h")).read()
    vals = {m.group(1): float(m.group(2)) for m in re.finditer(r"(kFlops\w+|kDf\w+) = ([0-9.]+)", src)}
    df = {m.group(1): (int(m.group(2)), int(m.group(3)))
          for m in re.finditer(r"(kFlops\w+DF) = (\d+) \* kDfAdd \+ (\d+) \* kDfMul", src)}
    return vals, df


def test_flop_constants_match_the_element_code(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir("/usr/local/cuda/include"):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "flop_count")
    subprocess.run([cxx, "-std=c++17", "-O0", "-I/usr/local/cuda/include", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "native", "flop_count.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    cnt = {ln.split()[0]: (int(ln.split()[1]), int(ln.split()[2])) for ln in out.strip().splitlines()}
    vals, df = _constants()
    tot = {k: a + m for k, (a, m) in cnt.items()}
    assert vals["kFlopsResidual"] == tot["residual"]
    assert vals["kFlopsState"] == tot["state"]
    assert vals["kFlopsJv"] == tot["jv"]
    assert vals["kFlopsJtv"] == tot["jtv"]
    assert vals["kFlopsSens"] == tot["sens"]
    assert vals["kFlopsJacColumn"] == tot["jac16"] / 16
    assert vals["kFlopsPicard"] == tot["picard"]
    assert vals["kFlopsPicardT"] == tot["picard_t"]
    assert df["kFlopsResidualDF"] == cnt["residual"]
    assert df["kFlopsStateDF"] == cnt["state"]
    assert df["kFlopsJtvDF"] == cnt["jtv"]
    assert df["kFlopsSensDF"] == cnt["sens"]
