"""The algorithmic flop counts the library reports (nc_launch.h) are those of its element code.

The element arithmetic (nc_element.cuh) is compiled on the host with a counting number type
(tests/native/flop_count.cpp) and its additions and multiplications per element are compared with
the constants behind the ALU rooflines: FP32/FP64 kernels count adds + multiplies, double-float
kernels 11 FP32 flops per add and 10 per multiply. The FP64 kernels use the element code's
Gauss-point form, the FP32 and double-float kernels its ScaleSums form.
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
    # FP64 kernels: the Gauss-point form
    assert vals["kFlopsResidual"] == tot["residual"]
    assert vals["kFlopsState"] == tot["state"]
    assert vals["kFlopsJv"] == tot["jv"]
    assert vals["kFlopsJtv"] == tot["jtv"]
    assert vals["kFlopsSens"] == tot["sens"]
    assert vals["kFlopsJacColumn"] == tot["jac16"] / 16
    # FP32 kernels: the ScaleSums form (row factors applied to the test sums)
    assert vals["kFlopsState"] == tot["state_sums"]
    assert vals["kFlopsJvS"] == tot["jv_sums"]
    assert vals["kFlopsJtvS"] == tot["jtv_sums"]
    assert vals["kFlopsJacColumnS"] == tot["jac16_sums"] / 16
    assert vals["kFlopsPicard"] == tot["picard_sums"] == tot["picard"]
    assert vals["kFlopsPicardT"] == tot["picard_t_sums"] == tot["picard_t"]
    assert vals["kFlopsPicardModal"] == tot["picard_modal"] < vals["kFlopsPicard"] / 2
    assert vals["kFlopsPicardModalT"] == tot["picard_modal_t"]
    # double-float kernels: the ScaleSums form
    assert df["kFlopsResidualDF"] == cnt["residual_sums"]
    assert df["kFlopsStateDF"] == cnt["state_sums"]
    assert df["kFlopsJtvDF"] == cnt["jtv_sums"]
    assert df["kFlopsSensDF"] == cnt["sens_sums"]
    # the ScaleSums form saves multiplications and no additions
    for k in ("residual", "jv", "jtv", "sens", "jac16"):
        assert cnt[k + "_sums"][0] == cnt[k][0] and cnt[k + "_sums"][1] < cnt[k][1]
