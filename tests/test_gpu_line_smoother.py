"""The z-line block-Jacobi smoother kernels against a dense FP64 solve of every node column's
block-tridiagonal system (tests/native/line_smoother_check.cu, linked against the library's own
launchers): forward and transposed operator, first sweep from x = 0 and an update of a given x,
float and double, both boundary-condition sets, columns of 2 to 101 nodes (below, at and above the
solve's 32-node chunks).
The smoother's effect on whole solves (state, adjoint, sensitivities equal to the oracle's) is in
test_gpu_parity.py's z-line variants."""

import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_line_smoother_matches_dense_column_solves(tmp_path):
    from paper_1904_00182_gb300 import build
    build.build()
    lib = os.path.join(ROOT, "paper_1904_00182_gb300", "lib")
    exe = str(tmp_path / "line_smoother_check")
    subprocess.run([build._nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_1904_00182_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "line_smoother_check.cu"), "-L" + lib, "-lnatconv",
                    "-Xlinker", "-rpath", "-Xlinker", lib, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ALL OK" in r.stdout
    assert r.stdout.count(" ok") == 40
