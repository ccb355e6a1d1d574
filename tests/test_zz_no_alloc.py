"""The allocation-free norm entry point against the library's existing residual-norm entry point.

nc_norm2_free_noalloc serves callers that cannot allocate device memory on this path (memory
handed out from their own pool, a hard budget, or no cudaMalloc/cudaFree because those can
synchronise the device). It must agree with the norm that nc_eval_residual reports, on two calls in
a row (the shared scratch array keeps the previous call's contents), and reject grids whose partial
sums would not fit its fixed scratch array. This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_norm_matches_eval_residual():
    import torch
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300 as nc
    from paper_1904_00182_gb300 import _abi
    from synthetic import filtered_random

    lib = _abi.load_library()
    n = 16
    pb = nc.Problem(n, n, n, 1.0 / n, alpha=1e4)
    pb.set_design(filtered_random(n, n, n, seed=4, volfrac=0.2))
    rng = np.random.default_rng(9)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    grid = _abi.Grid(n, n, n, 1.0 / n)
    for call in range(2):
        s = np.zeros(2 * pb.nn)
        s[0::2] = 30.0 * rng.standard_normal(pb.nn)
        s[1::2] = 0.2 * rng.random(pb.nn) * (call + 1)
        R, n2 = pb.eval_residual(s)              # existing entry point: R on the device and its norm
        torch.cuda.synchronize()
        status = lib.nc_norm2_free_noalloc(ctypes.byref(grid), ctypes.c_void_p(R.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), None)
        assert status == 0
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(n2, rel=1e-12)
    # sizes beyond the fixed scratch array are rejected before any device work
    big = _abi.Grid(1023, 1023, 1023, 1e-3)
    status = lib.nc_norm2_free_noalloc(ctypes.byref(big), ctypes.c_void_p(R.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert status == 1
    pb.close()
