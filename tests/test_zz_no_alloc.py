"""The allocation-free norm entry point against the library's existing residual-norm entry point.

nc_norm2_free_noalloc serves callers that cannot allocate device memory on this path (memory
handed out from their own pool, a hard budget, or no cudaMalloc/cudaFree because those can
synchronise the device). It must agree with the norm that nc_eval_residual reports, on two calls in
a row (the shared scratch array keeps the previous call's contents), for both boundary-condition
sets, on the legacy default stream and on another stream, without changing the device's free
memory, and reject grids whose partial sums would not fit its fixed scratch array. This file is
collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GEOM = dict(heat_nx=2, heat_ny=2, heated_layers=2, design_nx=6, design_ny=6, design_nz=10)


def _setup():
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300 as nc
    from paper_1904_00182_gb300 import _abi
    return nc, _abi, _abi.load_library()


def _call(lib, _abi, grid, bc, R, out, stream=None):
    st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    return lib.nc_norm2_free_noalloc(ctypes.byref(grid), bc, ctypes.c_void_p(R.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), st)


def test_noalloc_norm_matches_eval_residual():
    import torch
    nc, _abi, lib = _setup()
    from synthetic import filtered_random

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
        free0 = torch.cuda.mem_get_info()[0]
        assert _call(lib, _abi, grid, nc.NC_BC_TOP, R, out) == 0
        torch.cuda.synchronize()
        if call:   # the first call may load the library's device code (lazy module loading)
            assert torch.cuda.mem_get_info()[0] == free0     # nothing allocated on the device
        assert out.item() == pytest.approx(n2, rel=1e-12)
    # the same on a stream other than the legacy default one
    side = torch.cuda.Stream()
    out.zero_()
    torch.cuda.synchronize()
    assert _call(lib, _abi, grid, nc.NC_BC_TOP, R, out, side) == 0
    side.synchronize()
    assert out.item() == pytest.approx(n2, rel=1e-12)
    # sizes beyond the fixed scratch array, and unknown boundary conditions, are rejected before any
    # device work
    big = _abi.Grid(1023, 1023, 1023, 1e-3)
    assert _call(lib, _abi, big, nc.NC_BC_TOP, R, out) == 1
    assert _call(lib, _abi, grid, 7, R, out) == 1
    pb.close()


def test_noalloc_norm_cavity_skips_the_fixed_set():
    """Closed cavity (Sec. 6.1): for a state that meets the boundary conditions the norm equals the
    one nc_eval_residual reports; otherwise the fixed rows (which hold s there) are left out."""
    import torch
    nc, _abi, lib = _setup()
    from synthetic import filtered_random

    nx, ny, nz = 8, 8, 16
    pb = nc.Problem(nx, ny, nz, 1.0 / nz, alpha=1e4, bc=nc.NC_BC_CAVITY, **GEOM)
    pb.set_design(filtered_random(nx, ny, nz, seed=2, volfrac=0.3))
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    i, j, k = (a.transpose(2, 1, 0).ravel() for a in (i, j, k))     # node order: x fastest
    fixT = (i == nx) | (j == ny) | (k == nz)
    fixP = (i == nx) & (j == ny) & (k == nz)
    fixed = np.zeros(2 * pb.nn, dtype=bool)
    fixed[0::2], fixed[1::2] = fixP, fixT
    rng = np.random.default_rng(11)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    grid = _abi.Grid(nx, ny, nz, 1.0 / nz)
    for call in range(2):
        s = np.zeros(2 * pb.nn)
        s[0::2] = 30.0 * rng.standard_normal(pb.nn)
        s[1::2] = 0.3 * rng.random(pb.nn)
        s_bc = np.where(fixed, 0.0, s)
        R, n2 = pb.eval_residual(s_bc)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _call(lib, _abi, grid, nc.NC_BC_CAVITY, R, out) == 0
        torch.cuda.synchronize()
        if call:
            assert torch.cuda.mem_get_info()[0] == free0
        assert out.item() == pytest.approx(n2, rel=1e-12)
        # a state off the boundary conditions: the library's norm counts s^2 on the fixed rows
        R2, n2b = pb.eval_residual(s)
        torch.cuda.synchronize()
        assert _call(lib, _abi, grid, nc.NC_BC_CAVITY, R2, out) == 0
        torch.cuda.synchronize()
        expect = n2b - float(np.sum(s[fixed] ** 2))
        assert out.item() == pytest.approx(expect, rel=1e-10)
        Rh = R2.cpu().numpy()
        assert out.item() == pytest.approx(float(np.sum(Rh[~fixed] ** 2)), rel=1e-12)
    pb.close()
