"""The frozen-coefficient (Picard) finest-level multigrid operator against the oracle's.

The kernel computes in FP32 from FP64 inputs, so it is held to the FP32 operator bound of the exact
Jacobian product (1e-4 relative L2). Both the operator and its transpose (the adjoint's multigrid) are
checked, on the base-plate set-up (16^3, ragged 12 x 10 x 6) and on the closed cavity of Sec. 6.1, at
random states whose Darcy velocities make the frozen convection matter.
"""

import numpy as np
import pytest

import oracle
from synthetic import filtered_random

pytestmark = pytest.mark.gpu

GEOM = dict(heat_nx=2, heat_ny=2, heated_layers=2, design_nx=6, design_ny=6, design_nz=10)
CASES = [((16, 16, 16), 1e3, 0, "top"), ((12, 10, 6), 1e4, 1, "top"), ((8, 8, 16), 1e5, 2, "cavity")]


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.fixture(scope="module")
def lib():
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300 as nc
    return nc


@pytest.mark.parametrize("shape,alpha,seed,bc", CASES)
def test_picard_operator_and_transpose(lib, shape, alpha, seed, bc):
    nx, ny, nz = shape
    h = 1.0 / nz
    rho = filtered_random(nx, ny, nz, seed, volfrac=0.2)
    geom = GEOM if bc == "cavity" else {}
    gp = lib.Problem(nx, ny, nz, h, alpha=alpha, bc=lib.NC_BC_CAVITY if bc == "cavity" else lib.NC_BC_TOP, **geom)
    op = oracle.Problem(oracle.Mesh(nx, ny, nz, h), oracle.Params(alpha=alpha, bc=bc, **geom))
    gp.set_design(rho)
    op.set_design(rho)
    rng = np.random.default_rng(seed + 10)
    n = op.mesh.n_nodes
    for trial in range(2):
        s = np.empty(2 * n)
        s[0::2] = 5.0 / op.par.kappa_f * rng.standard_normal(n)   # Darcy speeds of order one and above
        s[1::2] = rng.random(n)
        s[op.dir_mask] = 0.0
        v = rng.standard_normal(2 * n)
        v[op.dir_mask] = 0.0
        expect = op.picard_jvp_raw(s, v)
        expect[op.dir_mask] = 0.0
        got = gp.apply_picard(s, v).cpu().numpy()
        assert rel(got, expect) < 1e-4, rel(got, expect)
        A = op.picard_matrix_full(s)
        f = op.free
        et = np.zeros_like(v)
        et[f] = A[f][:, f].T @ v[f]
        gt = gp.apply_picard(s, v, transpose=True).cpu().numpy()
        assert rel(gt, et) < 1e-4, rel(gt, et)
        # the energy rows differ from the exact Jacobian's at such states (the test is not vacuous)
        jv = op.jvp_raw(s, v)
        jv[op.dir_mask] = 0.0
        assert rel(expect[1::2], jv[1::2]) > 1e-3
    gp.close()


@pytest.mark.parametrize("chunk", [4, 16])
def test_column_walking_kernels(lib, chunk):
    """The column-walking form of the FP32 finest-level kernels (elem_chunk > 0) gives the same exact
    Jacobian product and frozen-coefficient operator as the oracle, on a ragged grid whose height is not
    a multiple of the chunk."""
    nx, ny, nz = 12, 10, 6
    h = 1.0 / nz
    rho = filtered_random(nx, ny, nz, 3, volfrac=0.2)
    gp = lib.Problem(nx, ny, nz, h, alpha=1e4, elem_chunk=chunk)
    op = oracle.Problem(oracle.Mesh(nx, ny, nz, h), oracle.Params(alpha=1e4))
    gp.set_design(rho)
    op.set_design(rho)
    rng = np.random.default_rng(7)
    n = op.mesh.n_nodes
    s = np.empty(2 * n)
    s[0::2] = 5.0 / op.par.kappa_f * rng.standard_normal(n)
    s[1::2] = rng.random(n)
    s[op.dir_mask] = 0.0
    v = rng.standard_normal(2 * n)
    v[op.dir_mask] = 0.0
    jv = op.jvp_raw(s, v)
    jv[op.dir_mask] = 0.0
    assert rel(gp.apply_jacobian(s, v, lib.NC_PREC_MIXED).cpu().numpy(), jv) < 1e-4
    pv = op.picard_jvp_raw(s, v)
    pv[op.dir_mask] = 0.0
    assert rel(gp.apply_picard(s, v).cpu().numpy(), pv) < 1e-4
    A = op.picard_matrix_full(s)
    f = op.free
    et = np.zeros_like(v)
    et[f] = A[f][:, f].T @ v[f]
    assert rel(gp.apply_picard(s, v, transpose=True).cpu().numpy(), et) < 1e-4
    gp.close()
