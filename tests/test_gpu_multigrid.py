"""The fused multigrid tail (the small coarse levels of a V-cycle in one thread-block cluster
kernel) performs the steps of the separate launches in the same order with the same node formulas;
only the compiler's fusion of multiply-adds may differ between the two kernels. So the preconditioner
agrees to FP32 rounding, the solver takes the same iterations (within one) and the state, adjoint and
sensitivities agree far inside the solver tolerance, for the V-cycle and its transpose."""

import numpy as np
import pytest

from synthetic import filtered_random

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc():
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300
    return paper_1904_00182_gb300


@pytest.mark.parametrize("shape,levels", [((32, 32, 32), 0), ((48, 40, 32), 4)])
def test_fused_tail_matches_launches(nc, shape, levels):
    nx, ny, nz = shape
    rho = filtered_random(nx, ny, nz, seed=9, volfrac=0.2)
    out = {}
    for tail in (0, 1 << 30):
        pb = nc.Problem(nx, ny, nz, 1.0 / nz, alpha=1e4, mg_levels=levels, mg_tail_nodes=tail)
        pb.set_design(rho)
        st = pb.solve_state()
        P, T, _ = pb.get_fields(velocity=False)
        f, ast = pb.solve_adjoint()
        g = pb.sensitivities()
        out[tail] = (P.cpu().numpy(), T.cpu().numpy(), g.cpu().numpy(), st["krylov_its"], ast["krylov_its"])
        pb.close()
    a, b = out[0], out[1 << 30]
    assert abs(a[3] - b[3]) <= 1 and abs(a[4] - b[4]) <= 1
    for x, y, tol in zip(a[:3], b[:3], (1e-8, 1e-8, 1e-6)):
        assert np.linalg.norm(x - y) <= tol * np.linalg.norm(y)


@pytest.mark.parametrize("precision", [1, 0])
def test_large_coarse_matrix(nc, precision):
    """A coarsest matrix too large for the single-block shared-memory inverse (2 levels at 12^3: 588
    free DOFs) goes through the multi-launch Gauss-Jordan inverse; the state, objective and
    sensitivities match the oracle as with 3 levels (96 free DOFs, shared-memory inverse)."""
    import oracle
    n = 12
    rho = filtered_random(n, n, n, seed=6, volfrac=0.2)
    tol = 1e-8 if precision == 1 else 1e-6
    op = oracle.Problem(oracle.Mesh(n, n, n, 1.0 / n), oracle.Params(alpha=1e4, newton_rtol=1e-10))
    op.set_design(rho)
    op.solve_state()
    Po, To = op.fields()
    op.solve_adjoint()
    go = op.sensitivities()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    for levels in (2, 3):
        pb = nc.Problem(n, n, n, 1.0 / n, alpha=1e4, mg_levels=levels, precision=precision, newton_rtol=1e-10)
        pb.set_design(rho)
        st = pb.solve_state()
        assert st["rel_residual"] <= 1e-10
        P, T, _ = pb.get_fields(velocity=False)
        f, _ = pb.solve_adjoint()
        g = pb.sensitivities().cpu().numpy()
        assert rel(P.cpu().numpy(), Po) < tol and rel(T.cpu().numpy(), To) < tol
        assert f == pytest.approx(op.objective(), rel=tol)
        assert rel(g, go) < 1e-6
        pb.close()


def test_four_levels_at_64(nc):
    """64^3 with 4 levels (coarsest 8^3 elements, 1296 free DOFs: the multi-launch inverse and a
    coarse solve staged for up to 2048 rows) reaches the tolerance and agrees with 5 levels."""
    n = 64
    rho = filtered_random(n, n, n, seed=7, volfrac=0.2)
    out = {}
    for levels in (4, 5):
        pb = nc.Problem(n, n, n, 1.0 / n, alpha=1e4, mg_levels=levels, newton_rtol=1e-10)
        pb.set_design(rho)
        st = pb.solve_state()
        assert st["rel_residual"] <= 1e-10
        P, T, _ = pb.get_fields(velocity=False)
        f, ast = pb.solve_adjoint()
        g = pb.sensitivities()
        out[levels] = (P.cpu().numpy(), T.cpu().numpy(), g.cpu().numpy(), f)
        pb.close()
    for x, y in zip(out[4][:3], out[5][:3]):
        assert np.linalg.norm(x - y) <= 1e-6 * np.linalg.norm(y)
    assert out[4][3] == pytest.approx(out[5][3], rel=1e-8)
