"""Parity of the CUDA path with the oracle on the closed-cavity geometry (Sec. 6.1, quarter domain):
T = 0 on the outer walls and the top, P = 0 at the top outer corner, symmetry planes x = 0 and
y = 0, a heated box at the symmetry corner, a design box above it and passive fluid elsewhere.

Operators as in the top-cooled parity tests (FP64 1e-12, FP32 1e-4 relative); solved state,
objective and sensitivities 1e-8 on the FP64 path and 1e-6 on the mixed paths; the fused multigrid
tail against separate launches; a 16 x 16 x 32 solve (4 multigrid levels, fused tail) against the
oracle.
"""

import numpy as np
import pytest

import oracle
from synthetic import filtered_random

pytestmark = pytest.mark.gpu

GEOM = dict(heat_nx=2, heat_ny=2, heated_layers=2, design_nx=6, design_ny=6, design_nz=10)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def lib():
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300 as nc
    return nc


def make_pair(nc, shape, alpha, seed, precision=1, rtol=1e-10, geom=GEOM, **kw):
    nx, ny, nz = shape
    h = 1.0 / nz
    rho = filtered_random(nx, ny, nz, seed, volfrac=0.3)
    gp = nc.Problem(nx, ny, nz, h, alpha=alpha, precision=precision, newton_rtol=rtol, bc=nc.NC_BC_CAVITY,
                    **geom, **kw)
    gp.set_design(rho)
    op = oracle.Problem(oracle.Mesh(nx, ny, nz, h), oracle.Params(alpha=alpha, newton_rtol=rtol, bc="cavity", **geom))
    op.set_design(rho)
    return gp, op


def random_state(op, seed):
    rng = np.random.default_rng(seed)
    n = op.mesh.n_nodes
    s = np.empty(2 * n)
    s[0::2] = 50.0 * rng.standard_normal(n)
    s[1::2] = 0.3 * rng.random(n)
    s[op.dir_mask] = 0.0
    return s


SHAPE = (8, 8, 16)


def test_design_fields_and_operators(lib):
    gp, op = make_pair(lib, SHAPE, 1e4, 0)
    gt, kap, k = [x.cpu().numpy() for x in gp.design_fields()]
    assert np.abs(gt - op.gamma_t).max() < 1e-10
    assert np.all(gt[op.fluid] == 0.0) and np.all(gt[op.heated] == 1.0)
    assert rel(kap, op.kappa) < 1e-9 and rel(k, op.k) < 1e-10
    s = random_state(op, 1)
    R, n2 = gp.eval_residual(s)
    Ro = op.residual(s)
    assert rel(R.cpu().numpy(), Ro) < 1e-12
    assert n2 == pytest.approx(np.dot(Ro[op.free], Ro[op.free]), rel=1e-12)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(s.shape)
    expect = op.jvp_raw(s, np.where(op.dir_mask, 0.0, v))
    expect[op.dir_mask] = 0.0
    assert rel(gp.apply_jacobian(s, v, lib.NC_PREC_FP64).cpu().numpy(), expect) < 1e-12
    assert rel(gp.apply_jacobian(s, v, lib.NC_PREC_MIXED).cpu().numpy(), expect) < 1e-4
    w = rng.standard_normal(s.shape)
    J = op.jacobian_full(s)
    f = op.free
    jt_expect = np.zeros_like(w)
    jt_expect[f] = J[f][:, f].T @ w[f]
    assert rel(gp.apply_jacobian_transpose(s, w).cpu().numpy(), jt_expect) < 1e-12
    gp.close()


VARIANTS = {"fp64": (1, 1e-8, {}), "mixed": (0, 1e-6, {}),
            "mixed_fast": (0, 1e-6, {"outer_arith": 0, "krylov_basis": 1}),
            "mixed_zline": (0, 1e-6, {"mg_smoother": 1, "omega": 0.7})}


@pytest.mark.parametrize("alpha", [1e3, 1e5])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_state_adjoint_sensitivities(lib, alpha, variant):
    precision, tol, kw = VARIANTS[variant]
    gp, op = make_pair(lib, SHAPE, alpha, 3, precision=precision, **kw)
    st = gp.solve_state()
    assert st["rel_residual"] <= 1e-10
    op.solve_state()
    P, T, u = gp.get_fields()
    Po, To = op.fields()
    assert rel(P.cpu().numpy(), Po) < tol and rel(T.cpu().numpy(), To) < tol
    assert rel(u.cpu().numpy(), op.velocities()) < tol
    Pn = P.cpu().numpy()
    assert Pn[-1] == 0.0                      # the pinned corner (nx, ny, nz) is the last node
    f, ast = gp.solve_adjoint()
    assert f == pytest.approx(op.objective(), rel=tol)
    op.solve_adjoint()
    g = gp.sensitivities().cpu().numpy()
    go = op.sensitivities()
    assert rel(g, go) < 1e-6
    assert np.all(g[op.passive] == 0.0)
    gp.close()


def test_fused_tail_matches_launches(lib):
    rho = filtered_random(16, 16, 32, 5, volfrac=0.3)
    out = {}
    geom = dict(heat_nx=2, heat_ny=2, heated_layers=2, design_nx=12, design_ny=12, design_nz=24)
    for tail in (0, 1 << 30):
        gp = lib.Problem(16, 16, 32, 1.0 / 32, alpha=1e4, bc=lib.NC_BC_CAVITY, mg_tail_nodes=tail, **geom)
        gp.set_design(rho)
        st = gp.solve_state()
        P, T, _ = gp.get_fields(velocity=False)
        f, ast = gp.solve_adjoint()
        g = gp.sensitivities()
        out[tail] = (P.cpu().numpy(), T.cpu().numpy(), g.cpu().numpy(), st["krylov_its"], ast["krylov_its"])
        gp.close()
    a, b = out[0], out[1 << 30]
    assert abs(a[3] - b[3]) <= 1 and abs(a[4] - b[4]) <= 1
    for x, y, tol in zip(a[:3], b[:3], (1e-8, 1e-8, 1e-6)):
        assert np.linalg.norm(x - y) <= tol * np.linalg.norm(y)
    # against the oracle at this size
    op = oracle.Problem(oracle.Mesh(16, 16, 32, 1.0 / 32), oracle.Params(alpha=1e4, bc="cavity", **geom))
    op.set_design(rho)
    op.solve_state()
    Po, To = op.fields()
    assert rel(b[0], Po) < 1e-6 and rel(b[1], To) < 1e-6
    op.solve_adjoint()
    assert rel(b[2], op.sensitivities()) < 1e-6


def test_parameters_and_errors(lib):
    with pytest.raises(lib.NatConvError):
        lib.Problem(8, 8, 16, 1.0 / 16, bc=lib.NC_BC_CAVITY, heat_nx=9)
    with pytest.raises(lib.NatConvError):
        lib.Problem(8, 8, 16, 1.0 / 16, bc=7)
    gp = lib.Problem(8, 8, 16, 1.0 / 16, bc=lib.NC_BC_CAVITY, **GEOM)
    with pytest.raises(lib.NatConvError):
        gp.set_params(bc=lib.NC_BC_TOP)
    gp.close()


@pytest.mark.parametrize("smoother", [0, 1])
def test_cylinder_regions(lib, smoother):
    """Sec. 7's suspended cylinder on the quarter cavity (12 x 12 x 24; heat radius 4, design radius 9,
    layers 8-13): filtered design, state, both objectives and sensitivities against the oracle on the
    mixed path, with block-Jacobi and with z-line smoothing of the coarse multigrid levels."""
    geom = dict(heat_radius=4.0, design_radius=9.0, heat_z0=8, heated_layers=6, Q=100.0)
    n, nz = 12, 24
    rho = filtered_random(n, n, nz, 2, volfrac=0.3)
    gp = lib.Problem(n, n, nz, 1.0 / nz, alpha=1e4, precision=0, newton_rtol=1e-10, bc=lib.NC_BC_CAVITY,
                     region_shape=lib.NC_REGION_CYLINDER, mg_smoother=smoother, **geom)
    gp.set_design(rho)
    op = oracle.Problem(oracle.Mesh(n, n, nz, 1.0 / nz),
                        oracle.Params(alpha=1e4, newton_rtol=1e-10, bc="cavity", region_shape="cylinder", **geom))
    op.set_design(rho)
    gt = gp.design_fields()[0].cpu().numpy()
    assert np.abs(gt - op.gamma_t).max() < 1e-10
    st = gp.solve_state()
    assert st["rel_residual"] <= 1e-10
    op.solve_state()
    P, T, _ = gp.get_fields(velocity=False)
    Po, To = op.fields()
    assert rel(P.cpu().numpy(), Po) < 1e-6 and rel(T.cpu().numpy(), To) < 1e-6
    assert gp.objective(lib.NC_OBJ_SUPG_COMPLIANCE) == pytest.approx(op.supg_compliance(), rel=1e-6)
    f, _ = gp.solve_adjoint()
    assert f == pytest.approx(op.objective(), rel=1e-6)
    op.solve_adjoint()
    g = gp.sensitivities().cpu().numpy()
    assert rel(g, op.sensitivities()) < 1e-6
    assert np.all(g[op.passive] == 0.0) and np.abs(g[op.design]).max() > 0
    gp.close()
