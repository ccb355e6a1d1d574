"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Sizes the oracle finishes in seconds: 16^3 (4096 elements, 32 blocks of the element kernels) and
a ragged 12 x 10 x 6 box. Tolerances: FP64 operators 1e-12 relative (only the summation order
differs), FP32 operators 1e-4, solved fields 1e-8 (FP64 path) / 1e-6 (mixed path) relative L2,
sensitivities 1e-6 relative L2 (the targets stated for this method's GPU path). The mixed path is
checked with its default precision assignment and with the fast one (double-float outer residuals,
FP32 Krylov basis); double-float operators are held to 1e-11.
"""

import numpy as np
import pytest

import oracle
from synthetic import filtered_random

pytestmark = pytest.mark.gpu

CASES = [((16, 16, 16), 1e3, 0), ((12, 10, 6), 1e4, 1)]


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


def make_pair(nc, shape, alpha, seed, precision=1, volfrac=0.2, rtol=1e-10, **kw):
    nx, ny, nz = shape
    h = 1.0 / nz
    rho = filtered_random(nx, ny, nz, seed, volfrac=volfrac)
    gp = nc.Problem(nx, ny, nz, h, alpha=alpha, precision=precision, newton_rtol=rtol, **kw)
    gp.set_design(rho)
    op = oracle.Problem(oracle.Mesh(nx, ny, nz, h), oracle.Params(alpha=alpha, newton_rtol=rtol))
    op.set_design(rho)
    return gp, op, rho


def random_state(op, seed):
    rng = np.random.default_rng(seed)
    n = op.mesh.n_nodes
    s = np.empty(2 * n)
    s[0::2] = 50.0 * rng.standard_normal(n)
    s[1::2] = 0.3 * rng.random(n)
    s[op.dir_mask] = 0.0
    return s


@pytest.mark.parametrize("shape,alpha,seed", CASES)
def test_design_fields(lib, shape, alpha, seed):
    gp, op, _ = make_pair(lib, shape, alpha, seed)
    gt, kap, k = [x.cpu().numpy() for x in gp.design_fields()]
    assert rel(gt, op.gamma_t) < 1e-10
    assert np.abs(gt - op.gamma_t).max() < 1e-10
    assert rel(kap, op.kappa) < 1e-9
    assert rel(k, op.k) < 1e-10
    gp.close()


@pytest.mark.parametrize("shape,alpha,seed", CASES)
def test_design_fields_both_filter_solvers(lib, shape, alpha, seed):
    """The filtered design from the spectral inner solve and from the Chebyshev one (both inside the
    FP64 refinement) equals the oracle's direct filter to 1e-10, and the two agree to 1e-10; the
    filter transpose through the sensitivities agrees between them to 1e-9."""
    out = {}
    for method in (lib.NC_FILTER_SPECTRAL, lib.NC_FILTER_CHEBYSHEV):
        gp, op, _ = make_pair(lib, shape, alpha, seed, filter_method=method)
        gt = gp.design_fields()[0].cpu().numpy()
        assert np.abs(gt - op.gamma_t).max() < 1e-10
        gp.solve_state()
        gp.solve_adjoint()
        out[method] = (gt, gp.sensitivities().cpu().numpy())
        gp.close()
    a, b = out[lib.NC_FILTER_SPECTRAL], out[lib.NC_FILTER_CHEBYSHEV]
    assert np.abs(a[0] - b[0]).max() < 1e-10
    assert rel(a[1], b[1]) < 1e-9


@pytest.mark.parametrize("shape,alpha,seed", CASES)
def test_residual(lib, shape, alpha, seed):
    gp, op, _ = make_pair(lib, shape, alpha, seed)
    for trial in range(2):
        s = random_state(op, 10 + trial)
        R, n2 = gp.eval_residual(s)
        Ro = op.residual(s)
        assert rel(R.cpu().numpy(), Ro) < 1e-12
        assert n2 == pytest.approx(np.dot(Ro[op.free], Ro[op.free]), rel=1e-12)
    gp.close()


@pytest.mark.parametrize("shape,alpha,seed", CASES)
def test_jacobian_products(lib, shape, alpha, seed):
    gp, op, _ = make_pair(lib, shape, alpha, seed)
    s = random_state(op, 3)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(s.shape)
    v[op.dir_mask] = 0.0
    expect = op.jvp_raw(s, v)
    expect[op.dir_mask] = 0.0
    j64 = gp.apply_jacobian(s, v, lib.NC_PREC_FP64).cpu().numpy()
    assert rel(j64, expect) < 1e-12
    j32 = gp.apply_jacobian(s, v, lib.NC_PREC_MIXED).cpu().numpy()
    assert rel(j32, expect) < 1e-4
    # transpose: (J_ff)^T w on the free rows
    w = rng.standard_normal(s.shape)
    w[op.dir_mask] = 0.0
    J = op.jacobian_full(s)
    f = op.free
    jt_expect = np.zeros_like(w)
    jt_expect[f] = J[f][:, f].T @ w[f]
    jt = gp.apply_jacobian_transpose(s, w).cpu().numpy()
    assert rel(jt, jt_expect) < 1e-12
    # adjoint identity on the GPU products alone
    assert np.dot(j64, w) == pytest.approx(np.dot(v, jt), rel=1e-11)
    gp.close()


@pytest.mark.parametrize("shape,alpha,seed", CASES)
def test_double_float_outer_operators(lib, shape, alpha, seed):
    """Mixed path, outer arithmetic double-float: R(s) and J(s)^T w against the FP64 oracle.
    A double-float sum errs by at most about 2 u^2 (|a| + |b|) with u = 2^-24, 64 times the FP64
    unit roundoff, so the FP64 operator bound (1e-12, summation order only) widens to 1e-11."""
    gp, op, _ = make_pair(lib, shape, alpha, seed, precision=lib.NC_PREC_MIXED, outer_arith=lib.NC_ARITH_DF64)
    for trial in range(2):
        s = random_state(op, 20 + trial)
        R, n2 = gp.eval_residual(s)
        Ro = op.residual(s)
        assert rel(R.cpu().numpy(), Ro) < 1e-11
        assert n2 == pytest.approx(np.dot(Ro[op.free], Ro[op.free]), rel=1e-11)
    s = random_state(op, 5)
    rng = np.random.default_rng(6)
    w = rng.standard_normal(s.shape)
    w[op.dir_mask] = 0.0
    J = op.jacobian_full(s)
    f = op.free
    jt_expect = np.zeros_like(w)
    jt_expect[f] = J[f][:, f].T @ w[f]
    jt = gp.apply_jacobian_transpose(s, w).cpu().numpy()
    assert rel(jt, jt_expect) < 1e-11
    gp.close()


# mixed path variants: the default (IEEE FP64 outer residuals and Krylov basis, frozen-coefficient
# finest multigrid level), the fast one (double-float outer residuals, FP32 Krylov basis) and the
# exact Jacobian on the finest multigrid level
VARIANTS = {"fp64": (1, 1e-8, {}), "mixed": (0, 1e-6, {}),
            "mixed_fp64_refinement": (0, 1e-6, {"adjoint_df64_steps": 0}),
            "mixed_fast": (0, 1e-6, {"outer_arith": 0, "krylov_basis": 1}),
            "mixed_exact_mg": (0, 1e-6, {"mg_op0": 0}),
            "mixed_exact_galerkin": (0, 1e-6, {"mg_galerkin": 0}),
            "mixed_coarse_sweeps": (0, 1e-6, {"mg_nu_coarse": 8, "nu_pre": 2}),
            "mixed_zline": (0, 1e-6, {"mg_smoother": 1}),
            "fp64_zline": (1, 1e-8, {"mg_smoother": 1})}


@pytest.mark.parametrize("shape,alpha,seed", CASES)
def test_adjoint_steering_residuals(lib, shape, alpha, seed):
    """Adjoint refinement residuals that only steer a correction run in double-float (their own
    kernel class); the residual that accepts lambda is FP64 and meets the tolerance. Lambda and the
    sensitivities agree with the all-FP64 refinement and with the oracle."""
    out = {}
    for steps in (0, 1):
        gp, op, rho = make_pair(lib, shape, alpha, seed, precision=0, adjoint_df64_steps=steps, adjoint_rtol=1e-10)
        gp.solve_state()
        gp.set_profiling(True)
        f, ast = gp.solve_adjoint()
        assert ast["rel_residual"] <= 1e-10
        out[steps] = (gp.adjoint().cpu().numpy(), gp.sensitivities().cpu().numpy(), gp.profile(), ast)
        gp.close()
    prof0, prof1 = out[0][2], out[1][2]
    assert prof0["adjoint_df64"][1] == 0 and prof1["adjoint_df64"][1] >= 1
    assert prof1["outer_op64"][1] >= 1            # the accepting residual
    assert rel(out[1][0], out[0][0]) < 1e-7
    assert rel(out[1][1], out[0][1]) < 1e-7
    op.solve_state()
    op.solve_adjoint()
    assert rel(out[1][1], op.sensitivities()) < 1e-6


@pytest.mark.parametrize("shape,alpha,seed", CASES)
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_state_adjoint_sensitivities(lib, shape, alpha, seed, variant):
    precision, tol, kw = VARIANTS[variant]
    gp, op, rho = make_pair(lib, shape, alpha, seed, precision=precision, **kw)
    stats = gp.solve_state()
    assert stats["rel_residual"] <= 1e-10
    op.solve_state()
    P, T, u = gp.get_fields()
    Po, To = op.fields()
    assert rel(P.cpu().numpy(), Po) < tol
    assert rel(T.cpu().numpy(), To) < tol
    assert rel(u.cpu().numpy(), op.velocities()) < tol
    f, ast = gp.solve_adjoint()
    assert f == pytest.approx(op.objective(), rel=tol)
    op.solve_adjoint()
    g = gp.sensitivities().cpu().numpy()
    go = op.sensitivities()
    assert rel(g, go) < 1e-6
    gp.close()


@pytest.mark.parametrize("shape,alpha,seed", CASES)
@pytest.mark.parametrize("precision,tol", [(1, 1e-8), (0, 1e-6)])
def test_supg_compliance_objective(lib, shape, alpha, seed, precision, tol):
    """Thermal compliance of Eq. objdiscr (SUPG-weighted source): value at the GPU state against the
    oracle (1e-12), and the objective, adjoint and sensitivities of the solved problem against the
    oracle's. The heated region gets the fluid permeability (kappa_s = kappa_f) so that its Darcy
    velocity, which the SUPG weights see, is not negligible."""
    nx, ny, nz = shape
    h = 1.0 / nz
    rho = filtered_random(nx, ny, nz, seed, volfrac=0.2)
    gp = lib.Problem(nx, ny, nz, h, alpha=alpha, precision=precision, newton_rtol=1e-10, kappa_ratio=1.0)
    op = oracle.Problem(oracle.Mesh(nx, ny, nz, h), oracle.Params(alpha=alpha, newton_rtol=1e-10, kappa_ratio=1.0))
    gp.set_design(rho)
    op.set_design(rho)
    gp.solve_state()
    op.solve_state()
    P, T, _ = gp.get_fields(velocity=False)
    s = np.empty(2 * op.mesh.n_nodes)
    s[0::2], s[1::2] = P.cpu().numpy(), T.cpu().numpy()
    f = gp.objective(lib.NC_OBJ_SUPG_COMPLIANCE)
    assert f == pytest.approx(op.supg_compliance(s), rel=1e-12)
    assert f == pytest.approx(op.supg_compliance(), rel=tol)
    fa, _ = gp.solve_adjoint(lib.NC_OBJ_SUPG_COMPLIANCE)
    assert fa == f
    lam_o = op.solve_adjoint("supg_compliance")
    assert rel(gp.adjoint().cpu().numpy(), lam_o) < 1e-6
    assert rel(gp.sensitivities().cpu().numpy(), op.sensitivities()) < 1e-6
    gp.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_other_parameters_and_warm_start(lib, precision):
    """Parameters off the defaults (3 heated layers, filter radius 1.5, alpha 1e5, conductivity
    ratio 10, RAMP q_c 0.881) on the ragged 12 x 10 x 6 box against the oracle, then a warm start
    (Sec. 5.4) from the solution of a neighbouring design reaching the same state as a cold start.
    At alpha = 1e5 the pressure (about -4e3, mostly hydrostatic) amplifies the stopping residual about
    1e3-fold in the state, so the FP64 path solves (GPU and oracle) to a relative residual of 1e-12 and
    is held to the 1e-8 state tolerance, the mixed path to 1e-10 and 1e-6; both are also held to the
    oracle's own residual at the GPU state."""
    nx, ny, nz = 12, 10, 6
    h = 1.0 / nz
    kw = dict(alpha=1e5, heated_layers=3, filter_radius=1.5, k_s=10.0, q_c=0.881)
    rho = filtered_random(nx, ny, nz, 4, volfrac=0.3)
    rtol = 1e-12 if precision == 1 else 1e-10
    tol = 1e-8 if precision == 1 else 1e-6
    gp = lib.Problem(nx, ny, nz, h, precision=precision, newton_rtol=rtol, **kw)
    op = oracle.Problem(oracle.Mesh(nx, ny, nz, h), oracle.Params(newton_rtol=rtol, **kw))
    gp.set_design(rho)
    op.set_design(rho)
    gt, _, _ = gp.design_fields()
    assert rel(gt.cpu().numpy(), op.gamma_t) < 1e-10
    gp.solve_state()
    op.solve_state()
    P, T, u = gp.get_fields()
    Po, To = op.fields()
    assert rel(P.cpu().numpy(), Po) < tol and rel(T.cpu().numpy(), To) < tol
    s = np.empty(2 * op.mesh.n_nodes)
    s[0::2], s[1::2] = P.cpu().numpy(), T.cpu().numpy()
    R = op.residual(s)
    assert np.linalg.norm(R[op.free]) <= (1e-11 if precision == 1 else 1e-9) * op.reference_norm()
    f, _ = gp.solve_adjoint()
    assert f == pytest.approx(op.objective(), rel=tol)
    op.solve_adjoint()
    assert rel(gp.sensitivities().cpu().numpy(), op.sensitivities()) < (1e-8 if precision == 1 else 1e-6)
    # warm start: solve a perturbed design cold, then return to rho starting from that state
    rho2 = np.clip(rho + 0.05 * np.random.default_rng(9).standard_normal(rho.size), 0.0, 1.0)
    gp.set_design(rho2)
    gp.solve_state()
    P2, T2, _ = gp.get_fields(velocity=False)
    gp.set_design(rho)
    gp.set_state(P2, T2)
    st = gp.solve_state()
    Pw, Tw, _ = gp.get_fields(velocity=False)
    assert rel(Pw.cpu().numpy(), Po) < tol and rel(Tw.cpu().numpy(), To) < tol
    assert st["rel_residual"] <= rtol
    gp.close()
