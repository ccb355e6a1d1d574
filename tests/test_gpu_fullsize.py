"""Full-size checks at 128^3 in the launch configuration the benchmark times (mixed precision,
6 multigrid levels, alpha = 1e4, 20 % solid filtered-random design), for the default mixed path and
its fast variant (double-float outer residuals, FP32 Krylov basis).

The oracle cannot solve at this size, so it checks the GPU results through properties that hold at
any size, evaluated independently on the CPU:

* design fields: the oracle's filter (CG to 1e-14) and RAMP give the same gamma~, kappa and k;
* residual: the GPU's R(s) at a random state equals the oracle's element sums on sampled nodes;
* state: the oracle's residual at the GPU solution is below the stopping tolerance on sampled free
  rows (|R_i| <= ||R_free|| <= 1e-8 ||R_free(0)||), and the Dirichlet rows hold exactly;
* adjoint: the oracle's J(s)^T lambda at the GPU state and adjoint equals df/ds on sampled free rows
  to the adjoint tolerance;
* sensitivities: the oracle's chain rule (Sec. 5.1) from the GPU's s and lambda equals the GPU's
  gradient over every element (both FP64; only rounding and the filter tolerance differ);
* the FP64 path reaches the same state to 1e-6 (relative L2), the mixed-precision tolerance.
"""

import numpy as np
import pytest

import oracle
from synthetic import filtered_random

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 128
ALPHA = 1e4


@pytest.fixture(scope="module")
def base():
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300 as nc
    rho = filtered_random(N, N, N, seed=0, volfrac=0.2)
    op = oracle.Problem(oracle.Mesh(N, N, N, 1.0 / N), oracle.Params(alpha=ALPHA))
    op.set_design(rho)
    rng = np.random.default_rng(77)
    nn = op.mesh.n_nodes
    ijk = op.mesh.node_ijk()
    # sampled nodes: uniform, plus the heated layers (k <= 2), the lid (k = N) and the side walls
    nodes = np.unique(np.concatenate([
        rng.choice(nn, 300, replace=False),
        rng.choice(np.flatnonzero(ijk[:, 2] <= 2), 60, replace=False),
        rng.choice(np.flatnonzero(ijk[:, 2] >= N - 1), 60, replace=False),
        rng.choice(np.flatnonzero((ijk[:, 0] == 0) | (ijk[:, 1] == N)), 60, replace=False)]))
    return nc, op, rho, nodes


@pytest.fixture(scope="module", params=["mixed", "mixed_fast"])
def setup(base, request):
    nc, op, rho, nodes = base
    kw = {} if request.param == "mixed" else {"outer_arith": nc.NC_ARITH_DF64, "krylov_basis": nc.NC_BASIS_FP32}
    pb = nc.Problem(N, N, N, 1.0 / N, alpha=ALPHA, mg_levels=6, precision=nc.NC_PREC_MIXED, **kw)
    pb.set_design(rho)
    yield nc, op, pb, rho, nodes
    pb.close()


def _free_rows(op, nodes):
    return ~op.dir_mask.reshape(-1, 2)[nodes]


def test_design_fields_128(setup):
    nc, op, pb, rho, nodes = setup
    gt, kap, k = (a.cpu().numpy() for a in pb.design_fields())
    assert np.abs(gt - op.gamma_t).max() <= 1e-10
    assert np.abs(kap - op.kappa).max() <= 1e-9 * op.kappa.max()
    assert np.abs(k - op.k).max() <= 1e-9 * op.k.max()


def test_residual_sampled_128(setup):
    nc, op, pb, rho, nodes = setup
    import torch
    rng = np.random.default_rng(5)
    s = 1e-2 * rng.standard_normal(2 * op.mesh.n_nodes)
    s[op.dir_mask] = 0.0
    R, _ = pb.eval_residual(torch.tensor(s, device=pb.device))
    R = R.cpu().numpy().reshape(-1, 2)[nodes]
    Ro = op.residual_at_nodes(s, nodes)
    free = _free_rows(op, nodes)
    tol = 1e-12 if pb.params.outer_arith == nc.NC_ARITH_FP64 else 1e-11   # double-float: 2^-48
    assert np.abs(R - Ro)[free].max() <= tol * np.abs(Ro[free]).max()


def test_state_adjoint_sensitivities_128(setup):
    nc, op, pb, rho, nodes = setup
    st = pb.solve_state()
    P, T, _ = pb.get_fields(velocity=False)
    s = np.empty(2 * op.mesh.n_nodes)
    s[0::2], s[1::2] = P.cpu().numpy(), T.cpu().numpy()
    free = _free_rows(op, nodes)

    # state: oracle residual at the GPU solution
    r0 = op.reference_norm()
    Rs = op.residual_at_nodes(s, nodes)
    print("128^3 mixed: %d Newton, %d Krylov; max sampled |R_free| / ||R_free(0)|| = %.2e"
          % (st["newton_its"], st["krylov_its"], np.abs(Rs[free]).max() / r0))
    assert np.abs(Rs[free]).max() <= 1e-8 * r0
    assert np.all(s[op.dir_mask] == 0.0)
    f = pb.objective()
    assert f == pytest.approx(op.objective(s), rel=1e-12)

    # adjoint: J(s)^T lambda = df/ds on sampled free rows
    pb.solve_adjoint()
    lam = pb.adjoint().cpu().numpy()
    d = op.objective_weights()
    Jt = op.jt_at_nodes(s, lam, nodes)
    dn = d.reshape(-1, 2)[nodes]
    resid = np.abs(Jt - dn)[free].max()
    print("128^3 adjoint: max sampled |J^T lam - df/ds| / ||df/ds|| = %.2e"
          % (resid / np.linalg.norm(d[op.free])))
    assert resid <= 1e-8 * np.linalg.norm(d[op.free])
    assert np.all(lam[op.dir_mask] == 0.0)

    # sensitivities from the same s and lambda, over every element
    g = pb.sensitivities().cpu().numpy()
    op.s, op.lam = s, lam
    go = op.sensitivities()
    err = np.linalg.norm(g - go) / np.linalg.norm(go)
    print("128^3 sensitivities vs the oracle's chain rule: rel L2 %.2e" % err)
    assert err <= 1e-9


def test_fp64_path_agrees_128(setup):
    nc, op, pb, rho, nodes = setup
    if pb.params.krylov_basis != nc.NC_BASIS_FP64:
        pytest.skip("compared once, for the default mixed path")
    pb.set_design(rho)
    pb.solve_state()
    Pm, Tm, _ = pb.get_fields(velocity=False)
    p64 = nc.Problem(N, N, N, 1.0 / N, alpha=ALPHA, mg_levels=6, precision=nc.NC_PREC_FP64)
    p64.set_design(rho)
    st = p64.solve_state()
    P, T, _ = p64.get_fields(velocity=False)
    p64.close()
    s = np.empty(2 * op.mesh.n_nodes)
    s[0::2], s[1::2] = P.cpu().numpy(), T.cpu().numpy()
    r0 = op.reference_norm()
    Rs = op.residual_at_nodes(s, nodes)
    assert np.abs(Rs[_free_rows(op, nodes)]).max() <= 1e-8 * r0
    sm = np.empty_like(s)
    sm[0::2], sm[1::2] = Pm.cpu().numpy(), Tm.cpu().numpy()
    err = np.linalg.norm(sm - s) / np.linalg.norm(s)
    print("128^3 FP64 path: %d Newton, %d Krylov; mixed vs FP64 state rel L2 %.2e"
          % (st["newton_its"], st["krylov_its"], err))
    assert err <= 1e-6


def test_state_256x128x128(base):
    """The workload's larger grid, 256 x 128 x 128 (4.2M elements), volume fraction 0.3, 6 levels
    (coarsest 8 x 4 x 4 elements, 360 DOFs): the oracle's residual at the GPU state on sampled rows
    is below the stopping tolerance."""
    nc = base[0]
    nx, ny, nz = 256, 128, 128
    rho = filtered_random(nx, ny, nz, seed=3, volfrac=0.3)
    op = oracle.Problem(oracle.Mesh(nx, ny, nz, 1.0 / nz), oracle.Params(alpha=ALPHA))
    op.set_design(rho)
    pb = nc.Problem(nx, ny, nz, 1.0 / nz, alpha=ALPHA, mg_levels=6)
    pb.set_design(rho)
    st = pb.solve_state()
    P, T, _ = pb.get_fields(velocity=False)
    pb.close()
    s = np.empty(2 * op.mesh.n_nodes)
    s[0::2], s[1::2] = P.cpu().numpy(), T.cpu().numpy()
    rng = np.random.default_rng(5)
    nodes = rng.choice(op.mesh.n_nodes, 400, replace=False)
    Rs = op.residual_at_nodes(s, nodes)
    worst = np.abs(Rs[_free_rows(op, nodes)]).max() / op.reference_norm()
    print("256x128x128: %d Newton, %d Krylov, %.1f ms; sampled |R_free| / ||R_free(0)|| = %.2e"
          % (st["newton_its"], st["krylov_its"], st["t_total_ms"], worst))
    assert worst <= 1e-8
