"""The paper's own geometries on the paper's 160 x 160 x 320 mesh (Sec. 6.2 Table 4, Sec. 7).

* The closed cavity of Sec. 6.1 (quarter domain, heated box under a design box, passive fluid) at
  alpha = 1e3 from the initial design gamma = 0.05.
* The suspended cylinder of Sec. 7 (heated cylinder and design annulus, kappa_f = 0.000676) at
  alpha = 1e5 and at the paper's alpha = 1e6 (with the z-line smoother of presets.solver_settings),
  from a radial-fin initial design (volume fraction 0.15).

The oracle cannot solve at this size (8.2 M elements), so it checks the GPU's state and adjoint on
sampled rows, with the element materials the GPU's design pipeline produced (the filter and RAMP are
checked against the oracle's at 128^3 and on the cavity at 16 x 16 x 32): the oracle's residual at the
GPU state is below the stopping tolerance, and the oracle's J(s)^T lambda equals df/ds to the adjoint
tolerance, on nodes spread over the domain, the heated and design regions, the walls and the fixed
set. The residual at s = 0 (the stopping test's reference) is checked on the same rows.
"""

import numpy as np
import pytest

import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 160


def _oracle_params(kind, alpha, geom):
    if kind == "cavity":
        keys = ("Q", "heat_nx", "heat_ny", "heated_layers", "design_nx", "design_ny", "design_nz")
        return oracle.Params(alpha=alpha, bc="cavity", **{k: geom[k] for k in keys})
    return oracle.Params(alpha=alpha, bc="cavity", region_shape="cylinder", Q=geom["Q"], kappa_f=geom["kappa_f"],
                         heat_radius=geom["heat_radius"], design_radius=geom["design_radius"],
                         heat_z0=geom["heat_z0"], heated_layers=geom["heated_layers"])


@pytest.mark.parametrize("kind,alpha", [("cavity", 1e3), ("cylinder", 1e5), ("cylinder", 1e6)])
def test_paper_mesh_state_and_adjoint(kind, alpha):
    import torch
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300 as nc
    from paper_1904_00182_gb300.optimize import cavity_params, cylinder_params
    from paper_1904_00182_gb300.paper_runs import fin_design
    from paper_1904_00182_gb300.presets import solver_settings

    geom = cavity_params(N) if kind == "cavity" else cylinder_params(N)
    nx, ny, nz = N, N, 2 * N
    pb = nc.Problem(nx, ny, nz, 1.0 / nz, alpha=alpha, **geom, **solver_settings(alpha))
    if kind == "cavity":
        rho = torch.full((nx * ny * nz,), 0.05, dtype=torch.float64)
    else:
        rho = fin_design(N, pb.params)
    pb.set_design(rho)
    st = pb.solve_state()
    P, T, _ = pb.get_fields(velocity=False)
    _, kap, k = (a.cpu().numpy() for a in pb.design_fields())
    R0, n0 = pb.eval_residual(torch.zeros(2 * (nx + 1) * (ny + 1) * (nz + 1), dtype=torch.float64))
    R0 = R0.cpu().numpy()
    pb.solve_adjoint()
    lam = pb.adjoint().cpu().numpy()
    pb.close()

    op = oracle.Problem(oracle.Mesh(nx, ny, nz, 1.0 / nz), _oracle_params(kind, alpha, geom))
    op.set_materials(kap, k)
    s = np.empty(2 * op.mesh.n_nodes)
    s[0::2], s[1::2] = P.cpu().numpy(), T.cpu().numpy()
    ijk = op.mesh.node_ijk()
    rng = np.random.default_rng(11)
    near_heat = op.conn[op.heated].ravel()
    near_design = op.conn[op.design].ravel()
    walls = np.flatnonzero((ijk[:, 0] == nx) | (ijk[:, 1] == ny) | (ijk[:, 2] == nz) | (ijk[:, 2] == 0))
    nodes = np.unique(np.concatenate([rng.choice(op.mesh.n_nodes, 200, replace=False),
                                      rng.choice(near_heat, 100, replace=False),
                                      rng.choice(near_design, 100, replace=False),
                                      rng.choice(walls, 100, replace=False)]))
    free = ~op.dir_mask.reshape(-1, 2)[nodes]

    # the reference residual R(0) on the sampled rows
    Ro0 = op.residual_at_nodes(np.zeros_like(s), nodes)
    g0 = R0.reshape(-1, 2)[nodes]
    assert np.abs(g0 - Ro0)[free].max() <= 1e-12 * np.abs(Ro0[free]).max()
    r0 = np.sqrt(n0)

    # state: the oracle's residual at the GPU solution
    Rs = op.residual_at_nodes(s, nodes)
    worst = np.abs(Rs[free]).max() / r0
    print("%s %dx%dx%d alpha %g: %d Newton, %d Krylov, %.0f ms; sampled |R_free| / ||R_free(0)|| = %.2e"
          % (kind, nx, ny, nz, alpha, st["newton_its"], st["krylov_its"], st["t_total_ms"], worst))
    assert st["rel_residual"] <= 1e-8
    assert worst <= 1e-8
    assert np.all(s[op.dir_mask] == 0.0)

    # adjoint: J(s)^T lambda = df/ds on the sampled free rows
    d = op.objective_weights()
    Jt = op.jt_at_nodes(s, lam, nodes)
    resid = np.abs(Jt - d.reshape(-1, 2)[nodes])[free].max() / np.linalg.norm(d[op.free])
    print("%s adjoint: sampled |J^T lam - df/ds| / ||df/ds|| = %.2e" % (kind, resid))
    assert resid <= 1e-8
    assert np.all(lam[op.dir_mask] == 0.0)
