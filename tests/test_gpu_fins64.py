"""64^3 fin-plate designs at alpha = 1e3, 1e4, 1e5: the FP64 path and the mixed-precision path
(FP32 multigrid inside FP64 FGMRES) both reach a relative residual of 1e-8, and their states agree
to 1e-6 (relative L2).

Too large for the oracle's direct solves, so the oracle checks each GPU state through its residual
on sampled nodes (|R_i| <= ||R_free|| <= 1e-8 ||R_free(0)|| on free rows). The multigrid has 5
levels here (4 levels, a 1296-DOF coarsest system, are checked against 5 in test_gpu_multigrid).
"""

import numpy as np
import pytest

import oracle
from synthetic import fin_plates

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 64


@pytest.fixture(scope="module")
def nc():
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300
    return paper_1904_00182_gb300


@pytest.mark.parametrize("alpha", [1e3, 1e4, 1e5])
def test_fins_fp64_vs_mixed(nc, alpha):
    rho = fin_plates(N, N, N, seed=11)
    op = oracle.Problem(oracle.Mesh(N, N, N, 1.0 / N), oracle.Params(alpha=alpha))
    op.set_design(rho)
    r0 = op.reference_norm()
    rng = np.random.default_rng(3)
    nodes = rng.choice(op.mesh.n_nodes, 400, replace=False)
    free = ~op.dir_mask.reshape(-1, 2)[nodes]
    states = {}
    for prec in (nc.NC_PREC_FP64, nc.NC_PREC_MIXED):
        pb = nc.Problem(N, N, N, 1.0 / N, alpha=alpha, mg_levels=5, newton_rtol=1e-8, precision=prec)
        pb.set_design(rho)
        st = pb.solve_state()
        P, T, _ = pb.get_fields(velocity=False)
        s = np.empty(2 * op.mesh.n_nodes)
        s[0::2], s[1::2] = P.cpu().numpy(), T.cpu().numpy()
        Rs = op.residual_at_nodes(s, nodes)
        worst = np.abs(Rs[free]).max() / r0
        print("alpha %.0e precision %d: %d Newton, %d Krylov, ramped %s, sampled |R|/R0 %.2e"
              % (alpha, prec, st["newton_its"], st["krylov_its"], st.get("ramped"), worst))
        assert worst <= 1e-8
        states[prec] = s
        pb.close()
    s64, s32 = states[nc.NC_PREC_FP64], states[nc.NC_PREC_MIXED]
    err = np.linalg.norm(s32 - s64) / np.linalg.norm(s64)
    print("alpha %.0e: mixed vs FP64 state rel L2 %.2e" % (alpha, err))
    assert err <= 1e-6
