"""Pins of the oracle's closed-cavity geometry (Sec. 6.1): the quarter of a closed cavity with
symmetry planes x = 0 and y = 0, T = 0 on the outer walls and the top, an insulated bottom, no
normal Darcy flow through any face and P = 0 at the top outer corner; a heated box at the symmetry
corner, a design box above it and passive fluid elsewhere.

* alpha = 0: the pressure equation has no source, so P = 0 and u = 0, the SUPG test function
  reduces to N and the temperature solves plain Q1 conduction. It is checked against a stiffness
  matrix and load assembled here from 1D Q1 element matrices by Kronecker products (exact for
  trilinear elements on a uniform grid).
* alpha = 1e3: the quarter solution equals the matching quarter of the mirrored full cavity (heat
  source centred, T = 0 on all four walls and the top, P = 0 at the four top corners), solved as a
  separate problem with explicit Dirichlet sets, which pins the natural (symmetry) boundary planes.
* The adjoint gradient of the mean heated-box temperature against central differences on design
  elements, and zero on passive elements.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import Mesh, Params, Problem

NX, NY, NZ, H = 4, 4, 8, 1.0 / 8.0


def _q1_1d(n, h):
    """1D Q1 mass and stiffness matrices on n elements of length h."""
    m = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    k = 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    M = np.zeros((n + 1, n + 1))
    K = np.zeros((n + 1, n + 1))
    for e in range(n):
        M[e:e + 2, e:e + 2] += m
        K[e:e + 2, e:e + 2] += k
    return M, K


def test_conduction_limit_matches_kronecker_assembly():
    m = Mesh(NX, NY, NZ, H)
    par = Params(alpha=0.0, kappa_f=1e-3, bc="cavity", heat_nx=2, heat_ny=1, heated_layers=2, Q=50.0,
                 newton_rtol=1e-13)
    pr = Problem(m, par)
    kc = 3.0
    pr.set_materials(1e-3, kc)
    pr.solve_state()
    P, T = pr.fields()
    assert np.abs(P).max() == 0.0 or np.abs(P).max() < 1e-12 * np.abs(T).max()
    Mx, Kx = _q1_1d(NX, H)
    My, Ky = _q1_1d(NY, H)
    Mz, Kz = _q1_1d(NZ, H)
    # node index i + NX1 * (j + NY1 * k): kron(z, kron(y, x))
    K = kc * (np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx)))
    # load Q int N over the heated box: element load h^3 / 8 per corner
    f = np.zeros(m.n_nodes)
    conn = m.connectivity()
    for e in np.flatnonzero(m.box_elems(2, 1, 0, 2)):
        f[conn[e]] += 50.0 * H ** 3 / 8.0
    _, maskT = m.cavity_dirichlet()
    free = np.flatnonzero(~maskT)
    Tk = np.zeros(m.n_nodes)
    Tk[free] = spla.spsolve(sp.csc_matrix(K[np.ix_(free, free)]), f[free])
    assert np.abs(T - Tk).max() <= 1e-10 * np.abs(Tk).max()
    assert np.abs(T[maskT]).max() == 0.0 and Tk.max() > 0.0


def test_quarter_matches_mirrored_full_cavity():
    hx, hy, hl, Q, alpha = 1, 2, 2, 200.0, 1e3
    mq = Mesh(NX, NY, NZ, H)
    pq = Problem(mq, Params(alpha=alpha, bc="cavity", heat_nx=hx, heat_ny=hy, heated_layers=hl, Q=Q,
                            newton_rtol=1e-12))
    rng = np.random.default_rng(3)
    gq = rng.random(mq.n_elems)
    pq.set_gamma_tilde(gq)
    pq.solve_state()
    Pq, Tq = pq.fields()

    mf = Mesh(2 * NX, 2 * NY, NZ, H)
    ijk = mf.node_ijk()
    maskT = (ijk[:, 0] == 0) | (ijk[:, 0] == 2 * NX) | (ijk[:, 1] == 0) | (ijk[:, 1] == 2 * NY) | (ijk[:, 2] == NZ)
    maskP = np.isin(ijk[:, 0], (0, 2 * NX)) & np.isin(ijk[:, 1], (0, 2 * NY)) & (ijk[:, 2] == NZ)
    e = mf.elem_ijk()
    iq = np.where(e[:, 0] >= NX, e[:, 0] - NX, NX - 1 - e[:, 0])     # mirror image in the quarter
    jq = np.where(e[:, 1] >= NY, e[:, 1] - NY, NY - 1 - e[:, 1])
    eq = iq + NX * (jq + NY * e[:, 2])
    heated_f = (iq < hx) & (jq < hy) & (e[:, 2] < hl)
    zeros = np.zeros(mf.n_nodes)
    pf = Problem(mf, Params(alpha=alpha, heated_layers=hl, Q=Q, newton_rtol=1e-12),
                 dirichlet=(maskP, zeros, maskT, zeros), Qe=np.where(heated_f, Q, 0.0))
    pf.set_gamma_tilde(gq[eq])
    pf.solve_state()
    Pf, Tf = pf.fields()
    nq = mq.node_ijk()
    nf = mf.node_index(nq[:, 0] + NX, nq[:, 1] + NY, nq[:, 2])
    assert np.abs(Tq - Tf[nf]).max() <= 1e-8 * np.abs(Tf).max()
    assert np.abs(Pq - Pf[nf]).max() <= 1e-8 * np.abs(Pf).max()
    assert np.abs(Pf).max() > 0 and np.abs(Tf).max() > 0
    # the mirrored field is symmetric about both centre planes
    nm = mf.node_index(2 * NX - nq[:, 0] - NX, nq[:, 1] + NY, nq[:, 2])
    assert np.abs(Tf[nm] - Tf[nf]).max() <= 1e-8 * np.abs(Tf).max()


def test_cavity_gradient_matches_central_differences():
    m = Mesh(NX, NY, NZ, H)
    par = Params(alpha=1e4, bc="cavity", heat_nx=1, heat_ny=1, heated_layers=1, design_nx=3, design_ny=3,
                 design_nz=5, newton_rtol=1e-12)
    pr = Problem(m, par)
    rng = np.random.default_rng(9)
    g0 = 0.2 + 0.6 * rng.random(m.n_elems)
    pr.set_design(g0)
    assert pr.fluid.sum() > 0 and pr.design.sum() == 3 * 3 * 5 - 0
    gt = pr.gamma_t
    assert np.all(gt[pr.heated] == 1.0) and np.all(gt[pr.fluid] == 0.0)
    pr.solve_state()
    pr.solve_adjoint()
    grad = pr.sensitivities()
    assert np.all(grad[pr.passive] == 0.0)
    picks = np.random.default_rng(2).choice(np.flatnonzero(pr.design), size=5, replace=False)
    eps = 1e-6
    for e in picks:
        vals = []
        for sgn in (1.0, -1.0):
            g = g0.copy()
            g[e] += sgn * eps
            pr.set_design(g)
            pr.solve_state(rtol=1e-13)
            vals.append(pr.objective())
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert grad[e] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(grad).max())
    # a passive element's design value changes nothing
    g = g0.copy()
    g[np.flatnonzero(pr.fluid)[0]] = 1.0 - g[np.flatnonzero(pr.fluid)[0]]
    pr.set_design(g)
    pr.solve_state(rtol=1e-13)
    f1 = pr.objective()
    pr.set_design(g0)
    pr.solve_state(rtol=1e-13)
    assert f1 == pytest.approx(pr.objective(), rel=1e-12)


def test_cylinder_regions_and_solution_symmetry():
    """Sec. 7's suspended cylinder (quarter domain): the voxelised heated cylinder and design annulus
    approach the quarter-disc areas, lie in the given layers and do not overlap; the solution is
    symmetric under the exchange x <-> y, which the quarter geometry and its boundary conditions keep."""
    n, nz = 12, 24
    m = Mesh(n, n, nz, 1.0 / nz)
    par = Params(alpha=1e4, bc="cavity", region_shape="cylinder", heat_radius=4.0, design_radius=9.0,
                 heat_z0=8, heated_layers=6, Q=100.0, newton_rtol=1e-12)
    pr = Problem(m, par)
    e = m.elem_ijk()
    assert np.all((e[pr.heated, 2] >= 8) & (e[pr.heated, 2] < 14)) and not np.any(pr.heated & pr.design)
    per_layer_h = pr.heated.sum() / 6
    per_layer_d = pr.design.sum() / 6
    assert abs(per_layer_h - np.pi * 16 / 4) < 0.2 * np.pi * 16 / 4
    assert abs(per_layer_h + per_layer_d - np.pi * 81 / 4) < 0.1 * np.pi * 81 / 4
    rng = np.random.default_rng(4)
    g = rng.random((nz, n, n))
    g = 0.5 * (g + g.transpose(0, 2, 1))                 # a design symmetric under x <-> y
    pr.set_design(g.ravel())
    pr.solve_state()
    P, T = pr.fields()
    Tn = T.reshape(nz + 1, n + 1, n + 1)
    Pn = P.reshape(nz + 1, n + 1, n + 1)
    assert np.abs(Tn - Tn.transpose(0, 2, 1)).max() <= 1e-9 * np.abs(Tn).max()
    assert np.abs(Pn - Pn.transpose(0, 2, 1)).max() <= 1e-9 * np.abs(Pn).max()
    assert pr.vol_h == pytest.approx(pr.heated.sum() / nz ** 3)
