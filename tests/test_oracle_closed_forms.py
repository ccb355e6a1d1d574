"""Pins of the oracle's state solve against closed-form solutions and exact invariants.

* uniform Darcy flow under a fixed pressure gradient (Eq. finaldarcy, linear P is exact in Q1);
* hydrostatic balance of a uniformly warm fluid (fixes the sign of the buoyancy term);
* linear and layered conduction without buoyancy (piecewise-linear T is exact in Q1);
* discrete divergence invariant of the pressure rows and the exact discrete energy balance
  at a converged convective solution;
* mirror symmetry of the solution.
"""

import numpy as np
import pytest

from oracle import Mesh, Params, Problem
from synthetic import filtered_random


def _dirichlet(mesh, maskP, valP, maskT, valT):
    return (maskP, valP, maskT, valT)


@pytest.mark.parametrize("axis", [0, 2])
def test_uniform_darcy_flow(axis):
    """alpha = 0, T = 0, uniform kappa; P fixed to G (L - x_axis) on the two faces normal to
    ``axis``. Exact: P linear, u = (kappa G / mu) e_axis in every element (Eq. finaldarcy)."""
    m = Mesh(4, 3, 5, 0.25)
    G, kappa, mu = 3.0, 0.3, 2.0
    X = m.node_coords()
    L = m.extent()[axis]
    faces = (np.isclose(X[:, axis], 0.0)) | (np.isclose(X[:, axis], L))
    valP = G * (L - X[:, axis])
    top = m.top_nodes()
    pr = Problem(m, Params(alpha=0.0, kappa_f=1.0, mu=mu),
                 dirichlet=_dirichlet(m, faces, valP, top, np.zeros(m.n_nodes)),
                 Qe=np.zeros(m.n_elems))
    pr.set_materials(kappa, 1.0)
    pr.solve_state(rtol=1e-13)
    P, T = pr.fields()
    assert np.allclose(P, G * (L - X[:, axis]), atol=1e-11)
    assert np.allclose(T, 0.0, atol=1e-13)
    u = pr.velocities()
    expect = np.zeros(3)
    expect[axis] = kappa * G / mu
    assert np.allclose(u, expect[None, :], atol=1e-11)


def test_hydrostatic_balance_fixes_buoyancy_sign():
    """Uniform T = T0 (all faces fixed, no source) with P = 0 on top: the exact state is at rest
    with P = -rho0 alpha g T0 (L_z - z), i.e. dP/dz = rho0 alpha g T0 for gravity along -z."""
    m = Mesh(3, 4, 5, 0.2)
    T0, alpha, rho0, g = 0.5, 2.0, 1.5, 0.8
    X = m.node_coords()
    ijk = m.node_ijk()
    bnd = ((ijk[:, 0] == 0) | (ijk[:, 0] == m.nx) | (ijk[:, 1] == 0) | (ijk[:, 1] == m.ny)
           | (ijk[:, 2] == 0) | (ijk[:, 2] == m.nz))
    top = m.top_nodes()
    pr = Problem(m, Params(alpha=alpha, kappa_f=1.0, rho0=rho0, g=g),
                 dirichlet=_dirichlet(m, top, np.zeros(m.n_nodes), bnd,
                                      np.full(m.n_nodes, T0)),
                 Qe=np.zeros(m.n_elems))
    pr.set_materials(0.7, 1.3)
    pr.solve_state(rtol=1e-13)
    P, T = pr.fields()
    Lz = m.extent()[2]
    assert np.allclose(T, T0, atol=1e-12)
    assert np.allclose(P, -rho0 * alpha * g * T0 * (Lz - X[:, 2]), atol=1e-10)
    assert np.allclose(pr.velocities(), 0.0, atol=1e-10)


def test_linear_and_layered_conduction():
    """alpha = 0, T = 1 at z = 0 and 0 at the top, insulated sides, Q = 0. With conductivity
    k_l in element layer l the exact T is piecewise linear with the series (harmonic) flux
    q = 1 / sum_l (h / k_l); Q1 reproduces it at the nodes."""
    m = Mesh(3, 2, 6, 1.0 / 6.0)
    ijk = m.node_ijk()
    bottom = ijk[:, 2] == 0
    top = ijk[:, 2] == m.nz
    maskT = bottom | top
    valT = np.where(bottom, 1.0, 0.0)
    k_layers = np.array([1.0, 100.0, 3.0, 0.5, 7.0, 1.0])
    k_e = k_layers[m.elem_ijk()[:, 2]]
    pr = Problem(m, Params(alpha=0.0, kappa_f=1.0),
                 dirichlet=_dirichlet(m, top, np.zeros(m.n_nodes), maskT, valT),
                 Qe=np.zeros(m.n_elems))
    pr.set_materials(1e-3, k_e)
    pr.solve_state(rtol=1e-13)
    _, T = pr.fields()
    q = 1.0 / np.sum(m.h / k_layers)
    plane_T = 1.0 - q * np.concatenate([[0.0], np.cumsum(m.h / k_layers)])
    assert np.allclose(T, plane_T[ijk[:, 2]], atol=1e-12)
    # uniform k: T = 1 - z / L_z
    pr.set_materials(1e-3, 2.0)
    pr.solve_state(rtol=1e-13)
    _, T = pr.fields()
    assert np.allclose(T, 1.0 - m.node_coords()[:, 2] / m.extent()[2], atol=1e-12)


@pytest.fixture(scope="module")
def convective_solution():
    m = Mesh(8, 6, 8, 1.0 / 8.0)
    pr = Problem(m, Params(alpha=1e5, newton_rtol=1e-12))
    pr.set_design(filtered_random(8, 6, 8, seed=3, volfrac=0.15))
    pr.solve_state()
    return pr


def test_divergence_invariant_of_pressure_rows(convective_solution):
    """The P rows are the weak divergence -int grad N_a . u_h. Their sum over all nodes vanishes
    for any state (partition of unity), so at convergence the P reactions on the open top face
    (the net mass flux through it) sum to zero."""
    pr = convective_solution
    Rraw = pr.residual_raw(pr.s)
    top = pr.mesh.top_nodes()
    scale = np.abs(Rraw[0::2]).max() + np.abs(pr.jvp_raw(pr.s, pr.s)[0::2]).max()
    assert abs(Rraw[0::2][top].sum()) < 1e-11 * scale
    assert np.abs(Rraw[0::2][~top]).max() < 1e-9 * scale
    # the invariant holds away from convergence too
    rng = np.random.default_rng(0)
    s = pr.s + 0.1 * rng.standard_normal(pr.s.shape) * np.abs(pr.s).max()
    assert abs(pr.residual_raw(s)[0::2].sum()) < 1e-11 * np.abs(pr.residual_raw(s)[0::2]).sum()


def test_exact_discrete_energy_balance(convective_solution):
    """Sum over nodes of the T rows is int (rho0 c_p u.grad T - Q) (the SUPG weights sum to 1).
    T_h vanishes on the top face, so it is a valid pressure test function and the converged P
    rows make int u_h . grad T_h = 0 with the same quadrature. Hence the heat leaving through
    the top (the T reactions there) equals the total source power (1) to solver accuracy,
    with convection present."""
    pr = convective_solution
    Rraw = pr.residual_raw(pr.s)
    top = pr.mesh.top_nodes()
    assert np.abs(pr.velocities()).max() > 1e-2          # convection is active
    total_power = np.sum(pr.Qe) * pr.mesh.h ** 3
    assert total_power == pytest.approx(1.0)
    assert Rraw[1::2][top].sum() == pytest.approx(-total_power, rel=1e-9)


def test_mirror_symmetry():
    """Mirroring the design in x (and y) mirrors P and T and flips u_x (u_y)."""
    m = Mesh(6, 5, 6, 1.0 / 6.0)
    g = filtered_random(6, 5, 6, seed=7, volfrac=0.2)
    base = Problem(m, Params(alpha=1e4, newton_rtol=1e-12))
    base.set_design(g)
    base.solve_state()
    P0, T0 = base.fields()
    u0 = base.velocities()
    shape_n = (m.nz + 1, m.ny + 1, m.nx + 1)
    shape_e = (m.nz, m.ny, m.nx)
    for ax_arr, comp in ((2, 0), (1, 1)):
        gm = g.reshape(shape_e)[(slice(None),) * ax_arr + (slice(None, None, -1),)].ravel()
        pr = Problem(m, Params(alpha=1e4, newton_rtol=1e-12))
        pr.set_design(gm)
        pr.solve_state()
        P1, T1 = pr.fields()
        flip = (slice(None),) * ax_arr + (slice(None, None, -1),)
        assert np.allclose(P1.reshape(shape_n)[flip].ravel(), P0, rtol=1e-9, atol=1e-12 * np.abs(P0).max())
        assert np.allclose(T1.reshape(shape_n)[flip].ravel(), T0, rtol=1e-9, atol=1e-14)
        u1 = pr.velocities().reshape(shape_e + (3,))[flip].reshape(-1, 3)
        u1[:, comp] *= -1
        assert np.allclose(u1, u0, atol=1e-9 * np.abs(u0).max())
