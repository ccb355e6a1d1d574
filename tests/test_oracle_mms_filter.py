"""Pins of the oracle by a manufactured solution (second-order convergence) and of the PDE
filter by its exact invariants and its damping of a smooth mode."""

import numpy as np
import pytest

from oracle import Mesh, Params, Problem
from oracle.element import GAUSS, corner_signs
from oracle.pde_filter import HelmholtzFilter

PI = np.pi


def _exact(X):
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    P = np.cos(PI * x) * np.sin(PI * y) * (z + 1.0)
    gP = np.stack([-PI * np.sin(PI * x) * np.sin(PI * y) * (z + 1.0),
                   PI * np.cos(PI * x) * np.cos(PI * y) * (z + 1.0),
                   np.cos(PI * x) * np.sin(PI * y)], axis=-1)
    lapP = -2.0 * PI ** 2 * np.cos(PI * x) * np.sin(PI * y) * (z + 1.0)
    sx, sy, sz = np.sin(PI * x), np.sin(PI * y), np.sin(PI * z)
    T = sx * sy * sz + (1.0 - z)
    gT = np.stack([PI * np.cos(PI * x) * sy * sz, PI * sx * np.cos(PI * y) * sz,
                   PI * sx * sy * np.cos(PI * z) - 1.0], axis=-1)
    lapT = -3.0 * PI ** 2 * sx * sy * sz
    return P, gP, lapP, T, gT, lapT


def _mms_errors(n, kappa=0.5, alpha=2.0, k=1.0):
    """Solve with the sources of the exact (P*, T*) and all-boundary Dirichlet data; return
    RMS nodal errors of P, T and the RMS centroid-velocity error."""
    m = Mesh(n, n, n, 1.0 / n)
    par = Params(alpha=alpha, kappa_f=1.0, newton_rtol=1e-12)
    beta = par.rho0 * alpha * par.g
    # Gauss-point coordinates of every element
    xq = (m.elem_ijk()[:, None, :] + 0.5 * (1.0 + GAUSS * corner_signs()[None, :, :])) * m.h
    P, gP, lapP, T, gT, lapT = _exact(xq)
    u = -kappa * gP
    u[..., 2] += kappa * beta * T
    dTdz = gT[..., 2]
    fP = -kappa * (lapP - beta * dTdz)                 # div u*
    fT = par.rho0 * par.cp * np.sum(u * gT, axis=-1) - k * lapT
    Xn = m.node_coords()
    Pn, _, _, Tn, _, _ = _exact(Xn)
    ijk = m.node_ijk()
    bnd = ((ijk == 0) | (ijk == np.array([m.nx, m.ny, m.nz]))).any(axis=1)
    pr = Problem(m, par, dirichlet=(bnd, Pn, bnd, Tn), Qe=np.zeros(m.n_elems), Qq_extra=fT,
                 fPq=fP)
    pr.set_materials(kappa, k)
    pr.solve_state()
    Ph, Th = pr.fields()
    Xc = m.elem_centroids()
    _, gPc, _, Tc, _, _ = _exact(Xc)
    uc = -kappa * gPc
    uc[:, 2] += kappa * beta * Tc
    rms = lambda a: np.sqrt(np.mean(a ** 2))
    return rms(Ph - Pn), rms(Th - Tn), rms(pr.velocities() - uc)


@pytest.mark.slow
def test_manufactured_solution_second_order():
    """Second-order convergence of P and T (and at least first order of u) over 6^3 -> 24^3.
    The SUPG scheme stays consistent: the dropped second-derivative term (App. A) vanishes
    for trilinear T with element-constant k."""
    errs = [_mms_errors(n) for n in (6, 12, 24)]
    for a, b in zip(errs[:-1], errs[1:]):
        rates = np.log2(np.array(a) / np.array(b))
        assert rates[0] > 1.8 and rates[1] > 1.8, rates
        assert rates[2] > 0.9, rates


def test_filter_preserves_constants_and_volume():
    m = Mesh(7, 5, 6, 0.1)
    f = HelmholtzFilter(m, 2.5)
    assert np.allclose(f.apply(np.full(m.n_elems, 0.37)), 0.37, rtol=1e-13)
    rng = np.random.default_rng(0)
    g = rng.random(m.n_elems)
    gt = f.apply(g)
    assert gt.sum() == pytest.approx(g.sum(), rel=1e-13)     # int gamma~ = int gamma
    assert gt.std() < g.std()


def test_filter_transpose_is_adjoint():
    m = Mesh(6, 6, 5, 0.2)
    f = HelmholtzFilter(m, 2.5)
    rng = np.random.default_rng(1)
    a = rng.random(m.n_elems)
    b = rng.random(m.n_elems)
    assert np.dot(f.apply(a), b) == pytest.approx(np.dot(a, f.apply_transpose(b)), rel=1e-13)


def test_filter_damps_a_smooth_mode_like_the_continuum():
    """-r^2 x'' + x = cos(k x) with Neumann ends has x = cos(k x) / (1 + r^2 k^2); the Q1
    solution agrees to O(h^2). R = 0.6 gives r = R/(2 sqrt 3) and a 1/(1 + r^2 pi^2) = 0.77
    damping at k = pi on the unit interval."""
    n = 64
    m = Mesh(n, 2, 2, 1.0 / n)
    R = 0.6
    f = HelmholtzFilter(m, R / m.h)
    xc = m.elem_centroids()[:, 0]
    kx = PI
    gt = f.apply(np.cos(kx * xc))
    r = R / (2.0 * np.sqrt(3.0))
    assert f.r == pytest.approx(r)
    expect = np.cos(kx * xc) / (1.0 + r * r * kx * kx)
    assert np.abs(gt - expect).max() < 2e-3
