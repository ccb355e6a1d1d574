"""Pins of the oracle's Jacobian, adjoint gradient and Newton convergence by finite differences.

Central differences with step 1e-6 (relative to the perturbed quantity's scale) against
the analytic element linearisation (including the derivatives of tau and N* with respect
to the state) and against the adjoint gradient through RAMP and the PDE filter.
"""

import numpy as np
import pytest

from oracle import Mesh, Params, Problem
from synthetic import filtered_random


@pytest.fixture(scope="module")
def solved():
    m = Mesh(5, 4, 6, 1.0 / 6.0)
    pr = Problem(m, Params(alpha=1e5, newton_rtol=1e-12))
    pr.set_design(filtered_random(5, 4, 6, seed=11, volfrac=0.2))
    pr.solve_state()
    return pr


def test_jacobian_matches_central_differences(solved):
    pr = solved
    rng = np.random.default_rng(1)
    # a state away from the solution, with large velocities so tau switches regime
    s = pr.s * (1.0 + 0.3 * rng.standard_normal(pr.s.shape))
    s[1::2] += 0.2 * rng.random(pr.mesh.n_nodes)
    J = pr.jacobian_full(s)
    for trial in range(3):
        v = rng.standard_normal(s.shape)
        v[0::2] *= np.abs(s[0::2]).max()
        v[1::2] *= np.abs(s[1::2]).max()
        eps = 1e-6
        fd = (pr.residual_raw(s + eps * v) - pr.residual_raw(s - eps * v)) / (2 * eps)
        Jv = J @ v
        assert np.linalg.norm(Jv - fd) <= 1e-6 * np.linalg.norm(fd)
        assert np.allclose(pr.jvp_raw(s, v), Jv, rtol=1e-12, atol=1e-12 * np.abs(Jv).max())


def test_design_derivatives_match_complex_step(solved):
    """dR_e/dkappa_e and dR_e/dk_e against complex-step derivatives of the element residual
    (Im R(x + i eps) / eps, free of cancellation; central differences lose all digits on
    the solid elements, where kappa ~ 1e-9 and dR/dkappa is large)."""
    pr = solved
    em = pr.em
    sl = slice(0, pr.mesh.n_elems)
    pe, te = pr.gather(pr.s, sl)
    kap, k, Qq = pr.kappa.copy(), pr.k.copy(), pr._Qq(sl)
    (dkP, dkT), (dcP, dcT) = em.design_derivatives(pe, te, kap, k, Qq)
    h = 1e-30
    RPk, RTk = em.residual(pe.astype(complex), te.astype(complex), kap + 1j * h * kap, k, Qq)
    RPc, RTc = em.residual(pe.astype(complex), te.astype(complex), kap, k + 1j * h * k, Qq)
    for got, cs, scale in ((dkP, RPk.imag / (h * kap[:, None]), None),
                           (dkT, RTk.imag / (h * kap[:, None]), None),
                           (dcP, RPc.imag / (h * k[:, None]), None),
                           (dcT, RTc.imag / (h * k[:, None]), None)):
        assert np.allclose(got, cs, rtol=1e-10, atol=1e-12 * (np.abs(cs).max() + 1e-300))
    assert np.abs(dkP).max() > 0 and np.abs(dcT).max() > 0
    assert np.all(dcP == 0.0)                    # conductivity does not enter the P rows


def test_gradient_matches_central_differences(solved):
    """df/dgamma from the adjoint (Sec. 5.1) against central differences of the full pipeline
    gamma -> filter -> RAMP -> Newton solve -> f, on seeded design entries."""
    pr = solved
    g0 = pr.gamma.copy()
    pr.set_design(g0)
    pr.solve_state()
    pr.solve_adjoint()
    grad = pr.sensitivities()
    rng = np.random.default_rng(5)
    design = np.flatnonzero(~pr.heated)
    picks = rng.choice(design, size=8, replace=False)
    eps = 1e-6
    for e in picks:
        vals = []
        for sgn in (1.0, -1.0):
            g = g0.copy()
            g[e] = np.clip(g[e] + sgn * eps, 0.0, 1.0)
            pr.set_design(g)
            pr.solve_state(rtol=1e-13)
            vals.append((pr.objective(), g[e]))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        assert grad[e] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(grad).max())
    # passive (heated) elements are not design variables: f does not depend on them
    assert np.all(grad[pr.heated] == 0.0)
    pr.set_design(g0)
    pr.solve_state()


def test_newton_converges_quadratically():
    """Exact Jacobian => quadratic convergence once close: r_{k+1} <= C r_k^2 with modest C."""
    m = Mesh(8, 8, 8, 1.0 / 8.0)
    pr = Problem(m, Params(alpha=1e5, newton_rtol=1e-13))
    pr.set_design(filtered_random(8, 8, 8, seed=2, volfrac=0.1))
    pr.solve_state()
    h = np.array(pr.history)
    assert h[-1] < 1e-12
    tail = [(h[i + 1], h[i]) for i in range(len(h) - 1) if 1e-11 < h[i + 1] and h[i] < 1e-1]
    assert tail, h
    for nxt, cur in tail:
        assert nxt <= 50.0 * cur ** 2, h
