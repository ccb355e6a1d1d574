"""The thermal compliance of Eq. objdiscr, f = sum_e f_tQ,e^T t_e with the SUPG-weighted source load
f_tQ,e (App. A), in the oracle.

Pins:
* with a zero Darcy velocity in the heated elements (uniform T, hydrostatic P) the SUPG weights
  reduce to N and f equals the Galerkin thermal compliance, i.e. the mean temperature times the
  total power (1);
* f equals minus the source part of the assembled T-residual dotted with t (the residual is pinned
  elsewhere): R^T(s; Q) - R^T(s; 0) = -f_tQ;
* the complex-step df/ds agrees with central differences of f;
* the adjoint gradient df/dgamma agrees with central differences of the whole pipeline, with the
  heated region given the fluid permeability (kappa_s = kappa_f) so that its velocity, and with it
  the SUPG part of f, is not negligible.
"""

import numpy as np
import pytest

from oracle import Mesh, Params, Problem
from synthetic import filtered_random


def _problem(kappa_ratio=1.0, alpha=1e5):
    m = Mesh(5, 4, 6, 1.0 / 6.0)
    pr = Problem(m, Params(alpha=alpha, kappa_ratio=kappa_ratio, newton_rtol=1e-12))
    pr.set_design(filtered_random(5, 4, 6, seed=11, volfrac=0.2))
    pr.solve_state()
    return pr


def test_zero_velocity_reduces_to_galerkin_compliance():
    pr = _problem()
    z = pr.mesh.node_ijk()[:, 2] * pr.mesh.h
    c = 0.7
    s = np.zeros(2 * pr.mesh.n_nodes)
    s[1::2] = c
    s[0::2] = pr.em.beta * c * (z - z.max())        # grad P = beta T e_z: u = 0 everywhere
    assert pr.supg_compliance(s) == pytest.approx(c, rel=1e-13)
    assert pr.supg_compliance(s) == pytest.approx(pr.objective(s), rel=1e-13)


def test_compliance_is_the_source_part_of_the_residual():
    pr = _problem()
    rng = np.random.default_rng(3)
    s = pr.s * (1.0 + 0.2 * rng.standard_normal(pr.s.shape))
    R_q = pr.residual_raw(s)
    Qe = pr.Qe.copy()
    pr.Qe = np.zeros_like(Qe)
    R_0 = pr.residual_raw(s)
    pr.Qe = Qe
    f_res = -float((R_q - R_0)[1::2] @ s[1::2])
    f = pr.supg_compliance(s)
    assert f == pytest.approx(f_res, rel=1e-12)
    assert abs(f - pr.objective(s)) > 1e-6 * abs(f)      # the SUPG part is present here


def test_weights_match_central_differences():
    pr = _problem()
    s = pr.s.copy()
    d = pr.supg_compliance_weights(s)
    rng = np.random.default_rng(4)
    free = pr.free
    for i in rng.choice(free, 12, replace=False):
        h = 1e-6 * max(1.0, abs(s[i]))
        sp, sm = s.copy(), s.copy()
        sp[i] += h
        sm[i] -= h
        fd = (pr.supg_compliance(sp) - pr.supg_compliance(sm)) / (2 * h)
        assert d[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(d).max())


def test_adjoint_gradient_matches_central_differences():
    pr = _problem()
    g0 = pr.gamma.copy()
    pr.solve_adjoint("supg_compliance")
    grad = pr.sensitivities()
    rng = np.random.default_rng(6)
    picks = rng.choice(np.flatnonzero(~pr.heated), size=6, replace=False)
    eps = 1e-6
    for e in picks:
        vals = []
        for sgn in (1.0, -1.0):
            g = g0.copy()
            g[e] = np.clip(g[e] + sgn * eps, 0.0, 1.0)
            pr.set_design(g)
            pr.solve_state(rtol=1e-13)
            vals.append((pr.supg_compliance(), g[e]))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        assert grad[e] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(grad).max())
    assert np.all(grad[pr.heated] == 0.0)
