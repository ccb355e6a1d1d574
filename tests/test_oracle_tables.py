"""Pins of the oracle's Q1 tables, RAMP and kappa_f against textbook values and the paper."""

import os

import numpy as np
import pytest

from oracle.element import ElementModel, corner_signs, shape_tables
from oracle.materials import (kappa_f_tuned, nusselt_enclosure_fluid, nusselt_enclosure_porous,
                              ramp_conductivity, ramp_permeability)
from oracle.solver import Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pair_class(a, b):
    """Number of reference coordinates in which corners a and b differ (0..3)."""
    return bin(a ^ b).count("1")


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_q1_stiffness_and_mass_closed_form(h):
    """Textbook Q1 cube matrices: K = h/12 [4, 0, -1, -1], M = h^3/216 [8, 4, 2, 1] by the
    number of coordinates in which the two corners differ (0, 1, 2, 3)."""
    N, D, w, _, _ = shape_tables(h)
    K = w * np.einsum("qai,qbi->ab", D, D)
    M = w * np.einsum("qa,qb->ab", N, N)
    kref = {0: 4.0, 1: 0.0, 2: -1.0, 3: -1.0}
    mref = {0: 8.0, 1: 4.0, 2: 2.0, 3: 1.0}
    for a in range(8):
        for b in range(8):
            c = _pair_class(a, b)
            assert K[a, b] == pytest.approx(h / 12.0 * kref[c], abs=1e-14)
            assert M[a, b] == pytest.approx(h ** 3 / 216.0 * mref[c], abs=1e-15)


def test_shape_function_identities():
    h = 0.5
    N, D, w, N0, D0 = shape_tables(h)
    assert np.allclose(N.sum(axis=1), 1.0)               # partition of unity
    assert np.allclose(D.sum(axis=1), 0.0)
    assert 8 * w == pytest.approx(h ** 3)
    # int_e dN_a/dx_i = xi_a,i h^2 / 4 (divergence theorem on one face)
    xa = corner_signs()
    assert np.allclose(w * D.sum(axis=0), xa * h * h / 4.0)
    # centroid values: N_a = 1/8, dN_a/dx_i = xi_a,i / (4 h)
    assert np.allclose(N0, 1.0 / 8.0)
    assert np.allclose(D0, xa / (4.0 * h))
    # N_a(xi_b) = delta_ab at the corners: interpolate the tables' polynomial at xi = corners
    f = 1.0 + xa[:, None, :] * xa[None, :, :]
    assert np.allclose(np.prod(f, axis=2) / 8.0, np.eye(8))


def test_ramp_endpoints_and_linear_limit():
    """Sec. 5.2: gamma = 1 solid, gamma = 0 fluid; q = 0 gives linear interpolation."""
    kf, ks, kaf, kas = 1.0, 100.0, 2e-3, 2e-9
    for q in (0.0, 0.881, 8.81, 881.0):
        k, _ = ramp_conductivity(np.array([0.0, 1.0]), kf, ks, q)
        assert k == pytest.approx([kf, ks])
        kap, _ = ramp_permeability(np.array([0.0, 1.0]), kaf, kas, q)
        assert kap == pytest.approx([kaf, kas], rel=1e-12)
    g = np.linspace(0, 1, 11)
    k, _ = ramp_conductivity(g, kf, ks, 0.0)
    assert np.allclose(k, kf + g * (ks - kf))
    kap, _ = ramp_permeability(g, kaf, kas, 0.0)
    assert np.allclose(kap, kas + (1 - g) * (kaf - kas))
    # penalisation: for q > 0 intermediate densities are less conductive / more permeable
    # than the linear mix (the purpose of RAMP stated in Sec. 5.2)
    k8, _ = ramp_conductivity(g[1:-1], kf, ks, 8.81)
    assert np.all(k8 < kf + g[1:-1] * (ks - kf))
    kap8, _ = ramp_permeability(g[1:-1], kaf, kas, 8.0)
    assert np.all(kap8 < kas + (1 - g[1:-1]) * (kaf - kas))


def test_ramp_derivatives_by_finite_differences():
    g = np.linspace(0.02, 0.98, 25)
    eps = 1e-6
    for q in (0.0, 8.81, 88.1):
        k, dk = ramp_conductivity(g, 1.0, 100.0, q)
        kp, _ = ramp_conductivity(g + eps, 1.0, 100.0, q)
        km, _ = ramp_conductivity(g - eps, 1.0, 100.0, q)
        assert np.allclose(dk, (kp - km) / (2 * eps), rtol=1e-7)
        kap, dkap = ramp_permeability(g, 3e-3, 3e-9, q)
        kapp, _ = ramp_permeability(g + eps, 3e-3, 3e-9, q)
        kapm, _ = ramp_permeability(g - eps, 3e-3, 3e-9, q)
        assert np.allclose(dkap, (kapp - kapm) / (2 * eps), rtol=1e-7)


def test_kappa_f_reproduces_table2_and_cylinder():
    """Eq. nusselt5 against Table 2 and the cylinder value of Sec. 7.2 (golden fixture).

    The printed values carry 3 significant digits and the last two Table 2 entries look
    truncated rather than rounded, so the bound is 3 %."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table2_kappa_f.txt"))
    for alpha, dT, L, printed in rows:
        val = kappa_f_tuned(alpha, dT=dT, H=1.0, L=L)
        assert abs(val - printed) / printed < 0.03, (alpha, val, printed)


@pytest.mark.parametrize("alpha", [1e3, 1e4, 1e5, 1e6])
def test_kappa_f_equates_the_two_nusselt_correlations(alpha):
    """Eq. nusselt5 is the kappa at which Eq. nusselt1 equals Eq. nusselt3 (H = 1): find that
    root independently by bisection on the two correlations and compare."""
    dT, H, L = 1.3, 1.0, 0.5
    lo, hi = 1e-12, 1.0
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if nusselt_enclosure_porous(alpha, dT, H, L, mid) < nusselt_enclosure_fluid(alpha, dT, H):
            lo = mid
        else:
            hi = mid
    assert kappa_f_tuned(alpha, dT=dT, H=H, L=L) == pytest.approx(np.sqrt(lo * hi), rel=1e-9)


def test_tau_limits():
    """App. A: tau combines the advective tau1 = h_e/(2|u0|) and diffusive tau3 = h_e^2/4
    limits; tau -> tau3 as |u0| -> 0 and tau*|u0| -> h_e/2 as |u0| -> infinity."""
    par = Params(alpha=1.0, kappa_f=1.0).resolved(type("M", (), {"h": 0.1})())
    em = ElementModel(par)
    he = np.sqrt(3.0) * 0.1
    pe = np.zeros((1, 8))
    te = np.zeros((1, 8))
    st = em.gauss_state(pe, te, np.array([1.0]))
    assert st["tau"][0] == pytest.approx(he ** 2 / 4.0, rel=1e-14)
    # a huge pressure gradient along x: u0 = -kappa dP/dx
    xa = corner_signs()
    pe = (1e9 * xa[:, 0] * 0.05)[None, :]
    st = em.gauss_state(pe, te, np.array([1.0]))
    speed = np.linalg.norm(st["u0"][0])
    assert speed == pytest.approx(1e9, rel=1e-12)
    assert st["tau"][0] * speed == pytest.approx(he / 2.0, rel=1e-9)
