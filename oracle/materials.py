"""Material interpolation and fluid-permeability tuning (test infrastructure only)."""

import numpy as np


def ramp_conductivity(gamma, k_f, k_s, q_c):
    """Eq. condRAMP (Sec. 5.2): k = k_f + gamma / (1 + q_c (1 - gamma)) (k_s - k_f).

    Returns (k, dk/dgamma). gamma = 1 is solid, gamma = 0 fluid (Sec. 2.2).
    """
    den = 1.0 + q_c * (1.0 - gamma)
    k = k_f + gamma / den * (k_s - k_f)
    dk = (k_s - k_f) * (1.0 + q_c) / den ** 2
    return k, dk


def ramp_permeability(gamma, kappa_f, kappa_s, q_p):
    """Eq. permRAMP (Sec. 5.2): kappa = kappa_s + (1 - gamma) / (1 + q_p gamma) (kappa_f - kappa_s).

    Returns (kappa, dkappa/dgamma).
    """
    den = 1.0 + q_p * gamma
    kappa = kappa_s + (1.0 - gamma) / den * (kappa_f - kappa_s)
    dkappa = -(kappa_f - kappa_s) * (1.0 + q_p) / den ** 2
    return kappa, dkappa


def kappa_f_tuned(alpha, dT=1.0, H=1.0, L=0.5, beta_m=1.0, nu=1.0, g=1.0, Pr=1.0):
    """Fluid permeability from equating the enclosure Nusselt correlations, Eq. nusselt5 (Sec. 3).

    kappa_f = beta_m H^1.74 / (nu^0.16 (g alpha dT)^0.42 L^2) * 0.0324 (Pr^2 / (0.2 + Pr))^0.58.
    The exponent of H is kept as printed (1.74); it has no effect for H = 1.
    """
    return (beta_m * H ** 1.74 / (nu ** 0.16 * (g * alpha * dT) ** 0.42 * L ** 2)
            * 0.0324 * (Pr ** 2 / (0.2 + Pr)) ** 0.58)


def nusselt_enclosure_fluid(alpha, dT, H, nu=1.0, g=1.0, Pr=1.0):
    """Eqs. nusselt1-2: Nu = 0.18 (Pr/(0.2+Pr) Ra_H)^0.29, Ra_H = g alpha dT H^3 / nu^2 * Pr."""
    Ra = g * alpha * dT * H ** 3 / nu ** 2 * Pr
    return 0.18 * (Pr / (0.2 + Pr) * Ra) ** 0.29


def nusselt_enclosure_porous(alpha, dT, H, L, kappa, beta_m=1.0, nu=1.0, g=1.0):
    """Eqs. nusselt3-4: Nu ~ (L/H) Ra^0.5, Ra = g alpha kappa H dT / (nu beta_m)."""
    Ra = g * alpha * kappa * H * dT / (nu * beta_m)
    return L / H * np.sqrt(Ra)
