"""Element-level weak form of the stabilised Darcy-Boussinesq model (test infrastructure only).

Follows Appendix A of the paper:

* trilinear (Q1) shape functions N for both P and T (Eq. A.3 "p(x) = N(x)^T p_e");
* the weak form Eq. weakstable: Darcy/continuity rows
  ``R^P_a = int kappa/mu dN_a/dx_i (dP/dx_i + rho0 alpha g_i T)``, energy rows
  ``R^T_a = int N*_a (rho0 c_p u.grad T - Q) + int k grad N_a . grad T``,
  with the Darcy velocity u of Eq. finaldarcy ``u = -kappa/mu (grad P + rho0 alpha g T)``;
* the streamline-upwind test function ``N* = N + tau u0 . grad N`` (Eq. "N^* = N + tau u_0^T B"),
  u0 taken at the element centroid, tau of Tezduyar type built from tau1 = h_e/(2|u0|) and
  tau3 = h_e^2/4 with h_e the element diagonal (the tau equation of App. A);
* the source load ``f_tQ,e = int N*^T Q`` (SUPG-weighted, App. A), and no boundary terms
  because the natural fluxes q_u = q_h = 0 in every setup used here.

Readings (where the paper is silent or garbled):

* quadrature: 2x2x2 Gauss-Legendre (exact for every product that appears except the
  convective term, which is cubic-by-quadratic);
* tau: the printed "(1/tau1^2 + 1/tau3^3)^(1/2)" is read as the Tezduyar combination
  ``tau = (tau1^-2 + tau3^-2)^(-1/2)``; tau3 = rho0 c_p h_e^2 / (4 k_f), which is the printed
  h_e^2/4 for the paper's unit parameters;
* the element matrix P_t,e printed without kappa/mu is read with kappa/mu as in the weak form;
* the convective velocity in the T^2, T^3 terms is the Gauss-point Darcy velocity; the
  SUPG direction is u0 at the centroid.

Everything is vectorised over elements with NumPy einsum; arrays are FP64.
"""

import numpy as np

GAUSS = 1.0 / np.sqrt(3.0)


def corner_signs():
    """Reference coordinates (+-1) of the 8 local nodes, a = ax + 2 ay + 4 az; shape (8, 3)."""
    return np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
                     for a in range(8)], dtype=np.float64)


def shape_tables(h):
    """Q1 tables on a cube of edge h, 2x2x2 Gauss rule.

    Returns (N, D, w, N0, D0): N[q, a] = N_a(xi_q); D[q, a, i] = dN_a/dx_i at xi_q;
    w = Gauss weight times det J = (h/2)^3; N0[a], D0[a, i] at the centroid.
    """
    xa = corner_signs()
    xq = GAUSS * xa                      # Gauss points ordered like the corners
    f = 1.0 + xq[:, None, :] * xa[None, :, :]          # (q, a, 3): 1 + xi_q,i xi_a,i
    N = np.prod(f, axis=2) / 8.0
    D = np.empty((8, 8, 3))
    for i in range(3):
        others = [j for j in range(3) if j != i]
        D[:, :, i] = xa[None, :, i] * f[:, :, others[0]] * f[:, :, others[1]] / 8.0 * (2.0 / h)
    w = (h / 2.0) ** 3
    N0 = np.full(8, 1.0 / 8.0)
    D0 = xa / 8.0 * (2.0 / h)
    return N, D, w, N0, D0


class ElementModel:
    """Per-element residual and derivatives for the parameters of one problem.

    ``par`` needs: h, mu, rho0, cp, alpha, g, k_f (for tau3).
    """

    def __init__(self, par):
        self.p = par
        self.N, self.D, self.w, self.N0, self.D0 = shape_tables(par.h)
        self.he = np.sqrt(3.0) * par.h
        self.beta = par.rho0 * par.alpha * par.g          # g vector = (0, 0, -g)
        self.tau3 = par.rho0 * par.cp * self.he ** 2 / (4.0 * par.k_f)

    # ---- state at the Gauss points -------------------------------------------------------
    def gauss_state(self, pe, te, kappa):
        """Gauss-point and centroid quantities of the element states pe, te (E, 8)."""
        N, D = self.N, self.D
        c = (kappa / self.p.mu)[:, None]
        Tq = te @ N.T                                   # (E, q)
        Gq = np.einsum("qai,ea->eqi", D, pe)            # grad P at q
        Hq = np.einsum("qai,ea->eqi", D, te)            # grad T at q
        uq = -c[:, :, None] * Gq
        uq[:, :, 2] += c * self.beta * Tq               # -(kappa/mu)(grad P + rho0 alpha g T)
        T0 = te @ self.N0
        G0 = pe @ self.D0
        u0 = -c * G0
        u0[:, 2] += c[:, 0] * self.beta * T0
        tau = 1.0 / np.sqrt(4.0 * np.sum(u0 * u0, axis=1) / self.he ** 2 + self.tau3 ** -2)
        return dict(Tq=Tq, Gq=Gq, Hq=Hq, uq=uq, u0=u0, tau=tau)

    # ---- residual ---------------------------------------------------------------------------
    def residual(self, pe, te, kappa, k, Qq, fPq=None):
        """Element residual vectors (RP, RT), each (E, 8).

        Qq: heat source at the Gauss points (E, 8) (the source term of Eq. goveq, SUPG weighted
        like f_tQ,e); fPq: optional mass source of the continuity equation (E, 8), used only by
        manufactured-solution tests.
        """
        st = self.gauss_state(pe, te, kappa)
        N, D, w = self.N, self.D, self.w
        RP = -w * np.einsum("qai,eqi->ea", D, st["uq"])
        if fPq is not None:
            RP -= w * fPq @ N
        S = self.p.rho0 * self.p.cp * np.einsum("eqi,eqi->eq", st["uq"], st["Hq"]) - Qq
        Nstar = N[None] + st["tau"][:, None, None] * np.einsum("ei,qai->eqa", st["u0"], D)
        RT = w * np.einsum("eqa,eq->ea", Nstar, S)
        RT += w * k[:, None] * np.einsum("qai,eqi->ea", D, st["Hq"])
        return RP, RT

    def supg_load(self, pe, te, kappa, Qq):
        """f_tQ,e of Eq. objdiscr: sum_q w Q_q N*_a(q), (E, 8); depends on the state through u0, tau."""
        st = self.gauss_state(pe, te, kappa)
        Nstar = self.N[None] + st["tau"][:, None, None] * np.einsum("ei,qai->eqa", st["u0"], self.D)
        return self.w * np.einsum("eqa,eq->ea", Nstar, Qq)

    # ---- directional derivative -------------------------------------------------------------
    def _dres(self, st, k, Qq, duq, du0, dHq, dk):
        """Linearised residual for given perturbations of u_q, u0, grad T_q and k."""
        N, D, w = self.N, self.D, self.w
        rc = self.p.rho0 * self.p.cp
        tau, u0 = st["tau"], st["u0"]
        dtau = -tau ** 3 * (4.0 / self.he ** 2) * np.sum(u0 * du0, axis=1)
        S = rc * np.einsum("eqi,eqi->eq", st["uq"], st["Hq"]) - Qq
        dS = rc * (np.einsum("eqi,eqi->eq", duq, st["Hq"]) + np.einsum("eqi,eqi->eq", st["uq"], dHq))
        u0D = np.einsum("ei,qai->eqa", u0, D)
        du0D = np.einsum("ei,qai->eqa", du0, D)
        Nstar = N[None] + tau[:, None, None] * u0D
        dNstar = dtau[:, None, None] * u0D + tau[:, None, None] * du0D
        dRP = -w * np.einsum("qai,eqi->ea", D, duq)
        dRT = w * (np.einsum("eqa,eq->ea", Nstar, dS) + np.einsum("eqa,eq->ea", dNstar, S))
        dRT += w * k[:, None] * np.einsum("qai,eqi->ea", D, dHq)
        if dk is not None:
            dRT += w * dk[:, None] * np.einsum("qai,eqi->ea", D, st["Hq"])
        return dRP, dRT

    def jvp(self, pe, te, kappa, k, Qq, dpe, dte):
        """Directional derivative of the element residual along (dpe, dte): J_e v_e."""
        st = self.gauss_state(pe, te, kappa)
        c = (kappa / self.p.mu)[:, None]
        dTq = dte @ self.N.T
        duq = -c[:, :, None] * np.einsum("qai,ea->eqi", self.D, dpe)
        duq[:, :, 2] += c * self.beta * dTq
        du0 = -c * (dpe @ self.D0)
        du0[:, 2] += c[:, 0] * self.beta * (dte @ self.N0)
        dHq = np.einsum("qai,ea->eqi", self.D, dte)
        return self._dres(st, k, Qq, duq, du0, dHq, None)

    def jacobian(self, pe, te, kappa, k, Qq):
        """Element Jacobian (E, 16, 16): rows (RP_0..7, RT_0..7), columns (p_0..7, t_0..7).

        Column b is the directional derivative along the unit vector e_b.
        """
        E = pe.shape[0]
        J = np.empty((E, 16, 16))
        for b in range(16):
            dp = np.zeros((E, 8))
            dt = np.zeros((E, 8))
            (dp if b < 8 else dt)[:, b % 8] = 1.0
            dRP, dRT = self.jvp(pe, te, kappa, k, Qq, dp, dt)
            J[:, :8, b] = dRP
            J[:, 8:, b] = dRT
        return J

    def design_derivatives(self, pe, te, kappa, k, Qq):
        """dR_e/dkappa_e and dR_e/dk_e, each as (dRP, dRT) of shape (E, 8)."""
        st = self.gauss_state(pe, te, kappa)
        dc = 1.0 / self.p.mu
        duq = -dc * st["Gq"].copy()
        duq[:, :, 2] += dc * self.beta * st["Tq"]
        du0 = -dc * (pe @ self.D0)
        du0[:, 2] += dc * self.beta * (te @ self.N0)
        zeros_H = np.zeros_like(st["Hq"])
        d_kappa = self._dres(st, k, Qq, duq, du0, zeros_H, None)
        d_k = self._dres(st, np.zeros_like(k), Qq, np.zeros_like(duq), np.zeros_like(du0),
                         zeros_H, np.ones_like(k))
        return d_kappa, d_k

    def picard_jvp(self, pe, te, kappa, k, dpe, dte):
        """Frozen-coefficient (Picard) linearisation of the element residual along (dpe, dte).

        Not a step of the paper's method: the library's multigrid may use this operator on its finest
        level as a cheaper stand-in for J (the outer Krylov solver is flexible, so the preconditioner
        may differ from J). Definition: the continuity rows exactly as in jvp (R^P is linear in the
        state); the energy rows with the convective velocity and the SUPG weight frozen at the
        element-constant centroid velocity u0 and tau of the state (pe, te), and no derivative of u,
        u0 or tau:  sum_q w [ N*_a(q) rho0 c_p u0 . grad dT_q + k grad N_a . grad dT_q ].
        """
        st = self.gauss_state(pe, te, kappa)
        c = (kappa / self.p.mu)[:, None]
        N, D, w = self.N, self.D, self.w
        dTq = dte @ N.T
        duq = -c[:, :, None] * np.einsum("qai,ea->eqi", D, dpe)
        duq[:, :, 2] += c * self.beta * dTq
        dRP = -w * np.einsum("qai,eqi->ea", D, duq)
        dHq = np.einsum("qai,ea->eqi", D, dte)
        u0, tau = st["u0"], st["tau"]
        conv = self.p.rho0 * self.p.cp * np.einsum("ei,eqi->eq", u0, dHq)
        Nstar = N[None] + tau[:, None, None] * np.einsum("ei,qai->eqa", u0, D)
        dRT = w * np.einsum("eqa,eq->ea", Nstar, conv)
        dRT += w * k[:, None] * np.einsum("qai,eqi->ea", D, dHq)
        return dRP, dRT

    def centroid_velocity(self, pe, te, kappa):
        """Darcy velocity u0 at each element centroid (E, 3), Eq. finaldarcy."""
        return self.gauss_state(pe, te, kappa)["u0"]
