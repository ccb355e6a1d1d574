"""Assembly, damped Newton, adjoint and sensitivities (test infrastructure only).

* Problem statement: Sec. 5.1, Eq. optprob (state equation R(s(gamma), gamma) = 0, s = [p; t]
  of Eq. finalsyseq).
* Design pipeline: PDE filter (Sec. 5.1), RAMP (Sec. 5.2, Eqs. condRAMP, permRAMP); the heated
  region Omega_h is solid and not designed (Sec. 2.2), so gamma and gamma~ are 1 there.
* Nonlinear solve: damped Newton whose damping factor minimises the L2 norm of the residual,
  stopping on a relative residual reduction, with source ramping on failure (Sec. 5.4).
  The paper does not say how the minimiser is found; the rule used here: the full step if it
  reduces phi = ||R||^2 by 1e-4 phi0, else the best of a parabola through phi(0), phi(1/2),
  phi(1) and those two points, else halving.
* Objective: the mean temperature over the heated region (Galerkin weights), the
  normalised thermal compliance of Eq. objfunc for a uniform source; and the discrete thermal
  compliance of Eq. objdiscr, sum_e f_tQ,e^T t_e with the SUPG-weighted source load (its state
  derivative by complex step; no explicit design derivative, since the source lies in the passive
  heated region).
* Adjoint: J^T lambda = df/ds on the free DOFs; sensitivities
  df/dgamma~_e = -lambda_e^T dR_e/dgamma~_e (Sec. 5.1 "adjoint sensitivity analysis"),
  then the filter transpose.

Linear systems are solved with SciPy's sparse direct solver (SuperLU). DOF numbering:
``2 * node + field`` with field 0 = P, 1 = T.
"""

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import ElementModel
from .materials import kappa_f_tuned, ramp_conductivity, ramp_permeability
from .mesh import Mesh
from .pde_filter import HelmholtzFilter


@dataclass
class Params:
    alpha: float = 1e3
    kappa_f: Optional[float] = None      # None: Eq. nusselt5 with dT = 1, H = 1, L = 0.5
    kappa_ratio: float = 1e-6            # kappa_s / kappa_f
    k_f: float = 1.0
    k_s: float = 100.0
    q_c: float = 8.81
    q_p: float = 8.0
    Q: Optional[float] = None            # None: total power 1 over the heated layers
    heated_layers: int = 2
    rho0: float = 1.0
    mu: float = 1.0
    cp: float = 1.0
    g: float = 1.0
    filter_radius: float = 2.5           # in element sizes
    newton_rtol: float = 1e-8
    newton_maxit: int = 50
    h: float = 1.0                       # set from the mesh
    # geometry: "top" (P = T = 0 on the top face) or "cavity" (Mesh.cavity_dirichlet); the heated box
    # (heat_nx, heat_ny) x heated_layers and the design box (design_nx, design_ny) x [heated_layers,
    # heated_layers + design_nz) at the corner x = y = 0 (None: the full extent); elements in neither
    # box are passive fluid
    bc: str = "top"
    heat_nx: Optional[int] = None
    heat_ny: Optional[int] = None
    design_nx: Optional[int] = None
    design_ny: Optional[int] = None
    design_nz: Optional[int] = None
    # region_shape "cylinder": heated cylinder of heat_radius and design annulus out to design_radius
    # (element sizes) about the z axis through x = y = 0, both over the layers [heat_z0, heat_z0 +
    # heated_layers); the box fields above are then unused
    region_shape: str = "box"
    heat_radius: float = 0.0
    design_radius: float = 0.0
    heat_z0: int = 0

    def resolved(self, mesh):
        kf = self.kappa_f if self.kappa_f else kappa_f_tuned(self.alpha)
        return replace(self, kappa_f=kf, h=mesh.h)


class NewtonFailure(RuntimeError):
    pass


class Problem:
    """One state problem on a structured grid.

    dirichlet: optional (maskP, valP, maskT, valT) over nodes; default P = T = 0 on the top face.
    Qe: optional per-element heat source overriding the heated-layer default.
    Qq_extra, fPq: optional Gauss-point sources (E, 8) for manufactured solutions.
    """

    CHUNK = 32768

    def __init__(self, mesh: Mesh, params: Params, dirichlet=None, Qe=None, Qq_extra=None,
                 fPq=None):
        self.mesh = mesh
        self.par = params.resolved(mesh)
        self.em = ElementModel(self.par)
        self.conn = mesh.connectivity()
        n = mesh.n_nodes
        if dirichlet is None:
            if self.par.bc == "top":
                top = mesh.top_nodes()
                dirichlet = (top, np.zeros(n), top, np.zeros(n))
            elif self.par.bc == "cavity":
                mP, mT = mesh.cavity_dirichlet()
                dirichlet = (mP, np.zeros(n), mT, np.zeros(n))
            else:
                raise ValueError("unknown bc")
        maskP, valP, maskT, valT = dirichlet
        self.dir_mask = np.zeros(2 * n, dtype=bool)
        self.dir_mask[0::2] = maskP
        self.dir_mask[1::2] = maskT
        self.dir_val = np.zeros(2 * n)
        self.dir_val[0::2] = np.where(maskP, valP, 0.0)
        self.dir_val[1::2] = np.where(maskT, valT, 0.0)
        self.free = np.flatnonzero(~self.dir_mask)
        par = self.par
        hl = par.heated_layers
        if par.region_shape == "cylinder":
            z0, z1 = par.heat_z0, par.heat_z0 + hl
            self.heated = mesh.cylinder_elems(par.heat_radius, z0, z1)
            self.design = mesh.cylinder_elems(par.design_radius, z0, z1, inner=par.heat_radius)
        elif par.region_shape == "box":
            self.heated = mesh.box_elems(par.heat_nx or mesh.nx, par.heat_ny or mesh.ny, 0, hl)
            self.design = mesh.box_elems(par.design_nx or mesh.nx, par.design_ny or mesh.ny, hl,
                                         hl + par.design_nz if par.design_nz else mesh.nz) & ~self.heated
        else:
            raise ValueError("unknown region_shape")
        self.passive = ~self.design                        # heated (solid) or passive fluid
        self.fluid = self.passive & ~self.heated
        vol_h = self.heated.sum() * mesh.h ** 3
        if Qe is None:
            Qval = self.par.Q if self.par.Q is not None else 1.0 / vol_h
            Qe = np.where(self.heated, Qval, 0.0)
        self.Qe = np.asarray(Qe, dtype=np.float64)
        self.Qq_extra = Qq_extra
        self.fPq = fPq
        self.q_scale = 1.0
        self.vol_h = vol_h
        self.filter = None
        self.kappa = None
        self.k = None

    # ---- design -> materials --------------------------------------------------------------
    def design_pipeline(self, gamma):
        """gamma (E) -> gamma~ (E): passive elements set (heated 1, fluid 0), PDE filter, passive set."""
        if self.filter is None:
            self.filter = HelmholtzFilter(self.mesh, self.par.filter_radius)
        passive_value = np.where(self.heated, 1.0, 0.0)
        g = np.where(self.passive, passive_value, gamma)
        gt = self.filter.apply(g)
        return np.where(self.passive, passive_value, gt)

    def set_design(self, gamma):
        gamma = np.asarray(gamma, dtype=np.float64)
        if gamma.shape != (self.mesh.n_elems,) or not np.all(np.isfinite(gamma)) \
                or gamma.min() < 0.0 or gamma.max() > 1.0:
            raise ValueError("design must be E finite values in [0, 1]")
        self.gamma = gamma
        self.gamma_t = self.design_pipeline(gamma)
        self.set_gamma_tilde(self.gamma_t)

    def set_gamma_tilde(self, gt):
        p = self.par
        kappa_s = p.kappa_ratio * p.kappa_f
        self.kappa, self.dkappa = ramp_permeability(gt, p.kappa_f, kappa_s, p.q_p)
        self.k, self.dk = ramp_conductivity(gt, p.k_f, p.k_s, p.q_c)

    def set_materials(self, kappa, k):
        self.kappa = np.asarray(kappa, dtype=np.float64) * np.ones(self.mesh.n_elems)
        self.k = np.asarray(k, dtype=np.float64) * np.ones(self.mesh.n_elems)

    # ---- element helpers ----------------------------------------------------------------
    def _Qq(self, sl):
        Qq = np.repeat(self.q_scale * self.Qe[sl, None], 8, axis=1)
        if self.Qq_extra is not None:
            Qq = Qq + self.Qq_extra[sl]
        return Qq

    def _chunks(self):
        E = self.mesh.n_elems
        for a in range(0, E, self.CHUNK):
            yield slice(a, min(E, a + self.CHUNK))

    def gather(self, s, sl):
        s2 = s.reshape(-1, 2)
        c = self.conn[sl]
        return s2[c, 0], s2[c, 1]

    def scatter(self, RP, RT, sl, out):
        c = self.conn[sl].ravel()
        n = self.mesh.n_nodes
        out[0::2] += np.bincount(c, RP.ravel(), minlength=n)
        out[1::2] += np.bincount(c, RT.ravel(), minlength=n)

    # ---- global operators -------------------------------------------------------------------
    def residual_raw(self, s):
        """Assembled R(s) = M(s) s - f (Eq. finalsyseq) over all DOFs, no BC rows applied."""
        out = np.zeros(2 * self.mesh.n_nodes)
        for sl in self._chunks():
            pe, te = self.gather(s, sl)
            fP = None if self.fPq is None else self.fPq[sl]
            RP, RT = self.em.residual(pe, te, self.kappa[sl], self.k[sl], self._Qq(sl), fP)
            self.scatter(RP, RT, sl, out)
        return out

    def residual(self, s):
        """R(s) with Dirichlet rows replaced by s_d - sbar_d."""
        R = self.residual_raw(s)
        R[self.dir_mask] = s[self.dir_mask] - self.dir_val[self.dir_mask]
        return R

    def jvp_raw(self, s, v):
        out = np.zeros(2 * self.mesh.n_nodes)
        for sl in self._chunks():
            pe, te = self.gather(s, sl)
            dp, dt = self.gather(v, sl)
            dRP, dRT = self.em.jvp(pe, te, self.kappa[sl], self.k[sl], self._Qq(sl), dp, dt)
            self.scatter(dRP, dRT, sl, out)
        return out

    def picard_jvp_raw(self, s, v):
        """Frozen-coefficient operator (ElementModel.picard_jvp) applied to v over all DOFs, no BC rows."""
        out = np.zeros(2 * self.mesh.n_nodes)
        for sl in self._chunks():
            pe, te = self.gather(s, sl)
            dp, dt = self.gather(v, sl)
            dRP, dRT = self.em.picard_jvp(pe, te, self.kappa[sl], self.k[sl], dp, dt)
            self.scatter(dRP, dRT, sl, out)
        return out

    def picard_matrix_full(self, s):
        """Assembled frozen-coefficient operator over all DOFs (no BC treatment), CSR; column b of an
        element's matrix is picard_jvp along the unit vector e_b."""
        rows, cols, vals = [], [], []
        for sl in self._chunks():
            pe, te = self.gather(s, sl)
            E = pe.shape[0]
            Je = np.empty((E, 16, 16))
            for b in range(16):
                dp = np.zeros((E, 8))
                dt = np.zeros((E, 8))
                (dp if b < 8 else dt)[:, b % 8] = 1.0
                dRP, dRT = self.em.picard_jvp(pe, te, self.kappa[sl], self.k[sl], dp, dt)
                Je[:, :8, b] = dRP
                Je[:, 8:, b] = dRT
            c = self.conn[sl]
            dof = np.concatenate([2 * c, 2 * c + 1], axis=1)
            rows.append(np.repeat(dof, 16, axis=1).ravel())
            cols.append(np.tile(dof, (1, 16)).ravel())
            vals.append(Je.ravel())
        n2 = 2 * self.mesh.n_nodes
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n2, n2))

    def jacobian_full(self, s):
        """Assembled sparse Jacobian dR/ds over all DOFs (no BC treatment), CSR."""
        rows, cols, vals = [], [], []
        for sl in self._chunks():
            pe, te = self.gather(s, sl)
            Je = self.em.jacobian(pe, te, self.kappa[sl], self.k[sl], self._Qq(sl))
            c = self.conn[sl]
            dof = np.concatenate([2 * c, 2 * c + 1], axis=1)          # (E, 16)
            rows.append(np.repeat(dof, 16, axis=1).ravel())
            cols.append(np.tile(dof, (1, 16)).ravel())
            vals.append(Je.ravel())
        n2 = 2 * self.mesh.n_nodes
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n2, n2))

    def jacobian_free(self, s):
        J = self.jacobian_full(s)
        return J[self.free][:, self.free].tocsc()

    # ---- Newton ---------------------------------------------------------------------------------
    def initial_state(self):
        return self.dir_val.copy()

    def _phi(self, s):
        R = self.residual(s)
        return float(np.dot(R[self.free], R[self.free])), R

    @staticmethod
    def damping(phi_fn, phi0):
        """Residual-minimising damping factor (Sec. 5.4); returns (lam, phi, R) or None."""
        phi1, R1 = phi_fn(1.0)
        if phi1 <= (1.0 - 1e-4) * phi0:
            return 1.0, phi1, R1
        phih, Rh = phi_fn(0.5)
        cands = [(phi1, 1.0, R1), (phih, 0.5, Rh)]
        c1 = 4.0 * phih - 3.0 * phi0 - phi1
        c2 = 2.0 * phi1 + 2.0 * phi0 - 4.0 * phih
        if c2 > 0.0:
            lam = min(1.0, max(0.05, -c1 / (2.0 * c2)))
            if lam not in (0.5, 1.0):
                p, R = phi_fn(lam)
                cands.append((p, lam, R))
        best = min(cands, key=lambda c: (c[0], -c[1]))
        if best[0] < phi0:
            return best[1], best[0], best[2]
        lam = 0.25
        for _ in range(8):
            p, R = phi_fn(lam)
            if p < phi0:
                return lam, p, R
            lam *= 0.5
        return None

    def newton(self, s0, rtol, maxit, ref_norm=None):
        s = s0.copy()
        phi, R = self._phi(s)
        ref = ref_norm if ref_norm is not None else np.sqrt(phi)
        hist = []
        for it in range(maxit + 1):
            rel = np.sqrt(phi) / ref if ref > 0 else 0.0
            hist.append(rel)
            if not np.isfinite(rel):
                raise NewtonFailure("non-finite residual")
            if rel <= rtol:
                return s, hist
            if it == maxit:
                break
            Jf = self.jacobian_free(s)
            d = np.zeros_like(s)
            d[self.free] = spla.spsolve(Jf, -R[self.free])
            res = self.damping(lambda lam: self._phi(s + lam * d), phi)
            if res is None:
                raise NewtonFailure("no damping factor reduces the residual")
            lam, phi, R = res
            s = s + lam * d
        raise NewtonFailure("Newton did not converge in %d iterations" % maxit)

    def reference_norm(self):
        """||R_free(s0)|| at the zero (BC-satisfying) state with the full source."""
        save = self.q_scale
        self.q_scale = 1.0
        phi, _ = self._phi(self.initial_state())
        self.q_scale = save
        return np.sqrt(phi)

    def solve_state(self, s0=None, rtol=None, maxit=None):
        """Damped Newton from s0 (default zero state); on failure ramp Q by 1/4, 1/2, 1."""
        rtol = self.par.newton_rtol if rtol is None else rtol
        maxit = self.par.newton_maxit if maxit is None else maxit
        start = self.initial_state() if s0 is None else np.asarray(s0, dtype=np.float64).copy()
        ref = self.reference_norm()
        self.q_scale = 1.0
        try:
            s, hist = self.newton(start, rtol, maxit, ref)
            self.ramped = False
        except NewtonFailure:
            s = start
            hist = []
            for scale in (0.25, 0.5, 1.0):
                self.q_scale = scale
                s, h = self.newton(s, rtol if scale == 1.0 else 1e-6, maxit,
                                   ref if scale == 1.0 else None)
                hist += h
            self.ramped = True
        self.q_scale = 1.0
        self.s = s
        self.history = hist
        return s

    # ---- outputs, objective, adjoint --------------------------------------------------------
    def fields(self, s=None):
        s = self.s if s is None else s
        return s[0::2].copy(), s[1::2].copy()

    def velocities(self, s=None):
        s = self.s if s is None else s
        out = np.empty((self.mesh.n_elems, 3))
        for sl in self._chunks():
            pe, te = self.gather(s, sl)
            out[sl] = self.em.centroid_velocity(pe, te, self.kappa[sl])
        return out

    def objective_weights(self):
        """df/ds: f = (1/|Omega_h|) sum_{e in Omega_h} int_e N t_e (mean T over the heated region)."""
        wN = self.em.w * self.em.N.sum(axis=0)            # int_e N_a
        d = np.zeros(2 * self.mesh.n_nodes)
        c = self.conn[self.heated]
        d[1::2] = np.bincount(c.ravel(), np.tile(wN, c.shape[0]), minlength=self.mesh.n_nodes)
        return d / self.vol_h

    def objective(self, s=None):
        s = self.s if s is None else s
        return float(self.objective_weights() @ s)

    # ---- thermal compliance of Eq. objdiscr (SUPG-weighted source) --------------------------
    def _supg_elems(self, s, sl, cplx_dof=None, h=1e-30):
        """Element values f_e = f_tQ,e . t_e of the heated elements sl; with cplx_dof = d (0..15)
        the d-th element DOF gets the imaginary step i h (complex-step derivative)."""
        pe, te = self.gather(s, sl)
        if cplx_dof is not None:
            pe, te = pe.astype(complex), te.astype(complex)
            (pe if cplx_dof < 8 else te)[:, cplx_dof % 8] += 1j * h
        Qq = np.repeat(self.q_scale * self.Qe[sl, None], 8, axis=1)
        return np.sum(self.em.supg_load(pe, te, self.kappa[sl], Qq) * te, axis=1)

    def supg_compliance(self, s=None):
        """f = sum_e f_tQ,e^T t_e (Eq. objdiscr), over the elements with a source."""
        s = self.s if s is None else s
        el = np.flatnonzero(self.Qe != 0.0)
        return float(np.sum(self._supg_elems(s, el)))

    def supg_compliance_weights(self, s=None):
        """df/ds of supg_compliance by complex-step differentiation of the element values."""
        s = self.s if s is None else s
        el = np.flatnonzero(self.Qe != 0.0)
        cn = self.conn[el]
        d = np.zeros(2 * self.mesh.n_nodes)
        h = 1e-30
        for dof in range(16):
            g = np.imag(self._supg_elems(s, el, dof, h)) / h
            d += np.bincount(2 * cn[:, dof % 8] + (1 if dof >= 8 else 0), g, minlength=d.size)
        d[self.dir_mask] = 0.0
        return d

    def solve_adjoint(self, objective="mean_T"):
        """J^T lambda = df/ds on the free DOFs; objective "mean_T" (default) or "supg_compliance"."""
        J = self.jacobian_full(self.s)
        Jf = J[self.free][:, self.free]
        w = self.objective_weights() if objective == "mean_T" else self.supg_compliance_weights()
        rhs = w[self.free]
        lam = np.zeros(2 * self.mesh.n_nodes)
        lam[self.free] = spla.spsolve(Jf.T.tocsc(), rhs)
        self.lam = lam
        return lam

    def sensitivity_gamma_tilde(self):
        """df/dgamma~_e = -lambda_e^T (dR_e/dkappa kappa' + dR_e/dk k'); 0 on passive elements."""
        out = np.empty(self.mesh.n_elems)
        for sl in self._chunks():
            pe, te = self.gather(self.s, sl)
            lp, lt = self.gather(self.lam, sl)
            (dkP, dkT), (dcP, dcT) = self.em.design_derivatives(
                pe, te, self.kappa[sl], self.k[sl], self._Qq(sl))
            dL_dkappa = (lp * dkP).sum(1) + (lt * dkT).sum(1)
            dL_dk = (lp * dcP).sum(1) + (lt * dcT).sum(1)
            out[sl] = -(dL_dkappa * self.dkappa[sl] + dL_dk * self.dk[sl])
        out[self.passive] = 0.0
        return out

    def sensitivities(self):
        """df/dgamma for the raw design (filter transpose applied); 0 on passive elements."""
        g = self.filter.apply_transpose(self.sensitivity_gamma_tilde())
        g[self.passive] = 0.0
        return g

    # ---- sampled rows (large-grid checks) -----------------------------------------------------
    def _elements_around(self, nodes):
        m = self.mesh
        ijk = m.node_ijk()[np.asarray(nodes)]
        elems = set()
        for (i, j, k) in ijk:
            for dk in (-1, 0):
                for dj in (-1, 0):
                    for di in (-1, 0):
                        a, b, c = i + di, j + dj, k + dk
                        if 0 <= a < m.nx and 0 <= b < m.ny and 0 <= c < m.nz:
                            elems.add(a + m.nx * (b + m.ny * c))
        return np.array(sorted(elems))

    def jt_at_nodes(self, s, lam, nodes):
        """(J(s)^T lam) at the given nodes (P and T entries), from the element Jacobians around them.
        lam is taken as 0 on the Dirichlet rows (the adjoint lives on the free DOFs)."""
        nodes = np.asarray(nodes)
        el = self._elements_around(nodes)
        s2 = s.reshape(-1, 2)
        l2 = np.where(self.dir_mask, 0.0, lam).reshape(-1, 2)
        cn = self.conn[el]
        Qq = np.repeat(self.q_scale * self.Qe[el, None], 8, axis=1)
        Je = self.em.jacobian(s2[cn, 0], s2[cn, 1], self.kappa[el], self.k[el], Qq)
        le = np.concatenate([l2[cn, 0], l2[cn, 1]], axis=1)          # (E, 16) row multipliers
        contrib = np.einsum("er,erc->ec", le, Je)                     # (E, 16) column sums
        out = np.zeros((len(nodes), 2))
        for r, nd in enumerate(nodes):
            hit = cn == nd
            out[r, 0] = contrib[:, :8][hit].sum()
            out[r, 1] = contrib[:, 8:][hit].sum()
        return out

    def residual_at_nodes(self, s, nodes):
        """R(s) at the given nodes (P and T rows), from the elements around them only."""
        nodes = np.asarray(nodes)
        el = self._elements_around(nodes)
        s2 = s.reshape(-1, 2)
        cn = self.conn[el]
        Qq = np.repeat(self.q_scale * self.Qe[el, None], 8, axis=1)
        RP, RT = self.em.residual(s2[cn, 0], s2[cn, 1], self.kappa[el], self.k[el], Qq)
        out = np.zeros((len(nodes), 2))
        for r, nd in enumerate(nodes):
            hit = cn == nd
            out[r, 0] = RP[hit].sum()
            out[r, 1] = RT[hit].sum()
        return out
