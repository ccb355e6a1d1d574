"""Topology optimisation loop around the state/adjoint path (Sec. 5).

Problem (Eq. optprob): minimise f(s(gamma), gamma) subject to the volume constraint of Eq. constr,
g(gamma) = sum_D gamma_e v_e / sum_D v_e - g* <= 0 over the design elements D (the design box minus
the heated box; with the default parameters everything above the heated layers), 0 <= gamma <= 1,
with R(s, gamma) = 0 solved by the library. f is the library's
objective (mean temperature over the heated region), its gradient the library's adjoint sensitivities.

Optimiser: the Method of Moving Asymptotes (Svanberg 1987), with the move limit of Sec. 6.1
(0.2) and the continuation of Eq. contsch1 (q_c, q_p and kappa_s changed at fixed iterations).
Each iteration warm-starts Newton from the previous state (Sec. 5.4).

MMA as implemented here, for n variables and one inequality constraint:
* asymptotes L, U around x: at the first two iterations x -/+ 0.5 (x_max - x_min); then moved
  outward (factor 1.2) where the last two steps had the same sign, inward (0.7) where they
  oscillated, and kept within [x - 10 (x_max - x_min), x - 0.01 (x_max - x_min)] (mirrored for U);
* box of the subproblem: alpha = max(x_min, L + 0.1 (x - L), x - move),
  beta = min(x_max, U - 0.1 (U - x), x + move);
* convex separable approximations f~_i(x) = r_i + sum_j p_ij / (U_j - x_j) + q_ij / (x_j - L_j) with
  p_ij = (U_j - x_j)^2 (max(d_ij, 0) + 1e-3 |d_ij| + 1e-5 / (x_max - x_min)),
  q_ij = (x_j - L_j)^2 (max(-d_ij, 0) + 1e-3 |d_ij| + 1e-5 / (x_max - x_min)), d_ij = df_i/dx_j,
  and r_i such that f~_i(x^k) = f_i(x^k);
* subproblem min f~_0 s.t. f~_1 <= 0 on [alpha, beta], solved through its one-dimensional dual:
  for a multiplier lam >= 0 each x_j minimises (p_0j + lam p_1j)/(U_j - x_j) + (q_0j + lam q_1j)/(x_j - L_j)
  in closed form, x_j = (sqrt(P) L_j + sqrt(Q) U_j) / (sqrt(P) + sqrt(Q)) clamped to [alpha_j, beta_j];
  f~_1(x(lam)) is non-increasing in lam, so the maximising lam is found by bisection on f~_1 = 0
  (lam = 0 when f~_1(x(0)) <= 0).
The loop scales the objective and the constraint so that their largest per-element gradients are
of order one, the scale MMA's fixed regularisation constants assume.
"""

import math
import time

import torch

from . import _abi
from .problem import Problem


class MMA:
    """Method of Moving Asymptotes for min f0(x) s.t. f1(x) <= 0, x_min <= x <= x_max (torch tensors)."""

    def __init__(self, x_min, x_max, move=0.2, s_init=0.5, s_grow=1.2, s_shrink=0.7):
        self.x_min, self.x_max = x_min, x_max
        self.move = move
        self.s_init, self.s_grow, self.s_shrink = s_init, s_grow, s_shrink
        self.k = 0
        self.x1 = self.x2 = None   # previous two iterates
        self.L = self.U = None

    def _asymptotes(self, x):
        span = self.x_max - self.x_min
        if self.k < 2:
            self.L = x - self.s_init * span
            self.U = x + self.s_init * span
        else:
            trend = (x - self.x1) * (self.x1 - self.x2)
            fac = torch.ones_like(x)
            fac = torch.where(trend > 0, torch.full_like(x, self.s_grow), fac)
            fac = torch.where(trend < 0, torch.full_like(x, self.s_shrink), fac)
            L = x - fac * (self.x1 - self.L)
            U = x + fac * (self.U - self.x1)
            self.L = torch.minimum(torch.maximum(L, x - 10.0 * span), x - 0.01 * span)
            self.U = torch.maximum(torch.minimum(U, x + 10.0 * span), x + 0.01 * span)

    def step(self, x, f0, df0, f1, df1, tol=1e-12, max_bisect=200):
        """One MMA iteration from x with objective f0, constraint f1 and their gradients; returns the
        new x (a new tensor)."""
        self._asymptotes(x)
        L, U = self.L, self.U
        span = self.x_max - self.x_min
        alpha = torch.maximum(torch.maximum(self.x_min, L + 0.1 * (x - L)), x - self.move)
        beta = torch.minimum(torch.minimum(self.x_max, U - 0.1 * (U - x)), x + self.move)
        ux, xl = U - x, x - L
        eps = 1e-5 / span

        def pq(d):
            p = ux * ux * (torch.clamp(d, min=0) + 1e-3 * d.abs() + eps)
            q = xl * xl * (torch.clamp(-d, min=0) + 1e-3 * d.abs() + eps)
            return p, q

        p0, q0 = pq(df0)
        p1, q1 = pq(df1)
        r1 = f1 - (p1 / ux + q1 / xl).sum()

        def x_of(lam):
            P = p0 + lam * p1
            Q = q0 + lam * q1
            sp, sq = torch.sqrt(P), torch.sqrt(Q)
            xs = (sp * L + sq * U) / (sp + sq)
            return torch.minimum(torch.maximum(xs, alpha), beta)

        def g1(xs):
            return float(r1 + (p1 / (U - xs) + q1 / (xs - L)).sum())

        xn = x_of(0.0)
        if g1(xn) > 0.0:
            lo, hi = 0.0, 1.0
            while g1(x_of(hi)) > 0.0:
                hi *= 10.0
                if hi > 1e30:
                    break
            for _ in range(max_bisect):
                mid = 0.5 * (lo + hi)
                if g1(x_of(mid)) > 0.0:
                    lo = mid
                else:
                    hi = mid
                if hi - lo <= tol * max(1.0, hi):
                    break
            xn = x_of(hi)
        self.x2, self.x1 = self.x1, x.clone()
        self.k += 1
        return xn


# Continuation of Eq. contsch1: (q_c, q_p, kappa_s) per stage; kappa_s in absolute units.
PAPER_CONTINUATION = ({"q_c": 0.881, "q_p": 8.0, "kappa_s": 1e-5}, {"q_c": 8.81, "q_p": 8.0, "kappa_s": 1e-5},
                      {"q_c": 88.1, "q_p": 8.0, "kappa_s": 1e-5}, {"q_c": 88.1, "q_p": 98.0, "kappa_s": 1e-6},
                      {"q_c": 881.0, "q_p": 998.0, "kappa_s": 1e-7})


def region_masks(nx, ny, nz, params):
    """Boolean masks (design, heated) of the elements (element e = i + nx (j + ny k)): the heated box
    [0, heat_nx) x [0, heat_ny) x [0, heated_layers) and the design box [0, design_nx) x [0, design_ny) x
    [heated_layers, heated_layers + design_nz) minus it, a zero extent meaning the full one (nc_params).
    Elements in neither are passive fluid."""
    hl = params.heated_layers
    k, j, i = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx), indexing="ij")
    i, j, k = i.reshape(-1), j.reshape(-1), k.reshape(-1)
    if params.region_shape == _abi.NC_REGION_CYLINDER:
        # centroid within the radius: (2i+1)^2 + (2j+1)^2 < 4 r^2
        q = (2 * i + 1) ** 2 + (2 * j + 1) ** 2
        layers = (k >= params.heat_z0) & (k < params.heat_z0 + hl)
        heated = layers & (q < 4.0 * params.heat_radius ** 2)
        return layers & (q < 4.0 * params.design_radius ** 2) & ~heated, heated
    hx, hy = params.heat_nx or nx, params.heat_ny or ny
    dx, dy = params.design_nx or nx, params.design_ny or ny
    z1 = hl + params.design_nz if params.design_nz else nz
    heated = (i < hx) & (j < hy) & (k < hl)
    return (i < dx) & (j < dy) & (k >= hl) & (k < z1) & ~heated, heated


def cavity_params(n):
    """The benchmark of Sec. 6.1 on the quarter cavity of n x n x 2n elements (h = 1 / 2n): heat source
    0.05^3 m (n / 10 elements per side), Q = 1e4 W/m^3, design box 0.375 x 0.375 x 0.75 m on top of it.
    n must be a multiple of 20 (80 gives the 80 x 80 x 160 mesh of Table 3)."""
    if n % 20:
        raise ValueError("n must be a multiple of 20")
    return dict(bc=_abi.NC_BC_CAVITY, Q=1e4, heat_nx=n // 10, heat_ny=n // 10, heated_layers=n // 10,
                design_nx=3 * n // 4, design_ny=3 * n // 4, design_nz=3 * n // 2)


def cylinder_params(n):
    """The suspended cylinder of Sec. 7 on the quarter cavity of n x n x 2n elements (h = 1 / 2n): heated
    cylinder of radius 0.1 m and height 0.2 m centred in the cavity (Q = 1e3 W/m^3), design annulus out to
    0.25 m over the same height, kappa_f = 0.000676 m^2 as the paper sets it. n must be a multiple of 5
    (160 gives the paper's 160 x 160 x 320 mesh)."""
    if n % 5:
        raise ValueError("n must be a multiple of 5")
    return dict(bc=_abi.NC_BC_CAVITY, region_shape=_abi.NC_REGION_CYLINDER, Q=1e3, kappa_f=0.000676,
                heat_radius=0.2 * n, design_radius=0.5 * n, heat_z0=4 * n // 5, heated_layers=2 * n // 5)


class LibraryEvaluator:
    """f, df/drho and the warm-start state of a design through the library (the default evaluator of
    optimize): set_design, Newton warm-started from the previous state (Sec. 5.4), adjoint,
    sensitivities."""

    def __init__(self, nx, ny, nz, alpha, device="cuda", **params):
        self.pb = Problem(nx, ny, nz, 1.0 / nz, device=device, alpha=alpha, **params)
        self.params = self.pb.params
        self.kappa_f, _ = self.pb.permeabilities()
        self.state = None

    def set_stage(self, **overrides):
        self.pb.set_params(**overrides)

    def __call__(self, rho):
        pb = self.pb
        pb.set_design(rho)
        if self.state is not None:
            pb.set_state(*self.state)
        sst = pb.solve_state()
        f, ast = pb.solve_adjoint()
        grad = pb.sensitivities()
        P, T, _ = pb.get_fields(velocity=False)
        self.state = (P.clone(), T.clone())
        return f, grad, {"newton_its": sst["newton_its"], "krylov_its": sst["krylov_its"],
                         "adjoint_krylov_its": ast["krylov_its"]}

    def close(self):
        self.pb.close()


def optimize(nx, ny, nz, alpha, volfrac, iters, move=0.2, stages=PAPER_CONTINUATION, stage_every=None,
             rho0=None, device="cuda", callback=None, evaluator=None, keep_iterates=False, **params):
    """Run `iters` MMA iterations of Eq. optprob on an nx x ny x nz grid (h = 1/nz).

    stages: continuation stages (dicts of q_c, q_p and kappa_s or kappa_ratio), each used for
    stage_every iterations (default: iters split evenly). evaluator: an object with `params` (nc_params
    of the regions), `kappa_f`, set_stage(**overrides), __call__(rho) -> (f, df/drho, stats dict) and
    close(); default LibraryEvaluator. Returns {"rho": final design, "history": one record per
    iteration (f, g, max change, stage, solver iterations, seconds; with keep_iterates the new design
    variables "x" as well)}.
    """
    ev = evaluator if evaluator is not None else LibraryEvaluator(nx, ny, nz, alpha, device=device, **params)
    ne = nx * ny * nz
    design, heated = (m.to(device) for m in region_masks(nx, ny, nz, ev.params))
    nd = int(design.sum())
    rho = torch.full((ne,), float(volfrac), dtype=torch.float64, device=device) if rho0 is None else \
        torch.as_tensor(rho0, dtype=torch.float64, device=device).clone()
    rho[~design] = heated[~design].double()   # passive: heated solid 1, fluid 0 (as set_design fixes them)
    x = rho[design].clone()
    mma = MMA(torch.zeros_like(x), torch.ones_like(x), move=move)
    stage_every = stage_every or max(1, math.ceil(iters / max(1, len(stages))))
    kf = ev.kappa_f
    history = []
    fscale = None
    stage = -1
    for it in range(iters):
        s = min(it // stage_every, len(stages) - 1) if stages else -1
        if s != stage and stages:
            stage = s
            st = dict(stages[s])
            if "kappa_s" in st:
                st["kappa_ratio"] = st.pop("kappa_s") / kf
            ev.set_stage(**st)
        t0 = time.perf_counter()
        rho[design] = x
        f, grad, stats = ev(rho)
        gval = float(x.mean()) - volfrac
        # scaling for MMA's fixed regularisation (1e-5 per variable): objective and constraint are
        # scaled so that their largest per-element gradients are of order one (the objective's scale
        # taken at the first iteration and kept)
        df = grad[design]
        if fscale is None:
            fscale = 1.0 / max(float(df.abs().max()), 1e-300)
        x_new = mma.step(x, f * fscale, df * fscale, gval * nd, torch.ones_like(x))
        change = float((x_new - x).abs().max())
        x = x_new
        rec = {"it": it, "f": f, "g": gval, "change": change, "stage": stage, "seconds": time.perf_counter() - t0}
        if keep_iterates:
            rec["x"] = x.clone()
        rec.update(stats)
        history.append(rec)
        if callback:
            callback(rec)
    rho[design] = x
    if evaluator is None:
        ev.close()
    return {"rho": rho, "history": history}


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="MMA topology optimisation with the GB300 state/adjoint path")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--alpha", type=float, default=1e3)
    ap.add_argument("--volfrac", type=float, default=0.1)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--cavity", action="store_true",
                    help="the Sec. 6.1 benchmark on the quarter cavity of n x n x 2n elements (n a multiple of 20)")
    ap.add_argument("--cylinder", action="store_true",
                    help="Sec. 7's suspended cylinder on the quarter cavity of n x n x 2n elements (n a multiple of 5)")
    a = ap.parse_args()
    from .presets import solver_settings
    geom = cavity_params(a.n) if a.cavity else cylinder_params(a.n) if a.cylinder else {}
    geom.update(solver_settings(a.alpha))
    out = optimize(a.n, a.n, 2 * a.n if (a.cavity or a.cylinder) else a.n, a.alpha, a.volfrac, a.iters, **geom,
                   callback=lambda r: print("it %3d f %.6e g %+.2e change %.3f stage %d newton %d krylov %d/%d %.3f s"
                                            % (r["it"], r["f"], r["g"], r["change"], r["stage"], r["newton_its"],
                                               r["krylov_its"], r["adjoint_krylov_its"], r["seconds"]), flush=True))
