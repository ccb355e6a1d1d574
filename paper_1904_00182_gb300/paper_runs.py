"""State and adjoint solves on the paper's own meshes and geometries, one GPU.

* The closed-cavity benchmark of Sec. 6.1 on the meshes of Sec. 6.2 (Tables 3 and 4): the quarter
  cavity on n x n x 2n elements for n = 80, 160, 320 (2.1 M to 131 M unknowns), alpha = 1e3 and
  1e6, from the paper's initial design gamma = 0.05 in the design box.
* The suspended cylinder of Sec. 7 on its 160 x 160 x 320 mesh, alpha = 1e6 (kappa_f = 0.000676 as
  the paper sets it), from an initial design of the paper's kind: four regularly spaced radial fins
  holding the volume fraction 0.15 of the design annulus (in the quarter domain one fin on its
  diagonal, solid, with fluid elsewhere in the annulus).

Each case creates the problem (footprint from nc_footprint_bytes) with the solver settings of its
alpha (presets.solver_settings: the z-line smoother at alpha = 1e6), solves the state from zero to a
relative residual of 1e-8, then the adjoint of the mean heated-region temperature and the
sensitivities, and prints one JSON line with the times (CUDA events on the problem's stream), the
Newton and Krylov iterations and the device memory the problem holds. When Newton does not converge
from zero, the state is reached by warm starts (Sec. 5.4) up the ladder alpha = 1e5, 2e5, 4e5, 7e5
and the last, warm-started solve is timed. The paper ran these meshes with MPI domain decomposition
on 16 to 640 CPU cores (Table 3); here each runs on one GPU.

  python -m paper_1904_00182_gb300.paper_runs [--cases cavity80,cavity160,cavity320,cylinder160]
"""

import argparse
import json
import math
import time

import torch

from . import _abi
from .optimize import cavity_params, cylinder_params, region_masks
from .presets import solver_settings
from .problem import Problem

CASES = {
    "cavity80": ("cavity", 80), "cavity160": ("cavity", 160), "cavity320": ("cavity", 320),
    "cylinder80": ("cylinder", 80), "cylinder160": ("cylinder", 160), "cylinder320": ("cylinder", 320),
}


def fin_design(n, params, volfrac=0.15):
    """Initial cylinder design of Sec. 7's kind: four regularly spaced radial fins holding `volfrac` of
    the design annulus. In the quarter domain (symmetry planes x = 0, y = 0) that is one fin along the
    diagonal x = y, of constant thickness; heated elements 1, every other element 0."""
    nz = 2 * n
    design, heated = region_masks(n, n, nz, params)
    k, j, i = torch.meshgrid(torch.arange(nz), torch.arange(n), torch.arange(n), indexing="ij")
    dist = ((i.reshape(-1) - j.reshape(-1)).abs().double()) / math.sqrt(2.0)   # centroid distance to x = y
    r_in, r_out = params.heat_radius, params.design_radius
    half = 0.5 * volfrac * (math.pi / 4.0) * (r_out ** 2 - r_in ** 2) / (r_out - r_in)
    rho = heated.double()
    rho[design & (dist < half)] = 1.0
    return rho


def run_case(kind, n, alpha, device="cuda", continuation=(), **overrides):
    geom = cavity_params(n) if kind == "cavity" else cylinder_params(n)
    geom.update(overrides)
    nx, ny, nz = n, n, 2 * n
    grid = _abi.Grid(nx, ny, nz, 1.0 / nz)
    footprint = _abi.footprint_bytes(grid, _abi.default_params(alpha=alpha, **geom))
    stream = torch.cuda.Stream(device=device)
    free0 = torch.cuda.mem_get_info(device)[0]
    t0 = time.perf_counter()
    pb = Problem(nx, ny, nz, 1.0 / nz, stream=stream.cuda_stream, device=device, alpha=alpha, timeout_s=3600.0,
                 **geom)
    t_create = time.perf_counter() - t0
    held = free0 - torch.cuda.mem_get_info(device)[0]
    ne = nx * ny * nz
    if kind == "cavity":
        rho = torch.full((ne,), 0.05, dtype=torch.float64, device=device)
    else:
        rho = fin_design(n, pb.params).to(device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    cont = []
    for a_c in continuation:
        # warm starts (Sec. 5.4) up an alpha ladder: each solve starts from the previous state
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pb.set_params(alpha=a_c)
        pb.set_design(rho)
        if cont:
            pb.set_state(*state)
        stc = pb.solve_state()
        P, T, _ = pb.get_fields(velocity=False)
        state = (P.clone(), T.clone())
        e1.record(stream)
        e1.synchronize()
        cont.append({"alpha": a_c, "ms": e0.elapsed_time(e1), "newton_its": stc["newton_its"],
                     "krylov_its": stc["krylov_its"]})
    if cont:
        pb.set_params(alpha=alpha)
    ev[0].record(stream)
    pb.set_design(rho)
    if cont:
        pb.set_state(*state)
    ev[1].record(stream)
    st = pb.solve_state()
    ev[2].record(stream)
    f, ast = pb.solve_adjoint()
    pb.sensitivities()
    ev[3].record(stream)
    ev[3].synchronize()
    out = {"case": "%s %dx%dx%d" % (kind, nx, ny, nz), "alpha": alpha, "elements": ne,
           "unknowns": 2 * (nx + 1) * (ny + 1) * (nz + 1), "footprint_gib": footprint / 2 ** 30,
           "device_memory_held_gib": held / 2 ** 30, "create_s": t_create,
           "design_ms": ev[0].elapsed_time(ev[1]), "state_ms": ev[1].elapsed_time(ev[2]),
           "adjoint_sens_ms": ev[2].elapsed_time(ev[3]), "newton_its": st["newton_its"],
           "krylov_its": st["krylov_its"], "krylov_per_newton": st["krylov_hist"], "rel_residual": st["rel_residual"],
           "adjoint_krylov_its": ast["krylov_its"], "adjoint_rel_residual": ast["rel_residual"], "f": f,
           "mg_setups": st["mg_setups"]}
    if cont:
        out["warm_start_from"] = cont
    pb.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--cases", default="cavity80,cavity160,cylinder160")
    ap.add_argument("--alphas", default="1e3,1e6")
    ap.add_argument("--mg-op0", default="picard", choices=["exact", "picard"])
    ap.add_argument("--library-defaults", action="store_true",
                    help="the library's default smoother at every alpha instead of presets.solver_settings")
    a = ap.parse_args()
    op0 = _abi.NC_MGOP_PICARD if a.mg_op0 == "picard" else _abi.NC_MGOP_EXACT
    for name in a.cases.split(","):
        kind, n = CASES[name]
        alphas = [1e6] if kind == "cylinder" else [float(x) for x in a.alphas.split(",")]
        for alpha in alphas:
            extra = {} if a.library_defaults else solver_settings(alpha)
            try:
                rec = run_case(kind, n, alpha, mg_op0=op0, **extra)
            except _abi.NatConvError as e:
                # from zero Newton may not reach the strongly convective state; the paper warm-starts
                # every solve from the previous one, so climb to alpha from a weakly convective state
                ladder = [a for a in (1e5, 2e5, 4e5, 7e5) if a < alpha]
                try:
                    rec = run_case(kind, n, alpha, mg_op0=op0, continuation=ladder, **extra)
                except _abi.NatConvError as e2:
                    rec = {"case": name, "alpha": alpha, "error": str(e2)}
                rec["from_zero"] = str(e)
            rec["mg_op0"] = a.mg_op0
            rec.update(extra)
            print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
