"""The MMA optimiser (Svanberg 1987) against closed-form optima, and the optimisation loop of
Eq. optprob around the GPU state/adjoint path.

* Svanberg's cantilever (five segments, minimise 0.0624 sum x_j s.t. sum c_j / x_j^3 <= 1 with
  c = 61, 37, 19, 7, 1): the Lagrange conditions give x_j = (sum_k c_k^(1/4))^(1/3) c_j^(1/4), i.e.
  x* = (6.016, 5.309, 4.494, 3.502, 2.153) and f* = 1.340.
* A separable problem min sum c_j / x_j s.t. mean(x) <= v, 0.001 <= x <= 1: x_j = min(1, sqrt(c_j / mu))
  with mu set by the constraint (bisection here, independent of MMA).
* GPU: 12 iterations at 32^3 lower the objective and keep every iterate feasible.
"""

import numpy as np
import pytest
import torch

from paper_1904_00182_gb300.optimize import MMA


def test_mma_svanberg_cantilever():
    c = torch.tensor([61.0, 37.0, 19.0, 7.0, 1.0], dtype=torch.float64)
    x = torch.full((5,), 5.0, dtype=torch.float64)
    mma = MMA(torch.full((5,), 1.0, dtype=torch.float64), torch.full((5,), 10.0, dtype=torch.float64), move=10.0)
    for _ in range(60):
        f0, df0 = float(0.0624 * x.sum()), torch.full_like(x, 0.0624)
        f1, df1 = float((c / x ** 3).sum() - 1.0), -3.0 * c / x ** 4
        x = mma.step(x, f0, df0, f1, df1)
    xs = (c ** 0.25).sum() ** (1.0 / 3.0) * c ** 0.25
    assert torch.allclose(x, xs, rtol=1e-4)
    assert float(0.0624 * x.sum()) == pytest.approx(1.340, abs=5e-4)
    assert float((c / x ** 3).sum() - 1.0) <= 1e-6


def test_mma_separable_volume_problem():
    rng = np.random.default_rng(1)
    n, v = 200, 0.3
    c = torch.tensor(rng.uniform(0.1, 2.0, n))
    x = torch.full((n,), v, dtype=torch.float64)
    mma = MMA(torch.full((n,), 1e-3, dtype=torch.float64), torch.ones(n, dtype=torch.float64), move=0.2)
    for _ in range(80):
        x = mma.step(x, float((c / x).sum()), -c / x ** 2, float(x.mean() - v), torch.full_like(x, 1.0 / n))
    lo, hi = 1e-8, 1e8                        # mu with mean(min(1, sqrt(c / mu))) = v
    for _ in range(200):
        mu = (lo * hi) ** 0.5
        if float(torch.clamp(torch.sqrt(c / mu), 1e-3, 1.0).mean()) > v:
            lo = mu
        else:
            hi = mu
    xs = torch.clamp(torch.sqrt(c / hi), 1e-3, 1.0)
    assert float((x - xs).abs().max()) <= 1e-4
    assert float(x.mean() - v) <= 1e-8


@pytest.mark.gpu
def test_optimisation_loop_32():
    from paper_1904_00182_gb300 import build
    build.build()
    from paper_1904_00182_gb300.optimize import optimize
    out = optimize(32, 32, 32, 1e3, 0.1, 12, stages=({"q_c": 8.81, "q_p": 8.0},))
    h = out["history"]
    print(" ".join("%.6e" % r["f"] for r in h))
    assert h[-1]["f"] < h[0]["f"]                  # the heated region cools
    assert all(r["g"] <= 1e-6 for r in h)          # every iterate meets the volume constraint
    rho = out["rho"].cpu().numpy()
    assert rho.min() >= 0.0 and rho.max() <= 1.0
    assert np.all(rho[: 2 * 32 * 32] == 1.0)       # the heated layers stay solid


def test_region_masks_and_cavity_setup():
    """Design and heated masks follow the boxes of nc_params; the cavity setup reproduces Sec. 6.1's
    proportions (80 -> 80 x 80 x 160 mesh, heat source 8^3 elements, design box 60 x 60 x 120)."""
    import torch
    from paper_1904_00182_gb300 import _abi
    from paper_1904_00182_gb300.optimize import cavity_params, region_masks
    p = _abi.default_params()
    d, h = region_masks(4, 3, 5, p)
    assert int(h.sum()) == 4 * 3 * 2 and int(d.sum()) == 4 * 3 * 3 and not bool((d & h).any())
    g = cavity_params(80)
    assert (g["heat_nx"], g["heated_layers"], g["design_nx"], g["design_nz"]) == (8, 8, 60, 120)
    p = _abi.default_params(**{k: v for k, v in g.items() if k != "Q"})
    d, h = region_masks(80, 80, 160, p)
    assert int(h.sum()) == 8 ** 3 and int(d.sum()) == 60 * 60 * 120
    e = torch.arange(80 * 80 * 160)
    i, j, k = e % 80, (e // 80) % 80, e // 6400
    assert bool(((i < 60) & (j < 60) & (k >= 8) & (k < 128))[d].all())
    with pytest.raises(ValueError):
        cavity_params(50)


def test_cylinder_setup_and_masks():
    """Sec. 7's cylinder proportions (160 -> radii 32 and 80 elements, layers 128-191) and the masks the
    volume constraint uses: heated and design elements in the right layers, annulus between the radii."""
    from paper_1904_00182_gb300 import _abi
    from paper_1904_00182_gb300.optimize import cylinder_params, region_masks
    g = cylinder_params(160)
    assert (g["heat_radius"], g["design_radius"], g["heat_z0"], g["heated_layers"]) == (32.0, 80.0, 128, 64)
    g = cylinder_params(20)
    p = _abi.default_params(**{k: v for k, v in g.items() if k not in ("Q", "kappa_f")})
    d, h = region_masks(20, 20, 40, p)
    i = np.arange(20 * 20 * 40) % 20
    j = (np.arange(20 * 20 * 40) // 20) % 20
    k = np.arange(20 * 20 * 40) // 400
    r2 = (i + 0.5) ** 2 + (j + 0.5) ** 2
    d, h = d.numpy(), h.numpy()
    assert np.all((k[h] >= 16) & (k[h] < 24)) and np.all(r2[h] < 16.0)
    assert np.all((r2[d] >= 16.0) & (r2[d] < 100.0)) and not np.any(d & h)
    assert int(h.sum()) == 8 * int((r2[:400] < 16.0).sum())


@pytest.mark.gpu
def test_optimisation_loop_cavity():
    """A few MMA iterations on the quarter cavity (24 x 24 x 48, the design box 3/4 of the width and
    36 layers on a 2^3 heat box, Q = 1e4, 5 % volume; four multigrid levels, so the stencil levels
    include top-plane nodes that are free in P): f decreases, every iterate is feasible, passive
    elements keep their values."""
    from paper_1904_00182_gb300 import build
    build.build()
    import paper_1904_00182_gb300 as nc
    from paper_1904_00182_gb300.optimize import optimize
    geom = dict(bc=nc.NC_BC_CAVITY, Q=1e4, heat_nx=2, heat_ny=2, heated_layers=2, design_nx=18, design_ny=18,
                design_nz=36)
    out = optimize(24, 24, 48, 1e3, 0.05, 8, stages=({"q_c": 8.81, "q_p": 8.0},), **geom)
    h = out["history"]
    assert h[-1]["f"] < h[0]["f"]
    assert all(r["g"] <= 1e-6 for r in h)
    rho = out["rho"].cpu().numpy().reshape(48, 24, 24)
    assert np.all(rho[:2, :2, :2] == 1.0) and np.all(rho[38:, :, :] == 0.0) and np.all(rho[2:38, :, 18:] == 0.0)


@pytest.mark.parametrize("shape", ["box", "cylinder"])
def test_region_masks_match_the_oracle(shape):
    """The optimiser's design and heated masks (the volume constraint's elements) are the oracle's
    regions for the same parameters."""
    import oracle
    from paper_1904_00182_gb300 import _abi
    from paper_1904_00182_gb300.optimize import region_masks
    n, nz = 10, 20
    if shape == "box":
        kw = dict(heat_nx=3, heat_ny=2, heated_layers=2, design_nx=8, design_ny=7, design_nz=12)
        okw = dict(kw)
    else:
        kw = dict(region_shape=_abi.NC_REGION_CYLINDER, heat_radius=3.0, design_radius=7.5, heat_z0=6,
                  heated_layers=5)
        okw = dict(region_shape="cylinder", heat_radius=3.0, design_radius=7.5, heat_z0=6, heated_layers=5)
    d, h = region_masks(n, n, nz, _abi.default_params(bc=_abi.NC_BC_CAVITY, **kw))
    op = oracle.Problem(oracle.Mesh(n, n, nz, 1.0 / nz), oracle.Params(bc="cavity", **okw))
    assert np.array_equal(d.numpy(), op.design) and np.array_equal(h.numpy(), op.heated)


def test_full_size_geometries_validate():
    """The paper's two set-ups at their full meshes pass the library's parameter validation and fit in
    one GPU's memory: the Sec. 6.1 cavity on 80 x 80 x 160 and the Sec. 7 cylinder on 160 x 160 x 320
    (both coarsen to a 5 x 5 x 10 coarsest level, 792 rows)."""
    from paper_1904_00182_gb300 import Grid, default_params, footprint_bytes
    from paper_1904_00182_gb300.optimize import cavity_params, cylinder_params
    for n, geom in ((80, cavity_params(80)), (160, cylinder_params(160))):
        p = default_params(**geom)
        b = footprint_bytes(Grid(n, n, 2 * n, 1.0 / (2 * n)), p)
        assert 0 < b < 40e9, (n, b)


class _OracleEvaluator:
    """f and df/drho of the FP64 oracle (Sec. 5.1 adjoint, filter transpose), with the same warm start
    (Sec. 5.4) and the same region parameters as the library's evaluator."""

    def __init__(self, n, alpha, lib_params, rtol):
        import oracle
        self.oracle = oracle
        self.n, self.alpha, self.rtol = n, alpha, rtol
        self.params = lib_params
        self.overrides = {}
        self.op = self._make()
        self.kappa_f = self.op.par.kappa_f
        self.state = None

    def _make(self):
        o = self.oracle
        return o.Problem(o.Mesh(self.n, self.n, self.n, 1.0 / self.n),
                         o.Params(alpha=self.alpha, newton_rtol=self.rtol, **self.overrides))

    def set_stage(self, **overrides):
        self.overrides.update(overrides)
        self.op = self._make()

    def __call__(self, rho):
        import torch
        op = self.op
        op.set_design(rho.cpu().numpy())
        op.solve_state(s0=self.state)
        self.state = op.s.copy()
        op.solve_adjoint()
        return op.objective(), torch.from_numpy(op.sensitivities()), {}

    def close(self):
        pass


@pytest.mark.gpu
def test_optimisation_iterates_follow_the_oracle():
    """Three MMA iterations of Eq. optprob (Sec. 5.1-5.3) driven by the library's objective and
    adjoint gradient give the same iterates as three driven by the oracle's, from the same start."""
    from paper_1904_00182_gb300 import build
    build.build()
    from paper_1904_00182_gb300.optimize import LibraryEvaluator, optimize
    n, alpha, rtol = 8, 1e4, 1e-10
    stages = ({"q_c": 8.81, "q_p": 8.0},)
    lib = LibraryEvaluator(n, n, n, alpha, newton_rtol=rtol)
    a = optimize(n, n, n, alpha, 0.2, 3, stages=stages, evaluator=lib, keep_iterates=True)
    ora = _OracleEvaluator(n, alpha, lib.params, rtol)
    assert ora.kappa_f == pytest.approx(lib.kappa_f, rel=1e-14)
    b = optimize(n, n, n, alpha, 0.2, 3, stages=stages, evaluator=ora, device="cpu", keep_iterates=True)
    lib.close()
    for ra, rb in zip(a["history"], b["history"]):
        assert ra["f"] == pytest.approx(rb["f"], rel=1e-6), (ra["it"], ra["f"], rb["f"])
        dx = float((ra["x"].cpu() - rb["x"]).abs().max())
        assert dx <= 1e-6, (ra["it"], dx)
    assert a["history"][-1]["f"] < a["history"][0]["f"]
    assert float((a["history"][-1]["x"].cpu() - a["history"][0]["x"].cpu()).abs().max()) > 1e-3   # the design moved
