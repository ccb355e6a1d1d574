"""Pins of the oracle's sampled-row helpers, which carry every check at grids too large to assemble.

``Problem.residual_at_nodes`` (rows of R(s) of Eq. finalsyseq, built from the elements around the
chosen nodes only) and ``Problem.jt_at_nodes`` (rows of J(s)^T lambda, the adjoint operator of
Sec. 5.1, with lambda taken as zero on the Dirichlet rows) must equal the same rows of the fully
assembled operators: ``residual_raw`` (pinned by the closed forms, the divergence invariant and the
energy balance) and ``jacobian_full`` (pinned by central differences of R). Every node of small
ragged grids is checked, so corners, edges, the top and bottom planes, the symmetry planes and each
fixed set (the top plane of the base-plate set-up; the outer walls, top and pressure corner of the
closed cavity of Sec. 6.1) are all covered, at random states with a random design.
"""

import numpy as np
import pytest

from oracle import Mesh, Params, Problem

CASES = {
    "top": (6, 5, 7, dict(alpha=1e4)),
    "cavity": (4, 4, 8, dict(alpha=1e4, bc="cavity", heat_nx=2, heat_ny=1, heated_layers=2,
                             design_nx=3, design_ny=3, design_nz=4, Q=20.0)),
    "cylinder": (6, 6, 8, dict(alpha=1e5, bc="cavity", region_shape="cylinder", heat_radius=2.0,
                               design_radius=4.0, heat_z0=3, heated_layers=2)),
}


def _problem(case, seed):
    nx, ny, nz, kw = CASES[case]
    pr = Problem(Mesh(nx, ny, nz, 1.0 / nz), Params(**kw))
    rng = np.random.default_rng(seed)
    pr.set_design(rng.uniform(0.0, 1.0, pr.mesh.n_elems))
    n2 = 2 * pr.mesh.n_nodes
    # a state with O(1) temperatures and pressures of the buoyancy scale, so that every term of the
    # residual (Darcy flux, buoyancy, convection with SUPG, diffusion, source) contributes
    s = rng.standard_normal(n2)
    s[0::2] *= pr.par.alpha * 0.1
    return pr, s, rng


@pytest.mark.parametrize("case", sorted(CASES))
def test_residual_at_nodes_equals_assembled_rows(case):
    pr, s, _ = _problem(case, 3)
    nodes = np.arange(pr.mesh.n_nodes)
    got = pr.residual_at_nodes(s, nodes)
    ref = pr.residual_raw(s).reshape(-1, 2)
    scale = np.abs(ref).max(axis=0)
    assert np.all(scale > 0.0)
    err = np.abs(got - ref).max(axis=0) / scale
    assert np.all(err <= 1e-13), err


@pytest.mark.parametrize("case", sorted(CASES))
def test_residual_at_nodes_subset_and_order(case):
    """An arbitrary subset in arbitrary order (repeats included) gives the same rows."""
    pr, s, rng = _problem(case, 4)
    ref = pr.residual_raw(s).reshape(-1, 2)
    nodes = rng.integers(0, pr.mesh.n_nodes, 40)
    got = pr.residual_at_nodes(s, nodes)
    scale = np.abs(ref).max(axis=0)
    assert np.all(np.abs(got - ref[nodes]).max(axis=0) <= 1e-13 * scale)


@pytest.mark.parametrize("case", sorted(CASES))
def test_jt_at_nodes_equals_assembled_transpose(case):
    pr, s, rng = _problem(case, 5)
    lam = rng.standard_normal(s.size)
    # the adjoint lives on the free DOFs: Dirichlet entries of lambda must not contribute
    lam[pr.dir_mask] = 1e3 * rng.standard_normal(int(pr.dir_mask.sum()))
    lam_free = np.where(pr.dir_mask, 0.0, lam)
    ref = (pr.jacobian_full(s).T @ lam_free).reshape(-1, 2)
    nodes = np.arange(pr.mesh.n_nodes)
    got = pr.jt_at_nodes(s, lam, nodes)
    scale = np.abs(ref).max(axis=0)
    assert np.all(scale > 0.0)
    err = np.abs(got - ref).max(axis=0) / scale
    assert np.all(err <= 1e-13), err


def test_jt_at_nodes_is_the_adjoint_of_the_jacobian_product():
    """<J^T lam, v> = <lam, J v> on the free DOFs, with J v from the matrix-free product jvp_raw
    (an independent code path from the assembled element Jacobians used by jt_at_nodes)."""
    pr, s, rng = _problem("top", 6)
    lam = np.where(pr.dir_mask, 0.0, rng.standard_normal(s.size))
    v = np.where(pr.dir_mask, 0.0, rng.standard_normal(s.size))
    jt = pr.jt_at_nodes(s, lam, np.arange(pr.mesh.n_nodes)).ravel()
    lhs = float(jt @ v)
    rhs = float(lam @ pr.jvp_raw(s, v))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(jt).max() * np.abs(v).sum())


def test_sampled_rows_detect_a_dropped_element():
    """The pin is sharp: removing one boundary element from the neighbourhood of a corner node changes
    that node's row (guards against a neighbourhood that skips boundary-adjacent elements)."""
    pr, s, _ = _problem("top", 7)
    m = pr.mesh
    node = int(m.node_index(m.nx, 0, 0))            # corner: exactly one adjacent element
    el = pr._elements_around([node])
    assert list(el) == [m.nx - 1]
    ref = pr.residual_raw(s).reshape(-1, 2)[node]
    assert np.abs(ref).max() > 0.0
    node_mid = int(m.node_index(2, 2, 3))            # interior node: eight adjacent elements
    assert len(pr._elements_around([node_mid])) == 8
