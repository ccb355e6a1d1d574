"""Pins of the oracle's frozen-coefficient (Picard) operator, the cheaper finest-level operator the
library's multigrid can use in place of the exact Jacobian (the flexible Krylov solver of Sec. 5.4
admits a preconditioner that differs from J).

* Where the state has no flow and no source (s = 0, Q = 0) nothing is frozen away: the operator equals
  the exact Jacobian (pinned by central differences of R).
* Where the Darcy velocity is uniform inside every element (P linear, T constant, so u_q = u0) and there
  is no source, the dropped terms (du . grad T, the variation of u over the element, d tau S, tau S du0)
  all vanish: the operator again equals the exact Jacobian, for every direction.
* At a general state the continuity rows equal the Jacobian's, the energy rows do not depend on dP, and
  the operator differs from J (so the pins above are sharp).
"""

import numpy as np

from oracle import Mesh, Params, Problem


def _problem(Q=None, alpha=1e4, n=(5, 4, 6), seed=1):
    nx, ny, nz = n
    par = Params(alpha=alpha, Q=Q)
    pr = Problem(Mesh(nx, ny, nz, 1.0 / nz), par)
    rng = np.random.default_rng(seed)
    pr.set_design(rng.uniform(0.0, 0.2, pr.mesh.n_elems))    # mostly fluid: flow carries heat
    return pr, rng


def test_equals_jacobian_without_flow_and_source():
    pr, rng = _problem(Q=0.0)
    pr.Qe[:] = 0.0
    s = np.zeros(2 * pr.mesh.n_nodes)
    A = pr.picard_matrix_full(s).toarray()
    J = pr.jacobian_full(s).toarray()
    assert np.abs(A - J).max() <= 1e-13 * np.abs(J).max()


def test_equals_jacobian_for_uniform_element_velocity():
    pr, rng = _problem(Q=0.0, alpha=3e3)
    pr.Qe[:] = 0.0
    xyz = pr.mesh.node_coords()
    s = np.zeros(2 * pr.mesh.n_nodes)
    s[0::2] = 40.0 * xyz[:, 0] - 25.0 * xyz[:, 1] + 60.0 * xyz[:, 2]     # linear P
    s[1::2] = 0.7                                                         # constant T
    for _ in range(3):
        v = rng.standard_normal(s.size)
        a = pr.picard_jvp_raw(s, v)
        b = pr.jvp_raw(s, v)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_structure_at_a_general_state():
    pr, rng = _problem()
    s = rng.standard_normal(2 * pr.mesh.n_nodes)
    s[0::2] *= 3e3 / pr.par.kappa_f                                   # Darcy speeds of order 1e3
    A = pr.picard_matrix_full(s).toarray()
    J = pr.jacobian_full(s).toarray()
    scale = np.abs(J).max()
    assert np.abs(A[0::2] - J[0::2]).max() <= 1e-13 * scale        # continuity rows exact
    assert np.abs(A[1::2, 0::2]).max() == 0.0                       # energy rows ignore dP
    assert np.abs(A[1::2] - J[1::2]).max() > 0.1 * np.abs(J[1::2]).max()
    v = rng.standard_normal(s.size)
    assert np.allclose(pr.picard_jvp_raw(s, v), A @ v, rtol=0, atol=1e-12 * np.abs(A).max() * np.abs(v).sum())
