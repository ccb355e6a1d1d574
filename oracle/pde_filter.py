"""PDE (Helmholtz) density filter (test infrastructure only).

Sec. 5.1 regularises the design with a PDE-based filter (Lazarov & Sigmund 2011; Aage et al.
2014) and Sec. 6.3 sets its radius to 2.5 element sizes. The paper gives no formula, so the
cited filter is written out here (readings listed in the design doc):

* continuous form  -r^2 lap(x) + x = gamma  with homogeneous Neumann conditions on the box;
* r = R / (2 sqrt 3) with R the filter radius (the Lazarov-Sigmund radius convention);
* Q1 nodal unknowns x, element-constant gamma: (r^2 K + M) x = T^T gamma, with
  T_{e,i} = int_e N_i dOmega;
* element value gamma~_e = mean of its 8 nodal values.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import shape_tables


class HelmholtzFilter:
    def __init__(self, mesh, radius_elems):
        self.mesh = mesh
        h = mesh.h
        self.r = radius_elems * h / (2.0 * np.sqrt(3.0))
        N, D, w, _, _ = shape_tables(h)
        self.K0 = w * np.einsum("qai,qbi->ab", D, D)
        self.M0 = w * np.einsum("qa,qb->ab", N, N)
        self.t0 = w * N.sum(axis=0)                 # int_e N_a, equal to h^3/8
        self.conn = mesh.connectivity()
        Ae = self.r ** 2 * self.K0 + self.M0
        rows = np.repeat(self.conn, 8, axis=1).ravel()
        cols = np.tile(self.conn, (1, 8)).ravel()
        vals = np.tile(Ae.ravel(), mesh.n_elems)
        n = mesh.n_nodes
        self.A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
        self._lu = spla.splu(self.A)

    def rhs(self, gamma):
        """T^T gamma: node i collects gamma_e int_e N_i from its elements."""
        b = np.zeros(self.mesh.n_nodes)
        np.add.at(b, self.conn, gamma[:, None] * self.t0[None, :])
        return b

    def nodal(self, gamma):
        return self._lu.solve(self.rhs(gamma))

    def apply(self, gamma):
        """gamma~ (per element) from gamma (per element)."""
        x = self.nodal(gamma)
        return x[self.conn].mean(axis=1)

    def apply_transpose(self, g_tilde):
        """Adjoint of ``apply``: the gradient with respect to gamma of sum(g_tilde * gamma~)."""
        b = np.zeros(self.mesh.n_nodes)
        np.add.at(b, self.conn, np.repeat(g_tilde[:, None] / 8.0, 8, axis=1))
        y = self._lu.solve(b)                        # A is symmetric
        return (y[self.conn] * self.t0[None, :]).sum(axis=1)
