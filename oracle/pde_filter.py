"""PDE (Helmholtz) density filter (test infrastructure only).

Sec. 5.1 regularises the design with a PDE-based filter (Lazarov & Sigmund 2011; Aage et al.
2014) and Sec. 6.3 sets its radius to 2.5 element sizes. The paper gives no formula, so the
cited filter is written out here, with these readings:

* continuous form  -r^2 lap(x) + x = gamma  with homogeneous Neumann conditions on the box;
* r = R / (2 sqrt 3) with R the filter radius (the Lazarov-Sigmund radius convention);
* Q1 nodal unknowns x, element-constant gamma: (r^2 K + M) x = T^T gamma, with
  T_{e,i} = int_e N_i dOmega;
* element value gamma~_e = mean of its 8 nodal values.

Small grids use a sparse direct solve; large ones a matrix-free, Jacobi-preconditioned conjugate
gradient solve to a relative residual of 1e-14.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import shape_tables


class HelmholtzFilter:
    DIRECT_MAX_NODES = 60000

    def __init__(self, mesh, radius_elems):
        self.mesh = mesh
        h = mesh.h
        self.r = radius_elems * h / (2.0 * np.sqrt(3.0))
        N, D, w, _, _ = shape_tables(h)
        self.K0 = w * np.einsum("qai,qbi->ab", D, D)
        self.M0 = w * np.einsum("qa,qb->ab", N, N)
        self.t0 = w * N.sum(axis=0)                 # int_e N_a, equal to h^3/8
        self.conn = mesh.connectivity()
        self.Ae = self.r ** 2 * self.K0 + self.M0
        n = mesh.n_nodes
        self.direct = n <= self.DIRECT_MAX_NODES
        if self.direct:
            rows = np.repeat(self.conn, 8, axis=1).ravel()
            cols = np.tile(self.conn, (1, 8)).ravel()
            vals = np.tile(self.Ae.ravel(), mesh.n_elems)
            self.A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
            self._lu = spla.splu(self.A)
        else:
            # large grids: matrix-free element-by-element operator and Jacobi-preconditioned CG
            diag = np.zeros(n)
            np.add.at(diag, self.conn, np.diag(self.Ae)[None, :].repeat(mesh.n_elems, axis=0))
            self._dinv = 1.0 / diag

    def rhs(self, gamma):
        """T^T gamma: node i collects gamma_e int_e N_i from its elements."""
        b = np.zeros(self.mesh.n_nodes)
        np.add.at(b, self.conn, gamma[:, None] * self.t0[None, :])
        return b

    def matvec(self, x):
        """(r^2 K + M) x assembled element by element."""
        y = x[self.conn] @ self.Ae.T
        return np.bincount(self.conn.ravel(), y.ravel(), minlength=self.mesh.n_nodes)

    def solve(self, b):
        if self.direct:
            return self._lu.solve(b)
        n = self.mesh.n_nodes
        A = spla.LinearOperator((n, n), matvec=self.matvec, dtype=np.float64)
        M = spla.LinearOperator((n, n), matvec=lambda v: self._dinv * v, dtype=np.float64)
        x, info = spla.cg(A, b, rtol=1e-14, atol=0.0, M=M, maxiter=1000)
        if info != 0:
            raise RuntimeError("filter CG did not converge")
        return x

    def nodal(self, gamma):
        return self.solve(self.rhs(gamma))

    def apply(self, gamma):
        """gamma~ (per element) from gamma (per element)."""
        x = self.nodal(gamma)
        return x[self.conn].mean(axis=1)

    def apply_transpose(self, g_tilde):
        """Adjoint of ``apply``: the gradient with respect to gamma of sum(g_tilde * gamma~)."""
        b = np.zeros(self.mesh.n_nodes)
        np.add.at(b, self.conn, np.repeat(g_tilde[:, None] / 8.0, 8, axis=1))
        y = self.solve(b)                            # A is symmetric
        return (y[self.conn] * self.t0[None, :]).sum(axis=1)
