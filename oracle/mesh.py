"""Structured hexahedral grid for the oracle (test infrastructure only).

The paper discretises a box with uniform trilinear hexahedra on a structured mesh
(Sec. 4 "Finite element formulation"; Sec. 6.2 uses 80x80x160 bricks). Here a grid is
``nx x ny x nz`` cubic elements of edge ``h``; nodes are numbered x fastest:
``node(i, j, k) = i + (nx+1) * (j + (ny+1) * k)``. Element ``(i, j, k)`` spans nodes
``(i..i+1, j..j+1, k..k+1)``; its local node ``a = ax + 2 ay + 4 az`` is node
``(i+ax, j+ay, k+az)``. Gravity points along -z.
"""

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Mesh:
    nx: int
    ny: int
    nz: int
    h: float

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_elems(self) -> int:
        return self.nx * self.ny * self.nz

    def node_index(self, i, j, k):
        return np.asarray(i) + (self.nx + 1) * (np.asarray(j) + (self.ny + 1) * np.asarray(k))

    def node_ijk(self):
        """Integer (i, j, k) of every node, shape (n_nodes, 3)."""
        k, j, i = np.meshgrid(np.arange(self.nz + 1), np.arange(self.ny + 1),
                              np.arange(self.nx + 1), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def node_coords(self):
        return self.node_ijk().astype(np.float64) * self.h

    def elem_ijk(self):
        """Integer (i, j, k) of every element, shape (n_elems, 3); element e = i + nx*(j + ny*k)."""
        k, j, i = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                              indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def connectivity(self):
        """Global node of each element's 8 local nodes, shape (n_elems, 8)."""
        e = self.elem_ijk()
        conn = np.empty((self.n_elems, 8), dtype=np.int64)
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            conn[:, a] = self.node_index(e[:, 0] + ax, e[:, 1] + ay, e[:, 2] + az)
        return conn

    def elem_centroids(self):
        return (self.elem_ijk().astype(np.float64) + 0.5) * self.h

    def top_nodes(self):
        """Boolean mask of the nodes on the top face z = nz*h."""
        return self.node_ijk()[:, 2] == self.nz

    def heated_elems(self, layers: int):
        """Boolean mask of the elements in the bottom ``layers`` element layers."""
        return self.elem_ijk()[:, 2] < layers

    def box_elems(self, nx, ny, z0, z1):
        """Boolean mask of the elements with i < nx, j < ny and z0 <= k < z1 (a box at the corner x = y = 0)."""
        e = self.elem_ijk()
        return (e[:, 0] < nx) & (e[:, 1] < ny) & (e[:, 2] >= z0) & (e[:, 2] < z1)

    def cylinder_elems(self, radius, z0, z1, inner=0.0):
        """Boolean mask of the elements whose centroid lies at distance in [inner, radius) (element sizes)
        from the z axis through the corner x = y = 0, in the layers z0 <= k < z1 (Sec. 7's suspended
        cylinder and the annulus around it, quarter domain)."""
        e = self.elem_ijk()
        r2 = (e[:, 0] + 0.5) ** 2 + (e[:, 1] + 0.5) ** 2
        return (r2 < radius ** 2) & (r2 >= inner ** 2) & (e[:, 2] >= z0) & (e[:, 2] < z1)

    def cavity_dirichlet(self):
        """(maskP, maskT) of the quarter cavity of Sec. 6.1 (symmetry planes x = 0 and y = 0): T fixed on
        the outer walls x = nx h, y = ny h and on the top; P fixed at the top outer corner."""
        ijk = self.node_ijk()
        maskT = (ijk[:, 0] == self.nx) | (ijk[:, 1] == self.ny) | (ijk[:, 2] == self.nz)
        maskP = (ijk[:, 0] == self.nx) & (ijk[:, 1] == self.ny) & (ijk[:, 2] == self.nz)
        return maskP, maskT

    def extent(self):
        return (self.nx * self.h, self.ny * self.h, self.nz * self.h)
