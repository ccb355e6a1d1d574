"""The fact behind the spectral filter solve: the cosine matrix C_ij = cos(pi i j / n) diagonalises
both the 1D Q1 stiffness matrix (1/h) tridiag(-1, 2, -1) and the consistent mass matrix
(h/6) tridiag(1, 4, 1) with Neumann ends (end diagonals halved), so the 3D filter operator
r^2 (K M M + M K M + M M K) + M M M is inverted by x = C3 D^-1 C3 b with D the products of the 1D
diagonals. Checked in float64 on several sizes, the 3D formula against a dense solve of the
assembled operator; the per-axis eigenvalue formulas of the library's set-up (v^T K v, v^T M v with
the assembled tridiagonals) are restated here from their definitions."""

import numpy as np
import pytest


def _mats(n, h):
    K = np.zeros((n + 1, n + 1))
    M = np.zeros((n + 1, n + 1))
    for e in range(n):
        K[e:e + 2, e:e + 2] += np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
        M[e:e + 2, e:e + 2] += np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0
    return K, M


def _cos(n):
    i = np.arange(n + 1)
    return np.cos(np.pi * np.outer(i, i) / n)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 33])
def test_cosine_basis_diagonalises_1d_stiffness_and_mass(n):
    h = 0.3
    K, M = _mats(n, h)
    C = _cos(n)
    for A in (K, M):
        D = C.T @ A @ C
        off = D - np.diag(np.diag(D))
        assert np.abs(off).max() <= 1e-12 * np.abs(D).max()


def test_three_dimensional_solve_matches_dense():
    nx, ny, nz, h = 4, 3, 6, 0.25
    r = 2.5 * h / (2.0 * np.sqrt(3.0))
    (Kx, Mx), (Ky, My), (Kz, Mz) = _mats(nx, h), _mats(ny, h), _mats(nz, h)
    kr = np.kron
    # node index i + NX j + NXY k: Kronecker order (z, y, x)
    A = r * r * (kr(Mz, kr(My, Kx)) + kr(Mz, kr(Ky, Mx)) + kr(Kz, kr(My, Mx))) + kr(Mz, kr(My, Mx))
    Cx, Cy, Cz = _cos(nx), _cos(ny), _cos(nz)
    eig = [(np.einsum("ij,ik,kj->j", C, Km, C), np.einsum("ij,ik,kj->j", C, Mm, C))
           for C, Km, Mm in ((Cx, Kx, Mx), (Cy, Ky, My), (Cz, Kz, Mz))]
    (lx, mx), (ly, my), (lz, mz) = eig
    D = (r * r * (np.einsum("k,j,i->kji", mz, my, lx) + np.einsum("k,j,i->kji", mz, ly, mx)
                  + np.einsum("k,j,i->kji", lz, my, mx)) + np.einsum("k,j,i->kji", mz, my, mx))
    b = np.random.default_rng(3).standard_normal(A.shape[0])

    def c3(v):
        v = np.einsum("ai,kji->kja", Cx, v)
        v = np.einsum("bj,kja->kba", Cy, v)
        return np.einsum("ck,kba->cba", Cz, v)

    x = c3(c3(b.reshape(nz + 1, ny + 1, nx + 1)) / D).ravel()
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12 * np.abs(x).max())
