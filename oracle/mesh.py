"""Structured triangulation of a rectangle (paper Sec. 3 and Sec. 5: uniform
simplicial triangulations with n_x x n_y cells; P1 spaces for the phase
fields, potentials and pressure, P2 for the velocity, Taylor-Hood).

Oracle conventions (TEST INFRASTRUCTURE; see package docstring):
  * n x n squares of size (Lx/n) x (Ly/n); square (i, j) is split along
    its lower-left -> upper-right diagonal into
        lower triangle  (i, j), (i+1, j),   (i+1, j+1)
        upper triangle  (i, j), (i+1, j+1), (i, j+1)
    element id 2*(j*n + i) + {0 lower, 1 upper}.
  * P1 node (i, j) has id j*(n+1) + i.
  * P2 nodes live on the once-refined (2n+1) x (2n+1) lattice; P2 node
    (I, J) has id J*(2n+1) + I; vertex (i, j) is lattice point (2i, 2j).
  * Local P2 numbering: vertices 0, 1, 2, then the midpoints of the edges
    opposite vertex 0, 1, 2 (i.e. (1,2), (0,2), (0,1)).
"""
from __future__ import annotations

import numpy as np


class Mesh:
    """top_free: the velocity is not prescribed on the top edge (do-nothing
    condition there, no-slip on the other three sides); default: no-slip on
    the whole boundary (eqn:bc)."""

    def __init__(self, n: int, lx: float = 1.0, ly: float = 1.0, top_free: bool = False):
        if n < 1:
            raise ValueError("n must be >= 1")
        self.top_free = bool(top_free)
        self.n, self.lx, self.ly = n, float(lx), float(ly)
        self.hx, self.hy = self.lx / n, self.ly / n
        self.N1 = (n + 1) ** 2
        self.N2 = (2 * n + 1) ** 2
        self.E = 2 * n * n
        i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        i, j = i.ravel(), j.ravel()                      # square index s = j*n + i
        v = lambda a, b: b * (n + 1) + a               # noqa: E731  P1 id
        tri = np.empty((self.E, 3), dtype=np.int64)
        tri[0::2] = np.stack([v(i, j), v(i + 1, j), v(i + 1, j + 1)], axis=1)
        tri[1::2] = np.stack([v(i, j), v(i + 1, j + 1), v(i, j + 1)], axis=1)
        self.tri = tri
        # vertex lattice coordinates (I, J) on the refined lattice, per element
        lat_i = 2 * (tri % (n + 1))
        lat_j = 2 * (tri // (n + 1))
        m = 2 * n + 1
        mid = lambda a, b: ((lat_j[:, a] + lat_j[:, b]) // 2) * m + (lat_i[:, a] + lat_i[:, b]) // 2  # noqa: E731
        tri2 = np.empty((self.E, 6), dtype=np.int64)
        tri2[:, :3] = lat_j * m + lat_i
        tri2[:, 3] = mid(1, 2)
        tri2[:, 4] = mid(0, 2)
        tri2[:, 5] = mid(0, 1)
        self.tri2 = tri2
        ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
        self.x1 = np.stack([ii.ravel() * self.hx, jj.ravel() * self.hy], axis=1)
        II, JJ = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
        self.x2 = np.stack([II.ravel() * self.hx / 2, JJ.ravel() * self.hy / 2], axis=1)
        self.lat2 = np.stack([II.ravel(), JJ.ravel()], axis=1)

    # ------------------------------------------------------------------
    def p2_boundary(self) -> np.ndarray:
        """Boolean mask of P2 nodes with prescribed (zero) velocity: the whole
        boundary (eqn:bc), or all but the open top edge when top_free (its two
        corners stay on the side walls)."""
        m = 2 * self.n
        I, J = self.lat2[:, 0], self.lat2[:, 1]
        top = (J == m) & (not self.top_free)
        return (I == 0) | (I == m) | (J == 0) | top

    def p1_top(self) -> np.ndarray:
        """Boolean mask of P1 nodes on Gamma_t (y = Ly)."""
        return np.arange(self.N1) // (self.n + 1) == self.n

    def top_reference_node(self) -> int:
        """P1 node (x = Lx/2, y = Ly): the reference point of phi_s^vap (Sec. 2.1)."""
        if self.n % 2:
            raise ValueError("the top reference point needs an even n")
        return self.n * (self.n + 1) + self.n // 2

    def element_geometry(self):
        """Per element: vertex coordinates (E,3,2), area (E,), barycentric
        gradients (E,3,2) with grad(lambda_k) for the affine map."""
        X = self.x1[self.tri]                              # (E,3,2)
        Jm = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)  # columns
        det = Jm[:, 0, 0] * Jm[:, 1, 1] - Jm[:, 0, 1] * Jm[:, 1, 0]
        inv = np.empty_like(Jm)
        inv[:, 0, 0] = Jm[:, 1, 1] / det
        inv[:, 0, 1] = -Jm[:, 0, 1] / det
        inv[:, 1, 0] = -Jm[:, 1, 0] / det
        inv[:, 1, 1] = Jm[:, 0, 0] / det
        # lambda_1 = row 0 of inv applied to (x - x0), lambda_2 = row 1
        g = np.empty((self.E, 3, 2))
        g[:, 1] = inv[:, 0, :]
        g[:, 2] = inv[:, 1, :]
        g[:, 0] = -g[:, 1] - g[:, 2]
        return X, 0.5 * np.abs(det), g


class TriMesh(Mesh):
    """A general triangulation given by its vertex coordinates x (N, 2) and
    counter-clockwise triangles tri (E, 3): the P1 forms of oracle.fem that
    need only x1, tri, N1, E and element_geometry work on it unchanged (the
    P2 lattice of the structured mesh does not exist here)."""

    def __init__(self, x, tri):
        self.x1 = np.asarray(x, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        self.N1 = self.x1.shape[0]
        self.E = self.tri.shape[0]
        self.n = None
        self.top_free = False
