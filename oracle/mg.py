"""Geometric multigrid used as the inner solves of the block preconditioners
(oracle; TEST INFRASTRUCTURE).

The paper approximates the inverses of its diagonal blocks with algebraic
multigrid from PyAMG (Sec. 4, Sec. 5).  On the structured meshes used here the
hierarchy is geometric: meshes n, n/2, ... while the size is even and at least
4; coarse operators are rediscretised with coefficients injected to the coarse
nodes; prolongation is nodal interpolation (linear for P1, quadratic for P2,
exact for the nested spaces) and restriction its transpose.  One V-cycle:
Chebyshev-Jacobi pre-smoothing from x = 0, coarse correction, post-smoothing;
dense LU with partial pivoting on the coarsest mesh while it has at most
COARSE_DENSE_MAX unknowns (always for the pressure Laplacian, dense_coarse),
else COARSE_DEGREE Chebyshev-Jacobi steps from zero on [hi / COARSE_RATIO,
hi] (the other blocks are mass-dominated on a coarse mesh, so a fixed
polynomial solves them well; a dense inverse of a 25 x 25 velocity level
would have 5202 rows).  Smoother interval
[hi / ratio, hi] with hi the Gershgorin bound max_i sum_j |a_ij| / |a_ii| of
D^{-1} A: degree 2, ratio 4 for the scalar P1 operators; degree 4, ratio 16
for the Taylor-Hood velocity operator (the paper leaves the AMG smoothing to
PyAMG; these values minimise the Oseen iteration count at fixed cost).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .krylov import chebyshev
from .mesh import Mesh
from . import fem

SMOOTH_DEGREE = 2
LO_RATIO = 4.0
VEL_SMOOTH_DEGREE = 4
VEL_LO_RATIO = 16.0
COARSE_DENSE_MAX = 256
COARSE_DEGREE = 16
COARSE_RATIO = 64.0


def level_sizes(n: int):
    sizes = [n]
    while sizes[-1] % 2 == 0 and sizes[-1] >= 4:
        sizes.append(sizes[-1] // 2)
    return sizes


def _bary(xi, eta):
    """Containing triangle (0 lower / 1 upper) and barycentric coordinates of
    a point with cell-local coordinates (xi, eta) in [0,1]^2."""
    lower = xi >= eta
    lam = np.where(lower[:, None],
                   np.stack([1 - xi, xi - eta, eta], axis=1),
                   np.stack([1 - eta, xi, eta - xi], axis=1))
    return lower, lam


def _locate(nc, X, Y):
    """X, Y in units of coarse cells; returns cell (i, j), local (xi, eta)."""
    i = np.minimum(np.floor(X).astype(np.int64), nc - 1)
    j = np.minimum(np.floor(Y).astype(np.int64), nc - 1)
    return i, j, X - i, Y - j


def prolongation_p1(coarse: Mesh):
    """Interpolate coarse P1 functions at the fine (2nc) P1 nodes."""
    nc = coarse.n
    nf = 2 * nc
    I, J = np.meshgrid(np.arange(nf + 1), np.arange(nf + 1), indexing="xy")
    X, Y = I.ravel() / 2.0, J.ravel() / 2.0
    i, j, xi, eta = _locate(nc, X, Y)
    lower, lam = _bary(xi, eta)
    e = 2 * (j * nc + i) + (~lower).astype(np.int64)
    cols = coarse.tri[e]                                       # (Nf,3)
    rows = np.repeat(np.arange(X.size), 3)
    P = sp.coo_matrix((lam.ravel(), (rows, cols.ravel())), shape=(X.size, coarse.N1)).tocsr()
    P.eliminate_zeros()
    return P


def prolongation_p2(coarse: Mesh):
    """Interpolate coarse P2 functions at the fine P2 nodes."""
    nc = coarse.n
    m = 4 * nc + 1                                             # fine refined lattice
    I, J = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    X, Y = I.ravel() / 4.0, J.ravel() / 4.0
    i, j, xi, eta = _locate(nc, X, Y)
    lower, lam = _bary(xi, eta)
    e = 2 * (j * nc + i) + (~lower).astype(np.int64)
    w = fem.p2_values(lam)                                    # (Nf,6)
    cols = coarse.tri2[e]
    rows = np.repeat(np.arange(X.size), 6)
    P = sp.coo_matrix((w.ravel(), (rows, cols.ravel())), shape=(X.size, coarse.N2)).tocsr()
    P.sum_duplicates()
    P.eliminate_zeros()
    return P


def prolongation_velocity(coarse: Mesh, fine: Mesh):
    """Quadratic interpolation per component, restricted to interior
    (non-Dirichlet) nodes on both meshes."""
    P = prolongation_p2(coarse)
    Df = sp.diags((~fine.p2_boundary()).astype(float))
    Dc = sp.diags((~coarse.p2_boundary()).astype(float))
    P = (Df @ P @ Dc).tocsr()
    P.eliminate_zeros()
    return sp.kron(P, sp.eye(2), format="csr")


def inject_p1(f, nf):
    """Values of a fine P1 field at the coarse (nf/2) vertices."""
    F = f.reshape(nf + 1, nf + 1)
    return np.ascontiguousarray(F[::2, ::2]).ravel()


def inject_velocity(v, nf):
    """Values of a fine P2 velocity at the coarse P2 nodes (fine lattice
    points (2a, 2b) of the refined lattice)."""
    m = 2 * nf + 1
    V = v.reshape(m, m, 2)
    return np.ascontiguousarray(V[::2, ::2, :]).ravel()


class MG:
    """One V-cycle of geometric multigrid for a hierarchy of matrices."""

    def __init__(self, mats, prolongs, singular=False, degree=None, ratio=None, dense_coarse=False, his=None):
        """his: per-level upper ends of the smoothing intervals in place of
        the Gershgorin bounds (the algebraic hierarchies of oracle.amg)."""
        self.mats = mats
        self.degree = SMOOTH_DEGREE if degree is None else degree
        self.ratio = LO_RATIO if ratio is None else ratio
        self.P = prolongs                     # P[l]: level l+1 -> level l
        self.singular = singular
        self.dinv, self.hi = [], []
        for l, A in enumerate(mats[:-1]):
            d = A.diagonal()
            self.dinv.append(1.0 / d)
            absA = abs(A)
            self.hi.append(float(np.max(np.asarray(absA.sum(axis=1)).ravel() / np.abs(d)))
                           if his is None else float(his[l]))
        self.coarse_iter = (len(mats) > 1 and not singular and not dense_coarse
                            and mats[-1].shape[0] > COARSE_DENSE_MAX)
        if self.coarse_iter:
            A = mats[-1]
            d = A.diagonal()
            self.cdinv = 1.0 / d
            self.chi = (float(np.max(np.asarray(abs(A).sum(axis=1)).ravel() / np.abs(d)))
                        if his is None else float(his[-1]))
            self.lu = None
        else:
            Ac = mats[-1].toarray()
            if singular:
                Ac = Ac + np.ones_like(Ac)
            self.lu = sla.lu_factor(Ac)

    def vcycle(self, b, level=0):
        if level == len(self.mats) - 1:
            if self.coarse_iter:
                A = self.mats[level]
                return chebyshev(lambda y: A @ y, self.cdinv, b, None, self.chi / COARSE_RATIO, self.chi,
                                 COARSE_DEGREE)
            return sla.lu_solve(self.lu, b)
        A = self.mats[level]
        dinv, hi = self.dinv[level], self.hi[level]
        lo = hi / self.ratio
        x = chebyshev(lambda y: A @ y, dinv, b, None, lo, hi, self.degree)
        r = b - A @ x
        P = self.P[level]
        ec = self.vcycle(P.T @ r, level + 1)
        x = x + P @ ec
        return chebyshev(lambda y: A @ y, dinv, b, x, lo, hi, self.degree)

    def __call__(self, b):
        if self.singular:
            b = b - b.mean()
            x = self.vcycle(b)
            return x - x.mean()
        return self.vcycle(b)

    def solve(self, b, rtol, maxit):
        """Multigrid as an inner solver with a tolerance (Sec. 5: the AMG
        preconditioners are applied to a relative tolerance): the stationary
        iteration x <- x + V(b - A x) from x = 0, stopped once
        ||b - A x|| <= rtol ||b|| or after maxit V-cycles.  Returns (x, cycles).
        For the singular pressure Laplacian b is first projected to mean
        zero, and every V-cycle projects its input and output."""
        A = self.mats[0]
        if self.singular:
            b = b - b.mean()
        nb = float(np.linalg.norm(b))
        x = self(b)
        r = b - A @ x
        cycles = 1
        while float(np.linalg.norm(r)) > rtol * nb and cycles < maxit:
            x = x + self(r)
            r = b - A @ x
            cycles += 1
        return x, cycles

    def inner(self, params):
        """The block inverse a preconditioner applies: one V-cycle
        (params["inner_rtol"] = 0) or solve() to inner_rtol."""
        rtol = params.get("inner_rtol", 0.0)
        if not rtol:
            return self
        maxit = params.get("inner_maxit", 20)
        return lambda b: self.solve(b, rtol, maxit)[0]
