"""Collapsed (Duffy) Gauss-Legendre rules on the reference triangle.

The paper assembles with DOLFINx and does not state its quadrature; the
oracle integrates every form exactly for the polynomial degree of its
integrand (P1/P2 bases, P1 fields, the polynomial potential eqn:appPotential).
Map (s, t) in [0,1]^2 to xi = s, eta = t (1 - s), Jacobian (1 - s); a
Gauss-Legendre rule with k points is exact to degree 2k - 1 in each variable.
"""
from __future__ import annotations

import numpy as np


def triangle_rule(degree: int):
    """Barycentric points (Q,3) and weights (Q,) with sum(w) = 1, so that
    integral_T g = |T| * sum_q w_q g(lambda_q) for polynomials g of total
    degree <= ``degree``."""
    kt = (degree + 2) // 2              # exact in t to degree 2kt-1 >= degree
    ks = (degree + 3) // 2              # (1-s) factor raises the s-degree by 1
    xs, ws = np.polynomial.legendre.leggauss(ks)
    xt, wt = np.polynomial.legendre.leggauss(kt)
    s, wsu = 0.5 * (xs + 1.0), 0.5 * ws
    t, wtu = 0.5 * (xt + 1.0), 0.5 * wt
    S, T = np.meshgrid(s, t, indexing="ij")
    W = np.outer(wsu, wtu) * (1.0 - S)
    xi = S.ravel()
    eta = (T * (1.0 - S)).ravel()
    lam = np.stack([1.0 - xi - eta, xi, eta], axis=1)
    w = 2.0 * W.ravel()                 # reference area is 1/2
    return lam, w


def edge_rule(degree: int):
    """Gauss-Legendre points in [0, 1] (parameter along an edge) and weights
    summing to 1, exact to ``degree``."""
    k = degree // 2 + 1
    x, w = np.polynomial.legendre.leggauss(k)
    return 0.5 * (x + 1.0), 0.5 * w


def tetra_rule(degree: int):
    """Barycentric points (Q,4) and weights (Q,) with sum(w) = 1, so that
    integral_T g = |T| * sum_q w_q g(lambda_q) on a tetrahedron for
    polynomials g of total degree <= ``degree``.  Collapsed map (s, t, u) in
    [0,1]^3 to xi = s, eta = t (1 - s), zeta = u (1 - s)(1 - t), Jacobian
    (1 - s)^2 (1 - t): Gauss-Legendre in each variable, exact to the raised
    degrees degree + 2 (s), degree + 1 (t), degree (u)."""
    ks, kt, ku = (degree + 4) // 2, (degree + 3) // 2, (degree + 2) // 2
    rules = [np.polynomial.legendre.leggauss(k) for k in (ks, kt, ku)]
    (xs, ws), (xt, wt), (xu, wu) = [(0.5 * (x + 1.0), 0.5 * w) for x, w in rules]
    S, T, U = np.meshgrid(xs, xt, xu, indexing="ij")
    W = np.einsum("i,j,k->ijk", ws, wt, wu) * (1.0 - S) ** 2 * (1.0 - T)
    xi = S.ravel()
    eta = (T * (1.0 - S)).ravel()
    zeta = (U * (1.0 - S) * (1.0 - T)).ravel()
    lam = np.stack([1.0 - xi - eta - zeta, xi, eta, zeta], axis=1)
    return lam, 6.0 * W.ravel()         # reference volume 1/6

