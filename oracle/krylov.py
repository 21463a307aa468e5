"""Krylov solvers and Chebyshev iteration (oracle; TEST INFRASTRUCTURE).

FGMRES(m) with right preconditioning (Saad, Iterative Methods, Sec. 9.4),
classical Gram-Schmidt applied twice, Givens rotations, x0 = 0, and the
stopping rule of Sec. 5: ||b - A z|| <= max(rtol ||b||, atol) on the true
residual.  When the Arnoldi estimate |g_{j+1}| meets the target, or the
restart length is reached, the iterate is formed and its true residual
decides; if it fails, GMRES restarts from that residual.
"""
from __future__ import annotations

import math
import numpy as np


def fgmres(apply_A, apply_P, b, rtol=1e-8, atol=0.0, restart=30, maxit=600):
    """Returns (x, info) with info = dict(iters, rel_residual, converged)."""
    n = b.shape[0]
    x = np.zeros(n)
    bnorm = float(np.linalg.norm(b))
    target = max(rtol * bnorm, atol)
    r = b.copy()
    rnorm = bnorm
    iters = 0
    if rnorm <= target:
        return x, {"iters": 0, "rel_residual": 0.0 if bnorm == 0 else rnorm / bnorm, "converged": True}
    m = restart
    while True:
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = rnorm
        V[0] = r / rnorm
        k = 0
        for j in range(m):
            Z[j] = apply_P(V[j])
            w = apply_A(Z[j])
            h1 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h1
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            hn = float(np.linalg.norm(w))
            H[: j + 1, j] = h1 + h2
            H[j + 1, j] = hn
            for i in range(j):                     # previous rotations
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            breakdown = hn == 0.0
            if not breakdown:
                V[j + 1] = w / hn
            if abs(g[j + 1]) <= target or iters >= maxit or breakdown:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):             # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        r = b - apply_A(x)
        rnorm = float(np.linalg.norm(r))
        if rnorm <= target:
            return x, {"iters": iters, "rel_residual": rnorm / bnorm, "converged": True}
        if iters >= maxit:
            return x, {"iters": iters, "rel_residual": rnorm / bnorm, "converged": False}


def pcg(A, b, dinv, rtol=1e-12, atol=0.0, maxit=1000):
    """Jacobi-preconditioned conjugate gradients (Hestenes-Stiefel), x0 = 0,
    stop on ||r|| <= max(rtol ||b||, atol) with the recursive residual."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = float(np.linalg.norm(b))
    target = max(rtol * bnorm, atol)
    if bnorm <= target:
        return x, {"iters": 0, "rel_residual": 0.0, "converged": True}
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rn = float(np.linalg.norm(r))
        if rn <= target:
            return x, {"iters": it, "rel_residual": rn / bnorm, "converged": True}
        z = dinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, {"iters": it, "rel_residual": float(np.linalg.norm(r)) / bnorm, "converged": False}


def chebyshev(apply_A, dinv, b, x0, lo, hi, degree):
    """Chebyshev acceleration of Jacobi on D^{-1} A with spectrum bounds
    [lo, hi] (Saad, Iterative Methods, Alg. 12.1 on the preconditioned
    operator): x <- x + q(D^{-1}A) D^{-1} (b - A x) where q has degree
    ``degree`` - 1 and 1 - l q(l) = T_d((hi + lo - 2 l) / (hi - lo)) /
    T_d((hi + lo) / (hi - lo)), d = ``degree``.  x0 = None means x0 = 0."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - apply_A(x)
    d = dinv * r / theta
    for k in range(degree):
        x = x + d
        if k == degree - 1:
            break
        r = r - apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x
