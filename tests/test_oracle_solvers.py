"""Pins of the oracle's solvers and preconditioners: textbook identities,
dense linear algebra, and the spectral bounds of Sec. 4 (CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, model
from oracle.krylov import chebyshev, fgmres, pcg
from oracle.mesh import Mesh
from oracle.mg import MG, VEL_LO_RATIO, VEL_SMOOTH_DEGREE, prolongation_p1, prolongation_velocity, level_sizes
from paper_2501_11767_gb300 import inputs


def _nonsym(n, seed):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 4 + rng.standard_normal((n, n)) / math.sqrt(n)


def test_fgmres_full_space_matches_dense_solve():
    A = _nonsym(40, 0)
    b = np.random.default_rng(1).standard_normal(40)
    x, info = fgmres(lambda y: A @ y, lambda y: y, b, rtol=1e-12, restart=40, maxit=40)
    assert info["converged"] and info["iters"] <= 40
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)


def test_fgmres_exact_preconditioner_one_iteration():
    A = _nonsym(30, 2)
    Ainv = np.linalg.inv(A)
    b = np.ones(30)
    x, info = fgmres(lambda y: A @ y, lambda y: Ainv @ y, b, rtol=1e-10)
    assert info["iters"] == 1
    assert np.allclose(A @ x, b, rtol=1e-10)


def test_fgmres_restart_and_zero_rhs():
    A = _nonsym(60, 3)
    b = np.random.default_rng(4).standard_normal(60)
    x, info = fgmres(lambda y: A @ y, lambda y: y, b, rtol=1e-10, restart=5, maxit=400)
    assert info["converged"] and info["iters"] > 5
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    x0, info0 = fgmres(lambda y: A @ y, lambda y: y, np.zeros(60))
    assert info0["iters"] == 0 and not np.any(x0)


def test_fgmres_reports_nonconvergence():
    A = _nonsym(60, 5)
    b = np.ones(60)
    x, info = fgmres(lambda y: A @ y, lambda y: y, b, rtol=1e-14, restart=3, maxit=4)
    assert not info["converged"] and info["iters"] == 4


def test_chebyshev_is_the_scaled_chebyshev_polynomial():
    """For D = I and A = diag(l), one application maps the error e to
    T_d((hi+lo-2l)/(hi-lo)) / T_d((hi+lo)/(hi-lo)) e."""
    lo, hi = 0.5, 2.0
    lam = np.linspace(0.3, 2.4, 23)
    A = np.diag(lam)
    xs = np.random.default_rng(0).standard_normal(lam.size)
    b = A @ xs
    x0 = np.random.default_rng(1).standard_normal(lam.size)
    for d in (1, 2, 3, 5):
        x = chebyshev(lambda y: A @ y, np.ones_like(lam), b, x0, lo, hi, d)
        c = np.zeros(d + 1); c[d] = 1
        factor = np.polynomial.chebyshev.chebval((hi + lo - 2 * lam) / (hi - lo), c) / \
            np.polynomial.chebyshev.chebval((hi + lo) / (hi - lo), c)
        assert np.allclose(xs - x, factor * (xs - x0), atol=1e-12)
        x = chebyshev(lambda y: A @ y, np.ones_like(lam), b, None, lo, hi, d)
        assert np.allclose(xs - x, factor * xs, atol=1e-12)


def test_pcg_matches_sparse_direct():
    mesh = Mesh(12)
    M = fem.mass_p1(mesh)
    b = np.random.default_rng(2).standard_normal(mesh.N1)
    x, info = pcg(M, b, 1.0 / M.diagonal(), rtol=1e-13)
    assert info["converged"]
    xe = spla.spsolve(M.tocsc(), b)
    assert np.linalg.norm(x - xe) <= 1e-11 * np.linalg.norm(xe)


def _contraction(mg, A, singular=False, its=12):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(A.shape[0])
    if singular:
        x -= x.mean()
    b = A @ x
    y = np.zeros_like(b)
    res = []
    for _ in range(its):
        y = y + mg(b - A @ y)
        e = x - y
        if singular:
            e -= e.mean()
        res.append(np.linalg.norm(e))
    return (res[-1] / res[3]) ** (1.0 / (its - 4))


def test_mg_contraction_is_mesh_independent():
    """V-cycle error contraction on the CH Schur factor X, the AC operator,
    the pressure Laplacian and the velocity operator stays bounded as h -> 0."""
    tau, a = 1e-3, math.sqrt(1e-3 / 4e-4)
    rates = {"X": [], "Kp": [], "vel": []}
    for n in (16, 32, 64):
        meshes = [Mesh(s) for s in level_sizes(n)]
        P1 = [prolongation_p1(meshes[l + 1]) for l in range(len(meshes) - 1)]
        X = [(tau * fem.stiffness_p1(m) + a * fem.mass_p1(m)).tocsr() for m in meshes]
        rates["X"].append(_contraction(MG(X, P1), X[0]))
        K = [fem.stiffness_p1(m) for m in meshes]
        rates["Kp"].append(_contraction(MG(K, P1, singular=True), K[0], singular=True))
        if n <= 32:
            Pv = [prolongation_velocity(meshes[l + 1], meshes[l]) for l in range(len(meshes) - 1)]
            V = []
            for m in meshes:
                Av = sp.kron(fem.mass_p2(m), sp.eye(2)) / tau + fem.ksym(m, 1.0)
                V.append(fem.velocity_dirichlet(Av.tocsr(), m.p2_boundary()))
            rates["vel"].append(_contraction(MG(V, Pv, degree=VEL_SMOOTH_DEGREE, ratio=VEL_LO_RATIO), V[0]))
    assert max(rates["X"]) < 0.15, rates
    assert max(rates["Kp"]) < 0.35, rates
    assert max(rates["vel"]) < 0.3, rates
    # the pure Laplacian is the h-independent case (X mixes mass and
    # stiffness in an h-dependent ratio at fixed tau)
    assert rates["Kp"][-1] < rates["Kp"][0] + 0.05, rates


def _ch_blocks(n=8, eps=0.02, tau=1e-3):
    mesh = Mesh(n)
    p = inputs.default_params()
    p.update(beta=[eps * eps] * 4, tau=tau)
    forms = model.Forms(mesh, p)
    st = inputs.initial_state(n)
    C = fem.convection_p1(mesh, st["v"])                   # v = 0: C = 0
    A, _, _, _ = model.ch_system(forms, st, p, 0, np.zeros(mesh.N1), C)
    A = A.toarray()
    N = mesh.N1
    return A[:N, :N], A[:N, N:], A[N:, :N], A[N:, N:], forms, p


def test_matching_schur_spectrum_in_half_one():
    """With C = 0 the matching approximation (tau gamma K + sqrt(tau gamma /
    beta) M) M^{-1} (same) of eqn::schurCH has eig(S~^{-1} S) in [1/2, 1]."""
    A11, A12, A21, A22, forms, p = _ch_blocks()
    S = -A22 + A21 @ np.linalg.solve(A11, A12)
    tau, g, b = p["tau"], p["gamma"][0], p["beta"][0]
    M, K = forms.M.toarray(), forms.K.toarray()
    X = tau * g * K + math.sqrt(tau * g / b) * M
    St = X @ np.linalg.solve(M, X)
    ev = sla.eigvals(S, St).real
    assert ev.min() >= 0.5 - 1e-10 and ev.max() <= 1 + 1e-10
    assert ev.min() < 0.55 and ev.max() > 0.95           # the bounds are attained closely


def test_block_diagonal_spectrum_ch():
    """Exact blocks P = diag(A11, S): eig(P^{-1} A) in [-1, (1-sqrt5)/2] U
    [1, (1+sqrt5)/2] (regularised saddle point, Murphy-Golub-Wathen type)."""
    A11, A12, A21, A22, _, _ = _ch_blocks()
    S = -A22 + A21 @ np.linalg.solve(A11, A12)
    A = np.block([[A11, A12], [A21, A22]])
    P = sla.block_diag(A11, S)
    ev = sla.eigvals(A, P)
    assert np.max(np.abs(ev.imag)) < 1e-8
    ev = ev.real
    neg, pos = ev[ev < 0], ev[ev > 0]
    r5 = math.sqrt(5.0)
    assert neg.min() >= -1 - 1e-9 and neg.max() <= (1 - r5) / 2 + 1e-9
    assert pos.min() >= 1 - 1e-9 and pos.max() <= (1 + r5) / 2 + 1e-9
    assert len(neg) == len(pos) == A11.shape[0]


def test_block_diagonal_spectrum_ns():
    """Exact A and exact Schur B A^{-1} B^T: eig(P^{-1} 𝒜) in {1, (1 +- sqrt5)/2}
    (Murphy, Golub, Wathen 2000, cited in Sec. 4), apart from the constant
    pressure mode."""
    n = 4
    mesh = Mesh(n)
    p = inputs.default_params()
    forms = model.Forms(mesh, p)
    st = inputs.initial_state(n)
    A, B, _, _, _ = model.ns_system(forms, st, p)
    A, B = A.toarray(), B.toarray()
    S = B @ np.linalg.solve(A, B.T)
    big = np.block([[A, B.T], [B, np.zeros((mesh.N1, mesh.N1))]])
    Sreg = S + np.ones_like(S) / mesh.N1
    P = sla.block_diag(A, Sreg)
    ev = sla.eigvals(big, P).real
    ev = ev[np.abs(ev) > 1e-8]
    r5 = math.sqrt(5.0)
    targets = np.array([1.0, (1 + r5) / 2, (1 - r5) / 2])
    dist = np.min(np.abs(ev[:, None] - targets[None]), axis=1)
    assert dist.max() < 1e-8
