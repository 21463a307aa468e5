"""Pins of oracle parts whose arithmetic the other oracle tests do not fix.

* The Korteweg tensor G of the momentum right-hand side (Sec. 3) and its load,
  2D and 3D, against hand-derived values for linear fields
  (tests/golden/korteweg_linear_fields.txt).
* The block preconditioners of Sec. 4 as compositions of block inverses:
  the CH one is diag(L^-1, X2^-1 M X1^-1) (eqn::schurCH with the matching
  factors), the Oseen one diag(A^-1, M_p^-1 A_p K_p^-1) (pressure
  convection-diffusion).  The multigrid blocks are made exact by the oracle's
  own inner-solve option (V-cycles iterated to 1e-13), so the applied
  operator can be compared with dense inverses built here from the formulas;
  M_p^-1 is the fixed degree-5 Chebyshev iteration, rebuilt here from its
  polynomial definition through a dense eigendecomposition.
* The order of the two matching factors, from the algebra of the CH blocks.
* Mesh-robust Oseen iteration counts of the enclosed-flow PCD.

A plausible mistake in any of these (the air term or beta_v dropped from G,
beta squared, A_p left out, X1 and X2 swapped under a concentration-dependent
mobility) fails a test here."""
import math
import os

import numpy as np
import pytest

from oracle import fem, model
from oracle import three_d as t3
from oracle.mesh import Mesh
from oracle.step import MASS_CHEB_BOUNDS, MASS_CHEB_DEGREE, Oracle
from paper_2501_11767_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "korteweg_linear_fields.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        out[k] = np.array([float(x) for x in v])
    return out


def _params(g):
    return dict(inputs.default_params(), beta=list(g["beta"][:4]), beta_v=float(g["beta"][4]))


# ---------------------------------------------------------------------------
def test_korteweg_tensor_2d_against_hand_values():
    g = _golden()
    n = int(g["load2_n"][0])
    mesh = Mesh(n)
    x, y = mesh.x1[:, 0], mesh.x1[:, 1]
    st = {"phi": np.stack([0.3 + 0.1 * x, 0.3 - 0.05 * y, 0.4 + 0.02 * x]), "Phi_v": 0.1 * y,
          "mu": np.zeros((4, mesh.N1))}
    Gt = model.korteweg_tensor(mesh, st, _params(g))
    want = g["G2"].reshape(2, 2)
    assert np.allclose(Gt, want[None], rtol=0, atol=1e-15)

    L = fem.korteweg(mesh, Gt).reshape(-1, 2)
    X, Y = mesh.x2[:, 0], mesh.x2[:, 1]
    h = 1.0 / n
    on = lambda a, b: np.isclose(a, b)  # noqa: E731
    inside = (X > 1e-12) & (X < 1 - 1e-12) & (Y > 1e-12) & (Y < 1 - 1e-12)
    vertex_x = on(np.round(X / h) * h, X)
    vertex_y = on(np.round(Y / h) * h, Y)
    top_in = on(Y, 1.0) & (X > 1e-12) & (X < 1 - 1e-12)
    right_in = on(X, 1.0) & (Y > 1e-12) & (Y < 1 - 1e-12)
    assert np.abs(L[inside]).max() < 1e-15
    assert np.allclose(L[top_in & vertex_x], g["load2_top_vertex"][None], rtol=1e-12, atol=0)
    assert np.allclose(L[top_in & ~vertex_x], g["load2_top_mid"][None], rtol=1e-12, atol=0)
    assert np.allclose(L[right_in & vertex_y], g["load2_right_vertex"][None], rtol=1e-12, atol=0)
    assert np.allclose(L[right_in & ~vertex_y], g["load2_right_mid"][None], rtol=1e-12, atol=0)
    # the bottom edge has the opposite normal: the negated top loads
    bot_in = on(Y, 0.0) & (X > 1e-12) & (X < 1 - 1e-12)
    assert np.allclose(L[bot_in & vertex_x], -g["load2_top_vertex"][None], rtol=1e-12, atol=0)


def test_korteweg_tensor_3d_against_hand_values():
    g = _golden()
    n = int(g["load3_n"][0])
    mesh = t3.Mesh3D(n)
    x, y, z = mesh.x1.T
    st = {"phi": np.stack([0.3 + 0.1 * x + 0.02 * z, 0.3 - 0.05 * y + 0.03 * z, 0.4 + 0.02 * x - 0.01 * z]),
          "Phi_v": 0.1 * y + 0.2 * z, "mu": np.zeros((4, mesh.N1)), "v": np.zeros(3 * mesh.N2)}
    Gt = t3.korteweg_tensor(mesh, st, _params(g))
    want = g["G3"].reshape(3, 3)
    assert np.allclose(Gt, want[None], rtol=0, atol=1e-15)

    L = t3.korteweg(mesh, Gt).reshape(-1, 3)
    lat, m = mesh.lat2, 2 * n
    inner = np.all((lat > 0) & (lat < m), axis=1)
    assert np.abs(L[inner]).max() < 1e-15
    top = (lat[:, 2] == m) & np.all((lat[:, :2] > 0) & (lat[:, :2] < m), axis=1)
    mid = top & ((lat[:, 0] % 2 == 1) | (lat[:, 1] % 2 == 1))
    assert mid.sum() > 0 and (top & ~mid).sum() > 0
    assert np.allclose(L[mid], g["load3_top_mid"][None], rtol=1e-12, atol=0)
    assert np.abs(L[top & ~mid]).max() < 1e-15


# ---------------------------------------------------------------------------
EXACT_INNER = {"inner_rtol": 1e-13, "inner_maxit": 400}


def _moving_state(n, seed=3):
    """Initial fields with a seeded smooth velocity (so that C(v), J(w) and
    A_p carry convection) and a concentration-dependent mobility worth
    having (phi_p far from constant)."""
    st = inputs.initial_state(n, seed=seed)
    mesh = Mesh(n)
    X, Y = mesh.x2[:, 0], mesh.x2[:, 1]
    bump = (X * (1 - X) * Y * (1 - Y))
    v = np.stack([3.0 * bump * (1 - 2 * Y), -3.0 * bump * (1 - 2 * X)], 1).ravel()
    x, y = mesh.x1[:, 0], mesh.x1[:, 1]
    st["v"] = v
    st["phi"][0] = 0.3 + 0.2 * np.sin(2 * np.pi * x) * np.cos(np.pi * y)
    return st


def test_ch_preconditioner_is_the_composition_of_block_inverses():
    """Applied operator = diag(L^-1, X2^-1 M X1^-1) with L = M + tau C,
    X1 = tau gamma K + a M, X2 = tau K_kappa + a M, a = sqrt(tau gamma / beta)
    (eqn::schurCH; concentration-dependent mobility, so X1 != X2 and their
    order matters)."""
    n = 8
    p = dict(inputs.default_params(), mobility_kind=1, **EXACT_INNER)
    o = Oracle(n, p)
    st = _moving_state(n)
    lstates = o.level_states(st)
    convs = [fem.convection_p1(f.mesh, s["v"]) for f, s in zip(o.forms, lstates)]
    N = o.mesh.N1
    F = o.forms[0]
    M, K, C = F.M.toarray(), F.K.toarray(), convs[0].toarray()
    r = np.random.default_rng(7).standard_normal(2 * N)
    for sp_ in (0, 2):
        tau, gam, beta = p["tau"], p["gamma"][sp_], p["beta"][sp_]
        a = math.sqrt(tau * gam / beta)
        Kk = fem.weighted_stiffness_p1(o.mesh, model.mobility_at(o.mesh, st["phi"][sp_], p, sp_)).toarray()
        L = M + tau * C
        X1 = tau * gam * K + a * M
        X2 = tau * Kk + a * M
        want = np.concatenate([np.linalg.solve(L, r[:N]), np.linalg.solve(X2, M @ np.linalg.solve(X1, r[N:]))])
        got = o.ch_preconditioner(sp_, lstates, convs)(r)
        assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want), sp_
        if sp_ == 0:
            # phi_p varies, so K_kappa is not a multiple of K and the order of
            # X1 and X2 matters (for the constant solvent field both factors
            # are functions of the same pencil (K, M) and commute)
            swapped = np.linalg.solve(X1, M @ np.linalg.solve(X2, r[N:]))
            assert np.linalg.norm(swapped - want[N:]) > 1e-3 * np.linalg.norm(want[N:])   # the test can tell


def test_matching_factor_order_follows_the_ch_blocks():
    """With C = 0 the negated Schur complement of eqn:CH_linear is
    (tau gamma / beta) M + (tau gamma K) M^-1 (tau K_kappa); the matching
    product X1 M^-1 X2 reproduces it up to the cross terms a (tau gamma K +
    tau K_kappa), and X2 M^-1 X1 does not (K and K_kappa do not commute)."""
    n = 8
    mesh = Mesh(n)
    p = dict(inputs.default_params(), mobility_kind=1)
    forms = model.Forms(mesh, p)
    st = _moving_state(n)
    st["v"] = np.zeros(2 * mesh.N2)
    C = fem.convection_p1(mesh, st["v"])
    A, _, _, Kk = model.ch_system(forms, st, p, 0, np.zeros(mesh.N1), C)
    A = A.toarray()
    N = mesh.N1
    A11, A12, A21, A22 = A[:N, :N], A[:N, N:], A[N:, :N], A[N:, N:]
    negS = -(A22 - A21 @ np.linalg.solve(A11, A12))
    tau, gam, beta = p["tau"], p["gamma"][0], p["beta"][0]
    a = math.sqrt(tau * gam / beta)
    M, K, Kk = forms.M.toarray(), forms.K.toarray(), Kk.toarray()
    X1 = tau * gam * K + a * M
    X2 = tau * Kk + a * M
    cross = a * (tau * gam * K + tau * Kk)
    good = X1 @ np.linalg.solve(M, X2) - cross
    bad = X2 @ np.linalg.solve(M, X1) - cross
    scale = np.abs(negS).max()
    assert np.abs(good - negS).max() <= 1e-12 * scale
    assert np.abs(bad - negS).max() > 1e-6 * scale


def _mass_chebyshev_dense(Mp, degree, lo, hi):
    """The degree-d Chebyshev iteration on D^-1 M from x0 = 0 as a matrix:
    the error x* - x is T_d((hi + lo - 2 l) / (hi - lo)) / T_d((hi + lo) /
    (hi - lo)) applied to x* = M^-1 b, l running over the spectrum of D^-1 M
    (taken from the symmetric D^-1/2 M D^-1/2)."""
    d = np.diag(Mp)
    Dh, Dmh = np.diag(np.sqrt(d)), np.diag(1.0 / np.sqrt(d))
    lam, U = np.linalg.eigh(Dmh @ Mp @ Dmh)
    c = np.zeros(degree + 1)
    c[degree] = 1.0
    fac = np.polynomial.chebyshev.chebval((hi + lo - 2 * lam) / (hi - lo), c) / \
        np.polynomial.chebyshev.chebval((hi + lo) / (hi - lo), c)
    E = Dmh @ U @ np.diag(fac) @ U.T @ Dh            # error map on x*
    return (np.eye(len(d)) - E) @ np.linalg.inv(Mp)


def test_ns_preconditioner_is_the_composition_of_block_inverses():
    """Applied operator = diag(A^-1, M_p^-1 A_p K_p^+) (Sec. 4, pressure
    convection-diffusion): A the Oseen velocity block, A_p = M_p / tau + eta
    K_p + J_p(w), K_p^+ the pseudo-inverse of the singular pressure Laplacian
    (enclosed flow), M_p^-1 the degree-5 Chebyshev iteration on [1/2, 2]."""
    n = 8
    p = dict(inputs.default_params(), **EXACT_INNER)
    o = Oracle(n, p)
    st = _moving_state(n)
    lstates = o.level_states(st)
    A, B, _, Ap, shift = model.ns_system(o.forms[0], st, p)
    F = o.forms[0]
    Mp, Kp = F.M.toarray(), F.K.toarray()
    Ap_formula = Mp / p["tau"] + p["eta"] * Kp + fem.convection_p1(o.mesh, st["v"], shift).toarray()
    assert np.abs(Ap.toarray() - Ap_formula).max() <= 1e-12 * np.abs(Ap_formula).max()
    nv = A.shape[0]
    r = np.random.default_rng(8).standard_normal(nv + o.mesh.N1)
    lo, hi = MASS_CHEB_BOUNDS
    Mcheb = _mass_chebyshev_dense(Mp, MASS_CHEB_DEGREE, lo, hi)
    want_v = np.linalg.solve(A.toarray(), r[:nv])
    want_p = Mcheb @ (Ap_formula @ (np.linalg.pinv(Kp, rcond=1e-10, hermitian=True) @ r[nv:]))
    got = o.ns_preconditioner(A, Ap, lstates)(r)
    assert np.linalg.norm(got[:nv] - want_v) <= 1e-9 * np.linalg.norm(want_v)
    assert np.linalg.norm(got[nv:] - want_p) <= 1e-9 * np.linalg.norm(want_p)
    without_ap = Mcheb @ (np.linalg.pinv(Kp, rcond=1e-10, hermitian=True) @ r[nv:])
    assert np.linalg.norm(without_ap - want_p) > 1e-2 * np.linalg.norm(want_p)   # the test can tell


@pytest.mark.parametrize("n", [16, 32, 64])
def test_enclosed_pcd_oseen_iterations_stay_flat(n):
    """The enclosed-flow PCD keeps the Oseen iteration count mesh-robust
    (Sec. 4 cites the PCD for its mesh independence): second step of the
    default parameter set, FGMRES(30) to 1e-8, at most 60 iterations on
    16^2, 32^2 and 64^2 (measured 37, 43, 48)."""
    p = inputs.default_params()
    o = Oracle(n, p)
    st = o.step(inputs.initial_state(n, seed=1))[0]
    info = o.step(st)[1]
    assert info["ns"]["converged"] and info["ns"]["iters"] <= 60, info["ns"]


# ---------------------------------------------------------------------------
def _forms(n, params):
    return model.Forms(Mesh(n), params)


def test_free_energy_local_part_of_constant_fields():
    """phi = (0.3, 0.3, 0.4), phi_a = 0: eqn:appPotential gives f_liq =
    3.5 * 0.09 * 0.09 + 0.3 * 0.16 = 0.07635 and f_gas = 3.5 * 0.09 * 2 + 2 *
    0.16 = 0.95; with p(Phi) = Phi^2 (3 - 2 Phi), p(1/2) = 1/2, so the
    density at Phi = 1/2 is 0.513175.  Area 2 (a 2 x 1 box)."""
    p = inputs.default_params()
    mesh = Mesh(4, 2.0, 1.0)
    forms = model.Forms(mesh, p)
    for Phi, dens in ((0.0, 0.07635), (1.0, 0.95), (0.5, 0.513175)):
        st = {"phi": np.stack([np.full(mesh.N1, 0.3), np.full(mesh.N1, 0.3), np.full(mesh.N1, 0.4)]),
              "Phi_v": np.full(mesh.N1, Phi), "v": np.zeros(2 * mesh.N2)}
        e = model.free_energy(forms, st, p)
        assert e["local"] == pytest.approx(2.0 * dens, rel=1e-13), Phi
        assert abs(e["gradient"]) < 1e-15 and e["kinetic"] == 0.0


def test_free_energy_gradient_part_is_half_the_trace_of_the_korteweg_tensor():
    """For linear fields the gradient energy density sum beta_i |grad
    phi_i|^2 / 2 + beta_v |grad Phi_v|^2 / 2 is constant and equals tr(G) / 2
    with G the Korteweg tensor of the golden file: (0.01312 + 0.00725) / 2 =
    0.010185 on the unit square."""
    g = _golden()
    p = _params(g)
    forms = _forms(4, p)
    mesh = forms.mesh
    x, y = mesh.x1[:, 0], mesh.x1[:, 1]
    st = {"phi": np.stack([0.3 + 0.1 * x, 0.3 - 0.05 * y, 0.4 + 0.02 * x]), "Phi_v": 0.1 * y,
          "v": np.zeros(2 * mesh.N2)}
    e = model.free_energy(forms, st, p)
    assert e["gradient"] == pytest.approx(0.010185, rel=1e-12)
    assert e["gradient"] == pytest.approx(0.5 * (g["G2"][0] + g["G2"][3]), rel=1e-12)


def test_free_energy_local_part_rule_is_exact_for_linear_fields():
    """With linear fields the density is a polynomial of degree 7 (degree 4 in
    phi times the cubic p(Phi)); the degree-7 rule must equal a degree-15 one."""
    from oracle.quadrature import triangle_rule
    p = inputs.default_params()
    forms = _forms(4, p)
    mesh = forms.mesh
    x, y = mesh.x1[:, 0], mesh.x1[:, 1]
    st = {"phi": np.stack([0.2 + 0.3 * x, 0.35 - 0.2 * y + 0.1 * x, 0.3 + 0.1 * y]), "Phi_v": 0.2 + 0.6 * x * 0 + 0.5 * y,
          "v": np.zeros(2 * mesh.N2)}
    e = model.free_energy(forms, st, p)
    lam, w = triangle_rule(15)
    _, area, _ = mesh.element_geometry()
    pp, pn, ps = (fem.p1_field_at(mesh, st["phi"][i], lam) for i in range(3))
    Ph = fem.p1_field_at(mesh, st["Phi_v"], lam)
    ref = float(np.sum(area[:, None] * w[None] * model.potential(pp, pn, ps, 1 - pp - pn - ps, Ph)))
    assert e["local"] == pytest.approx(ref, rel=1e-13)


def test_free_energy_kinetic_part_of_quadratic_free_velocities():
    """v = (1, 0): 1/2 int |v|^2 = 1/2; v = (x, y): 1/2 (1/3 + 1/3) = 1/3 on the
    unit square (both exact in the P2 velocity space)."""
    p = inputs.default_params()
    forms = _forms(4, p)
    mesh = forms.mesh
    X, Y = mesh.x2[:, 0], mesh.x2[:, 1]
    base = {"phi": np.zeros((3, mesh.N1)), "Phi_v": np.zeros(mesh.N1)}
    e1 = model.free_energy(forms, dict(base, v=np.stack([np.ones_like(X), np.zeros_like(X)], 1).ravel()), p)
    e2 = model.free_energy(forms, dict(base, v=np.stack([X, Y], 1).ravel()), p)
    assert e1["kinetic"] == pytest.approx(0.5, rel=1e-13)
    assert e2["kinetic"] == pytest.approx(1.0 / 3.0, rel=1e-13)


# ---------------------------------------------------------------------------
def test_iterative_coarsest_level_on_the_papers_2d_mesh():
    """n = 50 (a mesh of the paper's 2D runs) coarsens to 25 x 25: the
    velocity and the mass-dominated P1 blocks solve their coarsest level by 16
    Chebyshev-Jacobi steps, the pressure Laplacian keeps its dense inverse.
    The polynomial coarse solve of the velocity block is within 5 % of the
    exact coarse solve (the block is mass-dominated there), and a whole step
    stays within the Krylov tolerance's reach of the exact (sparse LU) step."""
    import scipy.sparse.linalg as spla
    from oracle.mg import COARSE_DEGREE, MG, VEL_LO_RATIO, VEL_SMOOTH_DEGREE
    n = 50
    p = inputs.default_params()
    o = Oracle(n, p)
    st = inputs.initial_state(n, seed=1)
    lstates = o.level_states(st)
    A, _, _, Ap, _ = model.ns_system(o.forms[0], st, p)
    o.ns_preconditioner(A, Ap, lstates)
    assert not o._Kp.coarse_iter and o._Kp.lu is not None
    mats = [A]
    for lev in range(1, len(o.sizes)):
        f, s_ = o.forms[lev], lstates[lev]
        vf = f.velocity_forms()
        J2 = fem.convection_p2(f.mesh, s_["v"], model.ns_shift(f.mesh, s_, p))
        import scipy.sparse as sp
        Al = vf["Mv"] / p["tau"] + sp.kron(J2, sp.eye(2), format="csr") + vf["Ksym"]
        mats.append(fem.velocity_dirichlet(Al.tocsr(), vf["bnd"]))
    mg = MG(mats, o.Pv(), degree=VEL_SMOOTH_DEGREE, ratio=VEL_LO_RATIO)
    assert mg.coarse_iter and mats[-1].shape[0] == 2 * 51 ** 2 and COARSE_DEGREE == 16
    b = np.random.default_rng(3).standard_normal(mats[-1].shape[0])
    exact = spla.spsolve(mats[-1].tocsc(), b)
    got = mg.vcycle(b, level=len(mats) - 1)
    assert np.linalg.norm(got - exact) <= 0.05 * np.linalg.norm(exact)
    oe = Oracle(n, p, exact=True)
    a, info = o.step(st)
    e, _ = oe.step(st)
    assert info["ns"]["converged"] and info["ns"]["iters"] <= 60
    for key, tol in (("phi", 1e-8), ("Phi_v", 1e-8), ("v", 1e-6), ("p", 1e-5), ("mu", 1e-5)):
        assert np.linalg.norm(a[key] - e[key]) <= tol * np.linalg.norm(e[key]), key
