"""Pins of the oracle's discretisation against closed forms, identities and
manufactured solutions (CPU only)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, model
from oracle.mesh import Mesh
from oracle.mg import prolongation_p1, prolongation_p2, inject_p1, inject_velocity
from oracle.quadrature import triangle_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
@pytest.mark.parametrize("degree", [1, 2, 3, 5, 7, 9])
def test_quadrature_exact_on_monomials(degree):
    """int_T xi^a eta^b = a! b! / (a+b+2)! on the reference triangle."""
    lam, w = triangle_rule(degree)
    xi, eta = lam[:, 1], lam[:, 2]
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = 0.5 * np.sum(w * xi**a * eta**b)
            assert abs(got - exact) <= 1e-15 + 1e-13 * exact


def test_quadrature_not_exact_beyond_degree():
    """Sanity: a degree-3 rule misses a degree-8 monomial (the pin above
    would notice a rule of too low degree)."""
    lam, w = triangle_rule(3)
    exact = math.factorial(8) * 1 / math.factorial(10)
    assert abs(0.5 * np.sum(w * lam[:, 1] ** 8) - exact) > 1e-6


@pytest.mark.parametrize("n,nnz", [(int(a), int(b)) for a, b in _golden_rows("p1_element.txt")])
def test_p1_pattern_nnz(n, nnz):
    M = fem.mass_p1(Mesh(n))
    assert M.nnz == nnz


def test_p1_mass_and_stiffness_closed_forms():
    n = 8
    mesh = Mesh(n)
    h = 1.0 / n
    M, K = fem.mass_p1(mesh).toarray(), fem.stiffness_p1(mesh).toarray()
    idx = lambda i, j: j * (n + 1) + i  # noqa: E731
    c = idx(4, 4)
    assert M[c, c] == pytest.approx(h * h / 2, rel=1e-13)
    for di, dj in [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)]:
        assert M[c, idx(4 + di, 4 + dj)] == pytest.approx(h * h / 12, rel=1e-13)
        # the 5-point stencil: axis neighbours -1, diagonal neighbours 0
        expect = 0.0 if di == dj else -1.0
        assert K[c, idx(4 + di, 4 + dj)] == pytest.approx(expect, abs=1e-13)
    assert K[c, c] == pytest.approx(4.0, rel=1e-13)
    assert np.count_nonzero(np.abs(K[c]) > 1e-14) == 5
    assert np.sum(M) == pytest.approx(1.0, rel=1e-13)          # area
    assert np.max(np.abs(K.sum(axis=1))) < 1e-12              # K 1 = 0
    assert np.min(np.linalg.eigvalsh(M)) > 0


def test_p1_element_mass_closed_form():
    """A single element: M_T = |T|/12 [[2,1,1],[1,2,1],[1,1,2]]."""
    mesh = Mesh(1, 2.0, 3.0)
    M = fem.mass_p1(mesh).toarray()
    area = 3.0
    # nodes 0 and 3 are shared by both triangles, 1 and 2 belong to one each
    assert M[1, 1] == pytest.approx(area / 12 * 2)
    assert M[0, 0] == pytest.approx(2 * area / 12 * 2)
    assert M[0, 3] == pytest.approx(2 * area / 12)
    assert M[1, 2] == 0.0


def test_p2_identities():
    mesh = Mesh(6, 1.0, 1.0)
    M2 = fem.mass_p2(mesh)
    x, y = mesh.x2[:, 0], mesh.x2[:, 1]
    one = np.ones(mesh.N2)
    assert one @ (M2 @ one) == pytest.approx(1.0, rel=1e-13)
    assert one @ (M2 @ (x * x * y)) == pytest.approx(1.0 / 6.0, rel=1e-12)  # int x^2 y
    # rigid motions are in the kernel of K_sym (before boundary conditions)
    Ks = fem.ksym(mesh, 1.7)
    for v in [np.stack([one, 0 * one], 1), np.stack([0 * one, one], 1), np.stack([-y, x], 1)]:
        assert np.max(np.abs(Ks @ v.ravel())) < 1e-11
    # a non-rigid field is not
    assert np.max(np.abs(Ks @ np.stack([x, 0 * one], 1).ravel())) > 1e-3
    # B annihilates exactly divergence-free P2 fields: v = (y^2, x^2), (x, -y)
    B = fem.divergence(mesh)
    for v in [np.stack([y * y, x * x], 1), np.stack([x, -y], 1)]:
        assert np.max(np.abs(B @ v.ravel())) < 1e-13
    # and B (x, 0) = -int psi_q
    M1 = fem.mass_p1(mesh)
    assert np.allclose(B @ np.stack([x, 0 * one], 1).ravel(), -(M1 @ np.ones(mesh.N1)), atol=1e-14)
    # convection of constants vanishes
    v = np.stack([1 + y * y, x * y], 1).ravel()
    assert np.max(np.abs(fem.convection_p1(mesh, v) @ np.ones(mesh.N1))) < 1e-14
    assert np.max(np.abs(fem.convection_p2(mesh, v) @ one)) < 1e-13


def test_symmetric_gradient_form_on_quadratics():
    """At interior P2 nodes K_sym u = -eta int div(2 sym grad u) zeta_a: (2, 0)
    for u = (y^2, 0) and (4, 0) for u = (x^2, 0); the Laplacian form would give
    2 for both, so this fixes the symmetric gradient and its factor 2 (the
    Stokes MMS uses a divergence-free field, for which the two forms agree)."""
    mesh = Mesh(6)
    eta = 1.3
    K = fem.ksym(mesh, eta)
    x, y = mesh.x2[:, 0], mesh.x2[:, 1]
    w = fem.mass_p2(mesh) @ np.ones(mesh.N2)
    inner = np.all((mesh.lat2 > 0) & (mesh.lat2 < 2 * mesh.n), axis=1)
    for ux, dx in ((y * y, 2.0), (x * x, 4.0)):
        r = (K @ np.stack([ux, 0 * ux], 1).ravel()).reshape(-1, 2)
        assert np.abs(r[inner, 0] + eta * dx * w[inner]).max() < 1e-11 * eta * dx * np.abs(w).max()
        assert np.abs(r[inner, 1]).max() < 1e-14


def test_convection_integration_by_parts():
    """C + C^T = int_{dOmega} (v.n) psi_a psi_b - int div(v) psi_a psi_b.
    For v = (y (1 - y), 0) (divergence-free, v.n = 0 on top and bottom) the
    rows of nodes off the side walls vanish and 1^T (C + C^T) 1 = 0."""
    mesh = Mesh(8)
    x, y = mesh.x2[:, 0], mesh.x2[:, 1]
    v = np.stack([y * (1 - y), 0 * x], 1).ravel()
    C = fem.convection_p1(mesh, v)
    S = (C + C.T).toarray()
    xs = mesh.x1[:, 0]
    off_side = (xs > 0) & (xs < 1)
    assert np.max(np.abs(S[off_side])) < 1e-15
    assert abs(S.sum()) < 1e-15
    assert np.max(np.abs(S[~off_side])) > 1e-4


def test_potential_partials_by_finite_differences():
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.05, 0.6, size=(20, 5))
    h = 1e-6
    for pp, pn, ps, pa, Ph in pts:
        d = model.potential_partials(pp, pn, ps, pa, Ph)
        args = [pp, pn, ps, pa, Ph]
        for k in range(5):
            up = list(args); dn = list(args)
            up[k] += h; dn[k] -= h
            fd = (model.potential(*up) - model.potential(*dn)) / (2 * h)
            assert d[k] == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_potential_loads_constant_fields():
    """Constant fields: int c psi_a = c (M 1)_a."""
    mesh = Mesh(4)
    phi = np.stack([np.full(mesh.N1, 0.3), np.full(mesh.N1, 0.25), np.full(mesh.N1, 0.4)])
    Phi = np.full(mesh.N1, 0.2)
    loads = model.potential_loads(mesh, phi, Phi)
    d = model.potential_partials(0.3, 0.25, 0.4, 0.05, 0.2)
    m1 = fem.mass_p1(mesh) @ np.ones(mesh.N1)
    for k in range(5):
        assert np.allclose(loads[k], d[k] * m1, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("model_kind", [0, 1])
def test_potential_loads_rule_degree_suffices(model_kind):
    """For linear fields the load integrands are polynomials of degree <= 7
    (eqn:appPotential; the solvent-air density with its degree-4 Taylor
    polynomials of x ln x): the degree-7 rule equals a degree-13 one."""
    from paper_2501_11767_gb300 import inputs
    mesh = Mesh(4)
    x, y = mesh.x1[:, 0], mesh.x1[:, 1]
    phi = np.stack([0.3 + 0.05 * x, 0.25 - 0.04 * y, 0.4 + 0.1 * (x - y)])
    Phi = 0.2 + 0.3 * y
    params = inputs.solvent_air_params() if model_kind else None
    loads = model.potential_loads(mesh, phi, Phi, params)
    for k in range(5):
        def integrand(lam, k=k):
            pp, pn, ps = (fem.p1_field_at(mesh, phi[i], lam) for i in range(3))
            pa, Ph = 1.0 - pp - pn - ps, fem.p1_field_at(mesh, Phi, lam)
            if model_kind:
                return model.fh_partials(ps, pa, Ph, params)[k - 2] if k >= 2 else 0.0 * pp
            return model.potential_partials(pp, pn, ps, pa, Ph)[k]
        ref = fem.load_p1(mesh, integrand, 13)
        assert np.allclose(loads[k], ref, rtol=1e-12, atol=1e-14 * max(np.abs(ref).max(), 1e-300)), k


def test_top_load_and_reference_node():
    mesh = Mesh(8, 2.0, 1.0)
    t = fem.top_load_p1(mesh)
    assert t.sum() == pytest.approx(2.0)
    assert np.all(t[~mesh.p1_top()] == 0)
    r = mesh.top_reference_node()
    assert np.allclose(mesh.x1[r], [1.0, 1.0])


def test_korteweg_vanishes_inside_for_linear_fields():
    mesh = Mesh(6)
    x, y = mesh.x1[:, 0], mesh.x1[:, 1]
    st = {"phi": np.stack([0.3 + 0.1 * x, 0.3 - 0.05 * y, 0.4 + 0.02 * x]), "Phi_v": 0.1 * y,
          "mu": np.zeros((4, mesh.N1))}
    params = {"beta": [0.1, 0.2, 0.3, 0.4], "beta_v": 0.5}
    G = fem.korteweg(mesh, model.korteweg_tensor(mesh, st, params)).reshape(-1, 2)
    inner = ~mesh.p2_boundary()
    assert np.max(np.abs(G[inner])) < 1e-14
    assert np.max(np.abs(G[~inner])) > 1e-4
    # constant G tensor: G_a = Gt . int grad zeta_a = boundary integral
    Gt = model.korteweg_tensor(mesh, st, params)[0]
    assert np.allclose(model.korteweg_tensor(mesh, st, params), Gt[None], atol=1e-15)


# --------------------------------------------------------------------------
def _rate(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_mms_p1_convection_diffusion_rate():
    """(M + K + C(v)) u = f with u = cos(pi x) cos(pi y) (natural Neumann
    data), v a P2-exact field: L2 error O(h^2)."""
    pi = math.pi
    u = lambda x, y: np.cos(pi * x) * np.cos(pi * y)  # noqa: E731
    ux = lambda x, y: -pi * np.sin(pi * x) * np.cos(pi * y)  # noqa: E731
    uy = lambda x, y: -pi * np.cos(pi * x) * np.sin(pi * y)  # noqa: E731
    vx = lambda x, y: y * (1 - y)  # noqa: E731
    vy = lambda x, y: x * (1 - x)  # noqa: E731
    f = lambda x, y: (1 + 2 * pi * pi) * u(x, y) + vx(x, y) * ux(x, y) + vy(x, y) * uy(x, y)  # noqa: E731
    errs = []
    for n in (8, 16, 32):
        mesh = Mesh(n)
        x2, y2 = mesh.x2[:, 0], mesh.x2[:, 1]
        v = np.stack([vx(x2, y2), vy(x2, y2)], 1).ravel()
        A = fem.mass_p1(mesh) + fem.stiffness_p1(mesh) + fem.convection_p1(mesh, v)
        X = lambda lam: fem.quad_points(mesh, lam)  # noqa: E731
        b = fem.load_p1(mesh, lambda lam: f(X(lam)[..., 0], X(lam)[..., 1]), 8)
        uh = spla.spsolve(A.tocsc(), b)
        errs.append(fem.l2_error_p1(mesh, uh, u))
    r = _rate(errs)
    assert min(r) > 1.9, (errs, r)


def test_mms_weighted_stiffness_rate():
    """-div(kappa grad u) + u = f with kappa = x(1-x) + m0, the mobility law
    phi (1 - phi) + m0 at phi = x."""
    pi, m0 = math.pi, 1e-3
    u = lambda x, y: np.cos(pi * x) * np.cos(pi * y)  # noqa: E731
    kap = lambda x: x * (1 - x) + m0  # noqa: E731
    # -div(kappa grad u) = -kappa' u_x - kappa lap u
    f = lambda x, y: u(x, y) - (1 - 2 * x) * (-pi * np.sin(pi * x) * np.cos(pi * y)) + kap(x) * 2 * pi * pi * u(x, y)  # noqa: E731,E501
    errs = []
    params = {"gamma": [1.0, 1.0, 1.0], "mobility_kind": 1, "mobility_m0": m0}
    for n in (8, 16, 32):
        mesh = Mesh(n)
        phi = mesh.x1[:, 0].copy()
        Kk = fem.weighted_stiffness_p1(mesh, model.mobility_at(mesh, phi, params, 0))
        A = fem.mass_p1(mesh) + Kk
        X = lambda lam: fem.quad_points(mesh, lam)  # noqa: E731
        b = fem.load_p1(mesh, lambda lam: f(X(lam)[..., 0], X(lam)[..., 1]), 8)
        uh = spla.spsolve(A.tocsc(), b)
        errs.append(fem.l2_error_p1(mesh, uh, u))
    assert min(_rate(errs)) > 1.9, errs


def _stokes_exact():
    import sympy as sy
    X, Y = sy.symbols("x y")
    psi = X**2 * (1 - X) ** 2 * Y**2 * (1 - Y) ** 2
    vx, vy = sy.diff(psi, Y), -sy.diff(psi, X)
    p = X**2 - sy.Rational(1, 3)
    lap = lambda g: sy.diff(g, X, 2) + sy.diff(g, Y, 2)  # noqa: E731
    return X, Y, vx, vy, p, lap, sy


def test_mms_taylor_hood_stokes_rates():
    """K_sym v + B^T p = f, B v = 0 with an exact divergence-free wall-bounded
    velocity: velocity L2 O(h^3), pressure L2 O(h^2) (Taylor-Hood)."""
    X, Y, vx, vy, p, lap, sy = _stokes_exact()
    eta = 1.0
    fx = -eta * lap(vx) + sy.diff(p, X)
    fy = -eta * lap(vy) + sy.diff(p, Y)
    F = sy.lambdify((X, Y), (fx, fy), "numpy")
    V = sy.lambdify((X, Y), (vx, vy), "numpy")
    P = sy.lambdify((X, Y), p, "numpy")
    ev, ep = [], []
    for n in (4, 8, 16):
        mesh = Mesh(n)
        bnd = mesh.p2_boundary()
        A = fem.velocity_dirichlet(fem.ksym(mesh, eta), bnd)
        B = fem.zero_velocity_columns(fem.divergence(mesh), bnd)
        f = fem.load_velocity(mesh, lambda x, y: tuple(np.broadcast_to(c, x.shape) for c in F(x, y)), 8)
        f[np.repeat(bnd, 2)] = 0
        m = fem.mass_p1(mesh) @ np.ones(mesh.N1)
        K = sp.bmat([[A, B.T, None], [B, None, sp.csr_matrix(m[:, None])],
                     [None, sp.csr_matrix(m[None, :]), None]], format="csc")
        sol = spla.spsolve(K, np.concatenate([f, np.zeros(mesh.N1 + 1)]))
        nv = 2 * mesh.N2
        ev.append(fem.l2_error_velocity(mesh, sol[:nv], lambda x, y: V(x, y)))
        ep.append(fem.l2_error_p1(mesh, sol[nv:nv + mesh.N1], lambda x, y: P(x, y)))
    assert min(_rate(ev)) > 2.8, ev
    assert min(_rate(ep)) > 1.8, ep


def test_mms_vector_convection_diffusion_rate():
    """(M_v + K_sym + J(w)) v = f for the same exact velocity: O(h^3)."""
    X, Y, vx, vy, p, lap, sy = _stokes_exact()
    wx, wy = 1 + Y**2, X
    fx = vx - lap(vx) + wx * sy.diff(vx, X) + wy * sy.diff(vx, Y)
    fy = vy - lap(vy) + wx * sy.diff(vy, X) + wy * sy.diff(vy, Y)
    F = sy.lambdify((X, Y), (fx, fy), "numpy")
    V = sy.lambdify((X, Y), (vx, vy), "numpy")
    errs = []
    for n in (4, 8, 16):
        mesh = Mesh(n)
        bnd = mesh.p2_boundary()
        x2, y2 = mesh.x2[:, 0], mesh.x2[:, 1]
        w = np.stack([1 + y2**2, x2], 1).ravel()
        A = (sp.kron(fem.mass_p2(mesh) + fem.convection_p2(mesh, w), sp.eye(2)) + fem.ksym(mesh, 1.0)).tocsr()
        A = fem.velocity_dirichlet(A, bnd)
        f = fem.load_velocity(mesh, lambda x, y: F(x, y), 9)
        f[np.repeat(bnd, 2)] = 0
        vh = spla.spsolve(A.tocsc(), f)
        errs.append(fem.l2_error_velocity(mesh, vh, lambda x, y: V(x, y)))
    assert min(_rate(errs)) > 2.8, errs


def test_convection_shift_matches_constant_field():
    """Shift g per element equals convecting with the constant field -g."""
    mesh = Mesh(5)
    x2 = mesh.x2[:, 0]
    v = np.stack([x2 * 0, x2 * 0], 1).ravel()
    g = np.tile([[0.3, -0.7]], (mesh.E, 1))
    vc = np.tile([-0.3, 0.7], mesh.N2)
    assert np.allclose(fem.convection_p2(mesh, v, g).toarray(), fem.convection_p2(mesh, vc).toarray(), atol=1e-15)
    assert np.allclose(fem.convection_p1(mesh, v, g).toarray(), fem.convection_p1(mesh, vc).toarray(), atol=1e-15)


# --------------------------------------------------------------------------
def test_prolongation_reproduces_polynomials():
    coarse, fine = Mesh(4), Mesh(8)
    P1 = prolongation_p1(coarse)
    xc, yc = coarse.x1[:, 0], coarse.x1[:, 1]
    xf, yf = fine.x1[:, 0], fine.x1[:, 1]
    assert np.allclose(P1 @ (2 * xc - 3 * yc + 1), 2 * xf - 3 * yf + 1, atol=1e-14)
    assert np.allclose(P1.sum(axis=1), 1.0)
    P2 = prolongation_p2(coarse)
    xc, yc = coarse.x2[:, 0], coarse.x2[:, 1]
    xf, yf = fine.x2[:, 0], fine.x2[:, 1]
    q = lambda x, y: 1 + x - 2 * y + 3 * x * y - x * x + 0.5 * y * y  # noqa: E731
    assert np.allclose(P2 @ q(xc, yc), q(xf, yf), atol=1e-14)
    # injection picks coarse nodes
    assert np.allclose(inject_p1(fine.x1[:, 0], 8), coarse.x1[:, 0])
    v = np.stack([xf, yf], 1).ravel()
    assert np.allclose(inject_velocity(v, 8), np.stack([xc, yc], 1).ravel())


@pytest.mark.parametrize("n", [2, 4, 6, 16])
def test_p1_operators_are_seven_point_stencils(n):
    """Every P1 operator of the step (mass, stiffness, convection with a P2
    velocity, weighted stiffness) couples node i = j (n+1) + k only to
    i + {-(n+2), -(n+1), -1, 0, 1, n+1, n+2} (the lower-left -> upper-right
    diagonals of the mesh), and interior rows couple to all seven: the
    precondition of the library's stencil layout for the P1 sweeps."""
    m = Mesh(n)
    nx = n + 1
    off = {-nx - 1, -nx, -1, 0, 1, nx, nx + 1}
    rng = np.random.default_rng(n)
    v = rng.standard_normal(2 * m.N2)
    kappa = lambda lam: 1.0 + np.outer(np.arange(m.E) % 3, lam[:, 0])   # (E, Q), positive
    A = (fem.mass_p1(m) + fem.stiffness_p1(m) + fem.convection_p1(m, v)
         + fem.weighted_stiffness_p1(m, kappa)).tocsr()
    A.sort_indices()
    for i in range(m.N1):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        assert set((cols - i).tolist()) <= off, i
        k, j = i % nx, i // nx
        if 0 < k < n and 0 < j < n:
            assert len(cols) == 7, i


def test_mms_cahn_hilliard_and_allen_cahn_systems():
    """The linear systems of one step (eqn:CH_linear, the AC system of Sec. 4)
    against their PDEs with manufactured data, no flow: CH
    (phi - phi_k) / tau = gamma lap mu, mu = -beta lap phi + f, with
    phi = cos(pi x) cos(pi y) and f = cos(2 pi x) / 2 (Neumann data zero, so
    phi_k follows by differentiation); AC (Phi - Phi_k) / tau = delta lap Phi
    - gamma_v f_v with Phi = cos(pi x) cos(2 pi y).  The P1 solutions converge
    at O(h^2) in L2: a wrong sign, a misplaced tau, gamma or beta, or a
    transposed block breaks the rate."""
    pi = math.pi
    tau, g, beta, delta, gv = 0.01, 1.3, 0.05, 0.7, 0.9
    phi = lambda x, y: np.cos(pi * x) * np.cos(pi * y)                                   # noqa: E731
    fch = lambda x, y: 0.5 * np.cos(2 * pi * x)                                          # noqa: E731
    mu = lambda x, y: 2 * pi * pi * beta * phi(x, y) + fch(x, y)                         # noqa: E731
    lap_mu = lambda x, y: -4 * pi ** 4 * beta * phi(x, y) - 2 * pi * pi * np.cos(2 * pi * x)  # noqa: E731
    phik = lambda x, y: phi(x, y) - tau * g * lap_mu(x, y)                               # noqa: E731
    Phi = lambda x, y: np.cos(pi * x) * np.cos(2 * pi * y)                               # noqa: E731
    fv = lambda x, y: np.cos(pi * y) ** 2                                                # noqa: E731
    Phik = lambda x, y: Phi(x, y) + tau * delta * 5 * pi * pi * Phi(x, y) + tau * gv * fv(x, y)  # noqa: E731
    params = dict(tau=tau, gamma=[g] * 3, beta=[beta] * 4, mobility_kind=0, delta_v=delta, gamma_v=gv,
                  ac_top_flux=0)
    e_phi, e_mu, e_Phi = [], [], []
    for n in (8, 16, 32):
        mesh = Mesh(n)
        forms = model.Forms(mesh, params)
        x, y = mesh.x1[:, 0], mesh.x1[:, 1]
        X = lambda lam: fem.quad_points(mesh, lam)                                       # noqa: E731
        load = lambda fn: fem.load_p1(mesh, lambda lam: fn(X(lam)[..., 0], X(lam)[..., 1]), 8)  # noqa: E731
        st = {"phi": np.stack([phik(x, y)] * 3), "Phi_v": Phik(x, y)}
        C = sp.csr_matrix((mesh.N1, mesh.N1))
        A, rhs, _, _ = model.ch_system(forms, st, params, 0, load(fch), C)
        sol = spla.spsolve(A.tocsc(), rhs)
        e_phi.append(fem.l2_error_p1(mesh, sol[:mesh.N1], phi))
        e_mu.append(fem.l2_error_p1(mesh, sol[mesh.N1:], mu))
        Aac, rac = model.ac_system(forms, st, params, load(fv), C, 0.0)
        e_Phi.append(fem.l2_error_p1(mesh, spla.spsolve(Aac.tocsc(), rac), Phi))
    for errs in (e_phi, e_mu, e_Phi):
        assert min(_rate(errs)) > 1.8, (errs, _rate(errs))
