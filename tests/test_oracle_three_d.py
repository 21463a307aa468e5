"""Pins of the 3D oracle (Kuhn tetrahedra, oracle/three_d.py): quadrature
exactness, mesh geometry, closed forms of the P1 matrices (the Kuhn P1
stiffness is the 7-point finite-difference Laplacian), Taylor-Hood
identities, nested transfers, manufactured-solution rates, closed forms of
the potential and Korteweg loads, the weighted stiffness of the
concentration-dependent mobility, the open top's masks, and properties of
whole steps: the Krylov step against sparse LU (also with the variable
mobility, inner solves and the open top), mass conservation, discretely
divergence-free velocity (CPU only)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import three_d as t3
from oracle.mg import MG
from oracle.quadrature import tetra_rule
from paper_2501_11767_gb300 import inputs


@pytest.mark.parametrize("degree", range(0, 9))
def test_tetra_rule_exact_on_monomials(degree):
    lam, w = tetra_rule(degree)
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                val = np.sum(w * lam[:, 1] ** a * lam[:, 2] ** b * lam[:, 3] ** c) / 6.0
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                assert val == pytest.approx(exact, rel=1e-12, abs=1e-16)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_mesh_geometry(n):
    m = t3.Mesh3D(n, 1.0, 2.0, 0.5)
    _, vol, g = m.element_geometry()
    assert np.all(vol > 0)
    assert vol.sum() == pytest.approx(1.0, rel=1e-13)
    assert np.allclose(g.sum(axis=1), 0.0, atol=1e-12)
    # every P1 and P2 node is used; edge midpoints lie halfway between the vertices
    assert np.unique(m.tet).size == m.N1
    assert np.unique(m.tet2).size == m.N2
    for q, (a, b) in enumerate(t3.EDGES):
        assert np.allclose(m.x2[m.tet2[:, 4 + q]], 0.5 * (m.x1[m.tet[:, a]] + m.x1[m.tet[:, b]]))


def test_p1_closed_forms():
    n = 4
    m = t3.Mesh3D(n)
    h = 1.0 / n
    M, K = t3.mass_p1(m), t3.stiffness_p1(m)
    assert M.sum() == pytest.approx(1.0, rel=1e-13)
    assert np.allclose(K @ np.ones(m.N1), 0.0, atol=1e-13)
    # the Kuhn P1 stiffness is the 7-point Laplacian times h: 6h on the
    # diagonal of an interior node, -h to its six axis neighbours, nothing else
    i = int(m.id1(np.array([2, 2, 2])))
    row = K.getrow(i).toarray().ravel()
    assert row[i] == pytest.approx(6 * h, rel=1e-12)
    for d in range(3):
        for s in (-1, 1):
            nb = np.array([2, 2, 2])
            nb[d] += s
            assert row[int(m.id1(nb))] == pytest.approx(-h, rel=1e-12)
    row[i] = 0.0
    assert np.sum(np.abs(row)) == pytest.approx(6 * h, rel=1e-12)
    # element mass |T| / 20 (1 + delta_ab): the lumped masses of an interior node
    assert M.getrow(i).sum() == pytest.approx(h ** 3, rel=1e-12)


def test_taylor_hood_identities():
    n = 2
    m = t3.Mesh3D(n)
    M2 = t3.mass_p2(m)
    assert M2.sum() == pytest.approx(1.0, rel=1e-12)
    Ks = t3.ksym(m, 1.0)
    x = m.x2
    rng = np.random.default_rng(0)
    for _ in range(3):     # rigid motions a + w x x are in the kernel of K_sym
        a, w = rng.standard_normal(3), rng.standard_normal(3)
        u = a[None, :] + np.cross(w[None, :], x)
        assert np.abs(Ks @ u.ravel()).max() < 1e-12
    B = t3.divergence(m)
    # B (grad of a quadratic) = - M-weighted Laplacian test: B u = - int q div u
    u = np.stack([x[:, 0] ** 2, x[:, 1] * x[:, 2], np.zeros(m.N2)], axis=1).ravel()   # div u = 2x + z
    ref = -t3.load_p1(m, lambda lam: (2.0 * t3.quad_points(m, lam)[..., 0] + t3.quad_points(m, lam)[..., 2]), 2)
    assert np.allclose(B @ u, ref, atol=1e-13)
    # convection of a constant field by a solenoidal P2 velocity vanishes; C 1 = 0
    v = np.stack([x[:, 1], x[:, 2], x[:, 0]], axis=1).ravel()
    assert np.abs(t3.convection_p1(m, v) @ np.ones(m.N1)).max() < 1e-13
    assert np.abs(t3.convection_p2(m, v) @ np.ones(m.N2)).max() < 1e-13


def test_prolongation_reproduces_polynomials():
    c = t3.Mesh3D(2)
    f = t3.Mesh3D(4)
    lin = lambda X: 1.0 + 2 * X[:, 0] - X[:, 1] + 0.5 * X[:, 2]                       # noqa: E731
    quad = lambda X: X[:, 0] * X[:, 1] - X[:, 2] ** 2 + 3 * X[:, 1] + 0.25            # noqa: E731
    assert np.allclose(t3.prolongation_p1(c) @ lin(c.x1), lin(f.x1), atol=1e-13)
    assert np.allclose(t3.prolongation_p2(c) @ quad(c.x2), quad(f.x2), atol=1e-13)
    assert np.array_equal(t3.inject_p1(np.arange(f.N1, dtype=float), 4),
                          np.array([int(f.id1(2 * c.lat1[k])) for k in range(c.N1)], dtype=float))


def test_mms_p1_rate():
    """(M + K) u = int f psi with u = cos(pi x) cos(pi y) cos(pi z) (natural
    Neumann data): L2 error O(h^2)."""
    ex = lambda x, y, z: np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)    # noqa: E731
    errs = []
    for n in (4, 8, 16):
        m = t3.Mesh3D(n)
        A = (t3.mass_p1(m) + t3.stiffness_p1(m)).tocsc()
        b = t3.load_p1(m, lambda lam: (1 + 3 * np.pi ** 2) * ex(*np.moveaxis(t3.quad_points(m, lam), -1, 0)), 6)
        errs.append(t3.l2_error_p1(m, spla.spsolve(A, b), ex))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert rates[1] > 1.85 and rates[1] > rates[0]      # 1.73, 1.91: approaching 2


def test_mms_taylor_hood_stokes_rates():
    """Stokes with no-slip: u = curl-type field of psi = sin^2 sin^2 sin^2
    (solenoidal, zero on every face), p = cos cos cos: velocity L2 O(h^3)."""
    sym = pytest.importorskip("sympy")
    X, Y, Z = sym.symbols("x y z")
    psi = sym.sin(sym.pi * X) ** 2 * sym.sin(sym.pi * Y) ** 2 * sym.sin(sym.pi * Z) ** 2
    u = [sym.diff(psi, Y), -sym.diff(psi, X), sym.Integer(0)]
    p = sym.cos(sym.pi * X) * sym.cos(sym.pi * Y) * sym.cos(sym.pi * Z)
    f = [-(sym.diff(c, X, 2) + sym.diff(c, Y, 2) + sym.diff(c, Z, 2)) + sym.diff(p, v) for c, v in zip(u, (X, Y, Z))]
    uf = [sym.lambdify((X, Y, Z), c, "numpy") for c in u]
    ff = [sym.lambdify((X, Y, Z), c, "numpy") for c in f]

    def vec(fs):
        return lambda x, y, z: tuple(np.broadcast_to(fn(x, y, z), np.shape(x)) for fn in fs)
    errs = []
    for n in (2, 4):
        m = t3.Mesh3D(n)
        bnd = m.p2_boundary()
        A = t3.velocity_dirichlet(t3.ksym(m, 1.0), bnd)
        B = t3.zero_velocity_columns(t3.divergence(m), bnd)
        rhs = t3.load_velocity(m, vec(ff), 6)
        rhs[np.repeat(bnd, 3)] = 0.0
        mvec = t3.mass_p1(m) @ np.ones(m.N1)
        K = sp.bmat([[A, B.T, None], [B, None, sp.csr_matrix(mvec[:, None])],
                     [None, sp.csr_matrix(mvec[None, :]), None]], format="csc")
        x = spla.spsolve(K, np.concatenate([rhs, np.zeros(m.N1 + 1)]))
        errs.append(t3.l2_error_velocity(m, x[:3 * m.N2], vec(uf)))
    assert math.log2(errs[0] / errs[1]) > 2.5


def test_mg_contraction_independent_of_mesh():
    """V-cycle contraction on tau K + a M: bounded and levelling off as
    levels are added (measured 0.09, 0.18, 0.22 at 8^3, 16^3, 32^3)."""
    rates = []
    for n in (8, 16, 32):
        sizes = t3.level_sizes(n)
        meshes = [t3.Mesh3D(s) for s in sizes]
        P = [t3.prolongation_p1(meshes[l + 1]) for l in range(len(sizes) - 1)]
        mats = [(1e-3 * t3.stiffness_p1(mm) + 0.05 * t3.mass_p1(mm)).tocsr() for mm in meshes]
        mg = MG(mats, P)
        A = mats[0]
        b = np.random.default_rng(n).standard_normal(A.shape[0])
        r = [np.linalg.norm(b - A @ mg.solve(b, 0.0, k)[0]) for k in (2, 3)]
        rates.append(r[1] / r[0])
    assert max(rates) < 0.3
    assert rates[2] - rates[1] < 0.6 * (rates[1] - rates[0])


@pytest.fixture(scope="module")
def two_steps():
    n = 4
    p = inputs.default_params()
    p.update(rtol=1e-11, alpha=[1e-2] * 4)
    o = t3.Oracle3D(n, p)
    ox = t3.Oracle3D(n, p, exact=True)
    s0 = inputs.initial_state_3d(n, seed=1)
    s1, i1 = o.step(s0)
    s2, i2 = o.step(s1)
    x1 = ox.step(s0)[0]
    x2 = ox.step(s1)[0]
    return o, s0, s1, s2, (i1, i2), (x1, x2)


def test_step_matches_sparse_lu(two_steps):
    o, s0, s1, s2, infos, (x1, x2) = two_steps
    for info in infos:
        for name in ("ch_p", "ch_N", "ch_s", "ac", "ns"):
            assert info[name]["converged"], name
    for got, ref in ((s1, x1), (s2, x2)):
        for key in ("phi", "mu", "Phi_v", "v", "p"):
            a, b = np.ravel(got[key]), np.ravel(ref[key])
            assert np.linalg.norm(a - b) <= 1e-7 * max(np.linalg.norm(b), 1e-30), key
    assert np.abs(s2["v"]).max() > 0.0          # the second step has flow


def test_mass_conservation_and_divergence(two_steps):
    o, s0, s1, s2, _, _ = two_steps
    d0, d1, d2 = (o.diagnostics(s) for s in (s0, s1, s2))
    for i in range(2):                          # polymer, NFA: no boundary flux
        assert d1["mass"][i] == pytest.approx(d0["mass"][i], rel=1e-9)
        assert d2["mass"][i] == pytest.approx(d0["mass"][i], rel=1e-9)
    assert d2["div"] < 1e-9
    assert abs(d2["p_mean"]) < 1e-12


def test_preconditioned_iterations_are_mesh_robust():
    """The block preconditioners keep the iteration counts nearly flat under
    refinement (the paper's 3D observation, Sec. 5): second step at 4^3,
    8^3, 16^3 cubes -- CH 19, 21, 24; AC 4, 5, 4; NS 53, 62, 65."""
    p = inputs.default_params()
    its = []
    for n in (4, 8, 16):
        o = t3.Oracle3D(n, p)
        s = o.step(inputs.initial_state_3d(n, seed=2))[0]
        its.append({k: v["iters"] for k, v in o.step(s)[1].items()})
    for a, b in zip(its, its[1:]):
        assert b["ch_p"] <= a["ch_p"] + 5 and b["ac"] <= a["ac"] + 2
    d1, d2 = its[1]["ns"] - its[0]["ns"], its[2]["ns"] - its[1]["ns"]
    assert d2 <= d1 and its[2]["ns"] <= 80


def test_weighted_stiffness_closed_forms():
    """K_kappa of the concentration-dependent mobility gamma (phi (1 - phi) + m0):
    symmetric, rows summing to zero (so CH mass stays conserved), gamma (c (1 - c)
    + m0) K for a constant phi = c, and for phi = x (exact in P1) the energy of
    u = x is int gamma (x (1 - x) + m0) dx = gamma (1/6 + m0) over the unit cube."""
    mesh = t3.Mesh3D(4)
    g, m0 = 1.3, 1e-3
    p = dict(inputs.default_params(), mobility_kind=1, mobility_m0=m0, gamma=[g, g, g])
    x = mesh.x1[:, 0]
    Kk = t3.weighted_stiffness_p1(mesh, t3.mobility_at(mesh, x, p, 0))
    assert abs(Kk - Kk.T).max() < 1e-14
    assert np.abs(Kk @ np.ones(mesh.N1)).max() < 1e-13
    assert x @ (Kk @ x) == pytest.approx(g * (1.0 / 6.0 + m0), rel=1e-13)
    c = 0.3
    Kc = t3.weighted_stiffness_p1(mesh, t3.mobility_at(mesh, np.full(mesh.N1, c), p, 0))
    assert abs(Kc - g * (c * (1 - c) + m0) * t3.stiffness_p1(mesh)).max() < 1e-13


def test_variable_mobility_step_matches_sparse_lu():
    """With the concentration-dependent mobility the first row's tau K_kappa and
    the Schur factor X2 = tau K_kappa + a M change; the preconditioned step still
    reaches the sparse-LU step, and polymer and NFA mass stay conserved."""
    n = 4
    p = inputs.default_params()
    p.update(rtol=1e-11, alpha=[1e-2] * 4, mobility_kind=1, gamma=[1.0, 0.8, 1.2])
    o, ox = t3.Oracle3D(n, p), t3.Oracle3D(n, p, exact=True)
    s0 = inputs.initial_state_3d(n, seed=3)
    s1, info = o.step(s0)
    x1 = ox.step(s0)[0]
    assert all(v["converged"] for v in info.values())
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        a, b = np.ravel(s1[key]), np.ravel(x1[key])
        assert np.linalg.norm(a - b) <= 1e-7 * max(np.linalg.norm(b), 1e-30), key
    d0, d1 = o.diagnostics(s0), o.diagnostics(s1)
    for i in range(2):
        assert d1["mass"][i] == pytest.approx(d0["mass"][i], rel=1e-9)


def test_inner_multigrid_step_matches_sparse_lu():
    """With every multigrid block iterated to inner_rtol = 1e-4 (Sec. 5's AMG
    tolerance) the preconditioners change but the step still reaches the
    sparse-LU step; the inner solves cut the AC iterations (4 -> 2 or 3)."""
    n = 4
    p = inputs.default_params()
    p.update(rtol=1e-11, alpha=[1e-2] * 4)
    s0 = inputs.initial_state_3d(n, seed=5)
    plain = t3.Oracle3D(n, p).step(s0)[1]
    o = t3.Oracle3D(n, dict(p, inner_rtol=1e-4, inner_maxit=20))
    s1, info = o.step(s0)
    x1 = t3.Oracle3D(n, p, exact=True).step(s0)[0]
    assert all(v["converged"] for v in info.values())
    assert info["ac"]["iters"] < plain["ac"]["iters"]
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        a, b = np.ravel(s1[key]), np.ravel(x1[key])
        assert np.linalg.norm(a - b) <= 1e-7 * max(np.linalg.norm(b), 1e-30), key


def test_open_top_masks():
    """Open top: the prescribed-velocity P2 nodes are every face but the
    interior of the top face ((2n - 1)^2 nodes fewer, its edges stay on the
    side walls); K_p with Dirichlet rows on the (n + 1)^2 top nodes is
    non-singular."""
    n = 4
    closed, open_ = t3.Mesh3D(n), t3.Mesh3D(n, top_free=True)
    a, b = closed.p2_boundary(), open_.p2_boundary()
    assert np.all(b <= a) and a.sum() - b.sum() == (2 * n - 1) ** 2
    freed = a & ~b
    assert np.all(open_.lat2[freed, 2] == 2 * n)
    assert np.all((open_.lat2[freed, :2] > 0) & (open_.lat2[freed, :2] < 2 * n))
    assert open_.p1_top().sum() == (n + 1) ** 2
    Kd = p1_dirichlet_dense(t3.stiffness_p1(open_), open_.p1_top())
    assert np.linalg.matrix_rank(Kd) == open_.N1


def p1_dirichlet_dense(K, mask):
    D = K.toarray()
    D[mask, :] = 0.0
    D[:, mask] = 0.0
    D[mask, mask] = 1.0
    return D


@pytest.fixture(scope="module")
def open_steps():
    n = 4
    p = inputs.default_params()
    p.update(rtol=1e-11, alpha=[1e-2] * 4, top_bc=1)
    o, ox = t3.Oracle3D(n, p), t3.Oracle3D(n, p, exact=True)
    s0 = inputs.initial_state_3d(n, seed=6)
    s1, i1 = o.step(s0)
    s2, i2 = o.step(s1)
    return o, (s1, s2), (i1, i2), (ox.step(s0)[0], ox.step(s1)[0])


def test_open_top_step_matches_sparse_lu(open_steps):
    o, steps, infos, exact = open_steps
    for info in infos:
        assert all(v["converged"] for v in info.values())
    for got, ref in zip(steps, exact):
        for key in ("phi", "mu", "Phi_v", "v", "p"):
            a, b = np.ravel(got[key]), np.ravel(ref[key])
            assert np.linalg.norm(a - b) <= 1e-7 * max(np.linalg.norm(b), 1e-30), key


def test_open_top_flow_leaves_through_the_top(open_steps):
    """The do-nothing top lets the velocity through the top face (zero there
    for enclosed flow); the velocity stays discretely divergence-free."""
    o, (s1, s2), _, _ = open_steps
    mesh = o.mesh
    top = (mesh.lat2[:, 2] == 2 * mesh.n) & ~mesh.p2_boundary()
    assert np.abs(s2["v"].reshape(-1, 3)[top]).max() > 1e-5
    assert np.abs(s2["v"].reshape(-1, 3)[mesh.p2_boundary()]).max() == 0.0
    assert o.diagnostics(s2)["div"] < 1e-9


def _linear_state(mesh):
    x, y, z = mesh.x1.T
    return {"phi": np.stack([0.3 + 0.05 * (x + 2 * y + 3 * z), 0.25 + 0.04 * (x - y), np.full(mesh.N1, 0.4)]),
            "Phi_v": 0.2 * z, "mu": np.zeros((4, mesh.N1)), "v": np.zeros(3 * mesh.N2)}


def test_korteweg_load_of_linear_fields():
    """Linear fields give a constant Korteweg tensor G, and then int G grad zeta_a
    is the boundary integral of zeta_a G n: zero at interior P2 nodes, and at a
    node inside the top face G e_z times int_top zeta_a, which is h^2 / 3 for an
    edge midpoint (two triangles of area h^2 / 2, a third each) and 0 for a
    vertex."""
    n = 4
    mesh = t3.Mesh3D(n)
    p = dict(inputs.default_params(), beta=[0.01, 0.02, 0.1, 1.0], beta_v=0.7)
    st = _linear_state(mesh)
    Gt = t3.korteweg_tensor(mesh, st, p)
    G = Gt[0]
    assert np.allclose(Gt, G[None], atol=1e-15) and np.abs(G).max() > 1e-3
    L = t3.korteweg(mesh, Gt).reshape(-1, 3)
    lat, m = mesh.lat2, 2 * n
    inner = np.all((lat > 0) & (lat < m), axis=1)
    assert np.abs(L[inner]).max() < 1e-15
    top = (lat[:, 2] == m) & np.all((lat[:, :2] > 0) & (lat[:, :2] < m), axis=1)
    mid = top & ((lat[:, 0] % 2 == 1) | (lat[:, 1] % 2 == 1))
    h2 = mesh.h[0] * mesh.h[1]
    assert np.allclose(L[mid], G[:, 2][None] * h2 / 3.0, rtol=1e-12, atol=1e-16)
    assert np.abs(L[top & ~mid]).max() < 1e-15


def test_potential_loads_constant_and_linear_fields():
    """Constant fields: int df/dphi_k psi_a = df/dphi_k (M 1)_a (the partials are
    pinned by finite differences in 2D).  Linear fields: the integrands are
    polynomials of degree <= 7, so a degree-11 rule gives the same loads."""
    mesh = t3.Mesh3D(3)
    c = np.full(mesh.N1, 1.0)
    loads = t3.potential_loads(mesh, np.stack([0.3 * c, 0.25 * c, 0.4 * c]), 0.2 * c)
    d = t3.potential_partials(0.3, 0.25, 0.4, 0.05, 0.2)
    m1 = t3.mass_p1(mesh) @ c
    for k in range(5):
        assert np.allclose(loads[k], d[k] * m1, rtol=1e-12, atol=1e-15)
    st = _linear_state(mesh)
    lin = t3.potential_loads(mesh, st["phi"], st["Phi_v"])
    for k in range(5):
        def integrand(lam, k=k):
            pp, pn, ps = (t3.p1_field_at(mesh, st["phi"][i], lam) for i in range(3))
            return t3.potential_partials(pp, pn, ps, 1.0 - pp - pn - ps, t3.p1_field_at(mesh, st["Phi_v"], lam))[k]
        ref = t3.load_p1(mesh, integrand, 11)
        assert np.allclose(lin[k], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_convection_of_polynomials():
    """P1 and P2 convection by a quadratic velocity (exact in P2) with a
    constant shift s: C(v, s) x = int (v_x - s_x) psi_a and
    J(v, s) q = int ((v - s) . grad q) zeta_a for the quadratic q = x y + z^2,
    computed from the analytic fields at the quadrature points."""
    m = t3.Mesh3D(2)
    X = m.x2
    vfun = lambda x, y, z: (y * y, x * z, x + y)                                        # noqa: E731
    v = np.stack(vfun(X[:, 0], X[:, 1], X[:, 2]), axis=1).ravel()
    s = np.array([0.3, -0.2, 0.1])
    shift = np.tile(s, (m.E, 1))
    C = t3.convection_p1(m, v, shift)
    ref = t3.load_p1(m, lambda lam: vfun(*np.moveaxis(t3.quad_points(m, lam), -1, 0))[0] - s[0], 3)
    assert np.allclose(C @ m.x1[:, 0], ref, rtol=1e-12, atol=1e-15)
    q = X[:, 0] * X[:, 1] + X[:, 2] ** 2
    J = t3.convection_p2(m, v, shift)

    def vgq(x, y, z):
        vx, vy, vz = vfun(x, y, z)
        val = (vx - s[0]) * y + (vy - s[1]) * x + (vz - s[2]) * 2 * z
        return val, 0.0 * x, 0.0 * x
    ref2 = t3.load_velocity(m, vgq, 5)[0::3]
    assert np.allclose(J @ q, ref2, rtol=1e-12, atol=1e-15)


def test_symmetric_gradient_form_on_quadratics():
    """At interior P2 nodes K_sym u = -eta int div(2 sym grad u) zeta_a: for
    u = (y^2, 0, 0) the divergence is (2, 0, 0), for u = (x^2, 0, 0) it is
    (4, 0, 0) (the Laplacian form would give 2 for both)."""
    m = t3.Mesh3D(4)
    eta = 1.3
    K = t3.ksym(m, eta)
    X = m.x2
    w = t3.mass_p2(m) @ np.ones(m.N2)
    inner = np.all((m.lat2 > 0) & (m.lat2 < 2 * m.n), axis=1)
    zero = np.zeros(m.N2)
    for ux, dx in ((X[:, 1] ** 2, 2.0), (X[:, 0] ** 2, 4.0)):
        r = (K @ np.stack([ux, zero, zero], axis=1).ravel()).reshape(-1, 3)
        assert np.abs(r[inner, 0] + eta * dx * w[inner]).max() < 1e-11 * eta * dx * np.abs(w).max()
        assert np.abs(r[inner, 1:]).max() < 1e-14


def test_open_top_with_inner_solves_and_variable_mobility():
    """The open top, the concentration-dependent mobility and inner solves to
    1e-4 together (K_p with Dirichlet top rows as an inner solve, X2 per
    species): the step still reaches the sparse-LU step."""
    n = 4
    p = inputs.default_params()
    p.update(rtol=1e-11, alpha=[1e-2] * 4, top_bc=1, mobility_kind=1, inner_rtol=1e-4, inner_maxit=20)
    s0 = inputs.initial_state_3d(n, seed=9)
    s1, info = t3.Oracle3D(n, p).step(s0)
    x1 = t3.Oracle3D(n, p, exact=True).step(s0)[0]
    assert all(v["converged"] for v in info.values())
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        a, b = np.ravel(s1[key]), np.ravel(x1[key])
        assert np.linalg.norm(a - b) <= 1e-7 * max(np.linalg.norm(b), 1e-30), key
