"""The semi-implicit step on tetrahedral meshes of a box (oracle; TEST
INFRASTRUCTURE: only tests/ and the CPU legs of the bench use it).

The paper's 3D runs (Sec. 5: n_x = n_y = n_z = 40, polymer / NFA / solvent
Cahn-Hilliard with the polynomial potential eqn:appPotential, Allen-Cahn,
Navier-Stokes) use uniform tetrahedral meshes of a cube.  Here the box
[0,lx] x [0,ly] x [0,lz] is cut into n^3 cubes, each split into the six
Kuhn (Freudenthal) tetrahedra along its main diagonal: the 3D analogue of
the diagonal split of the 2D meshes, nested under dyadic refinement.  P1
for the phase fields, potentials and pressure; P2 (vertices and edge
midpoints, i.e. the points of the doubled lattice) for the velocity
(Taylor-Hood).  The step, its systems and its solvers are those of
oracle/step.py with every form integrated exactly on tetrahedra: CH for
three species with diag(MG(M + tau C), X^{-1} M X^{-1}), AC with MG, the air
potential by Jacobi-PCG, Oseen with diag(MG(A), M_p^{-1} A_p K_p^{-1}),
FGMRES(30) with CGS2, geometric multigrid with rediscretised coarse
operators and injected coefficients.  Enclosed flow (no-slip on every face),
or with top_bc = 1 the open top of oracle/step.py: no-slip on the bottom and
the side walls, the do-nothing condition on the top face (natural in the weak
form), Dirichlet outflow rows of A_p and K_p on the top face in the PCD and
no pressure normalisation; evaporation through the top face z = lz,
reference point (lx/2, ly/2, lz).

Conventions.  Cube (i, j, k) has id (k n + j) n + i; its tetrahedron p
(p = index of the axis order sigma in PERMS) has vertices v0 = (i, j, k),
v1 = v0 + e_sigma0, v2 = v1 + e_sigma1, v3 = (i+1, j+1, k+1) and element id
6 cube + p.  P1 node (a, b, c) has id (c (n+1) + b)(n+1) + a; P2 node
(A, B, C) of the doubled lattice has id (C m + B) m + A, m = 2n + 1.  Local
P2 numbering: the four vertices, then the midpoints of the edges in EDGES.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import p1_dirichlet
from .krylov import chebyshev, fgmres, pcg
from .mg import MG
from .model import potential_partials
from .quadrature import tetra_rule

PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
VEL_SMOOTH_DEGREE, VEL_LO_RATIO = 4, 16.0   # Taylor-Hood velocity operator
MASS_CHEB_DEGREE = 5
MASS_CHEB_BOUNDS = (0.5, 2.5)               # spectrum of D^{-1} M for P1 tetrahedra (Wathen)


# ----------------------------------------------------------------------------
class Mesh3D:
    def __init__(self, n: int, lx: float = 1.0, ly: float = 1.0, lz: float = 1.0, top_free: bool = False):
        if n < 1:
            raise ValueError("n must be >= 1")
        self.n = n
        self.top_free = top_free
        self.L = np.array([lx, ly, lz], dtype=float)
        self.h = self.L / n
        self.N1 = (n + 1) ** 3
        self.N2 = (2 * n + 1) ** 3
        self.E = 6 * n ** 3
        c = np.arange(n ** 3)
        base = np.stack([c % n, (c // n) % n, c // (n * n)], axis=1)
        lat = np.empty((n ** 3, 6, 4, 3), dtype=np.int64)
        for p, perm in enumerate(PERMS):
            v = base.copy()
            lat[:, p, 0] = v
            for s in range(3):
                v = v.copy()
                v[:, perm[s]] += 1
                lat[:, p, s + 1] = v
        lat = lat.reshape(self.E, 4, 3)
        self.tet = self.id1(lat)
        tet2 = np.empty((self.E, 10), dtype=np.int64)
        tet2[:, :4] = self.id2(2 * lat)
        for q, (a, b) in enumerate(EDGES):
            tet2[:, 4 + q] = self.id2(lat[:, a] + lat[:, b])
        self.tet2 = tet2
        g1 = np.stack(np.meshgrid(*(np.arange(n + 1),) * 3, indexing="ij"), axis=-1)   # (a, b, c)
        lat1 = g1.transpose(2, 1, 0, 3).reshape(-1, 3)                                   # id order
        self.lat1 = lat1
        self.x1 = lat1 * self.h
        m = 2 * n + 1
        g2 = np.stack(np.meshgrid(*(np.arange(m),) * 3, indexing="ij"), axis=-1)
        self.lat2 = g2.transpose(2, 1, 0, 3).reshape(-1, 3)
        self.x2 = self.lat2 * (self.h / 2)

    def id1(self, lat):
        n1 = self.n + 1
        return (lat[..., 2] * n1 + lat[..., 1]) * n1 + lat[..., 0]

    def id2(self, lat):
        m = 2 * self.n + 1
        return (lat[..., 2] * m + lat[..., 1]) * m + lat[..., 0]

    def p2_boundary(self):
        """P2 nodes with prescribed (zero) velocity: every face (eqn:bc), or,
        on a top_free mesh, all but the open top face (its edges stay on the
        side walls)."""
        m = 2 * self.n
        side = np.any((self.lat2[:, :2] == 0) | (self.lat2[:, :2] == m), axis=1)
        top = (self.lat2[:, 2] == m) & (not self.top_free)
        return side | (self.lat2[:, 2] == 0) | top

    def p1_top(self):
        return self.lat1[:, 2] == self.n

    def top_reference_node(self) -> int:
        if self.n % 2:
            raise ValueError("the top reference point needs an even n")
        return int(self.id1(np.array([self.n // 2, self.n // 2, self.n])))

    def element_geometry(self):
        """Vertex coordinates (E,4,3), volumes (E,), barycentric gradients (E,4,3)."""
        X = self.x1[self.tet]
        Jm = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
        inv = np.linalg.inv(Jm)
        g = np.empty((self.E, 4, 3))
        g[:, 1:] = inv
        g[:, 0] = -inv.sum(axis=1)
        return X, np.abs(np.linalg.det(Jm)) / 6.0, g


# ----------------------------------------------------------------------------
# basis functions at barycentric points lam (Q,4)
def p2_values(lam):
    out = [lam[:, a] * (2 * lam[:, a] - 1) for a in range(4)]
    out += [4 * lam[:, a] * lam[:, b] for a, b in EDGES]
    return np.stack(out, axis=1)                                  # (Q,10)


def p2_grads(lam, g):
    """(E,Q,10,3) gradients of the P2 basis for barycentric gradients g (E,4,3)."""
    L = [lam[:, a][None, :, None] for a in range(4)]
    G = [g[:, a][:, None, :] for a in range(4)]
    out = [(4 * L[a] - 1) * G[a] for a in range(4)]
    out += [4 * (L[a] * G[b] + L[b] * G[a]) for a, b in EDGES]
    return np.stack(out, axis=2)


def p1_field_at(mesh, f, lam):
    return np.einsum("qa,ea->eq", lam, f[mesh.tet])


def p2_field_at(mesh, v, lam):
    vn = v.reshape(-1, 3)[mesh.tet2]                              # (E,10,3)
    return np.einsum("qa,ead->eqd", p2_values(lam), vn)


def p1_gradient(mesh, f):
    _, _, g = mesh.element_geometry()
    return np.einsum("ea,ead->ed", f[mesh.tet], g)


def _scatter(local, rows, cols, shape):
    E, na, nb = local.shape
    r = np.repeat(rows, nb, axis=1).reshape(E, na, nb)
    c = np.tile(cols, (1, na)).reshape(E, na, nb)
    A = sp.coo_matrix((local.ravel(), (r.ravel(), c.ravel())), shape=shape).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def _scatter_vec(local, rows, size):
    out = np.zeros(size)
    np.add.at(out, rows.ravel(), local.ravel())
    return out


def vel_dofs(mesh):
    return (3 * mesh.tet2[:, :, None] + np.arange(3)[None, None, :]).reshape(mesh.E, 30)


# ----------------------------------------------------------------------------
# forms (Sec. 4), exact on tetrahedra
def mass_p1(mesh):
    lam, w = tetra_rule(2)
    _, vol, _ = mesh.element_geometry()
    loc = vol[:, None, None] * np.einsum("q,qa,qb->ab", w, lam, lam)[None]
    return _scatter(loc, mesh.tet, mesh.tet, (mesh.N1, mesh.N1))


def stiffness_p1(mesh):
    _, vol, g = mesh.element_geometry()
    loc = vol[:, None, None] * np.einsum("ead,ebd->eab", g, g)
    return _scatter(loc, mesh.tet, mesh.tet, (mesh.N1, mesh.N1))


def weighted_stiffness_p1(mesh, kappa_at):
    lam, w = tetra_rule(2)
    _, vol, g = mesh.element_geometry()
    loc = (vol * (kappa_at(lam) @ w))[:, None, None] * np.einsum("ead,ebd->eab", g, g)
    return _scatter(loc, mesh.tet, mesh.tet, (mesh.N1, mesh.N1))


def convection_p1(mesh, v, shift=None):
    """C_ab = int ((v - shift) . grad psi_b) psi_a, v a P2 velocity."""
    lam, w = tetra_rule(3)
    _, vol, g = mesh.element_geometry()
    vq = p2_field_at(mesh, v, lam)
    if shift is not None:
        vq = vq - shift[:, None, :]
    vg = np.einsum("eqd,ebd->eqb", vq, g)
    loc = vol[:, None, None] * np.einsum("q,qa,eqb->eab", w, lam, vg)
    return _scatter(loc, mesh.tet, mesh.tet, (mesh.N1, mesh.N1))


def mass_p2(mesh):
    lam, w = tetra_rule(4)
    _, vol, _ = mesh.element_geometry()
    N = p2_values(lam)
    loc = vol[:, None, None] * np.einsum("q,qa,qb->ab", w, N, N)[None]
    return _scatter(loc, mesh.tet2, mesh.tet2, (mesh.N2, mesh.N2))


def convection_p2(mesh, v, shift=None):
    lam, w = tetra_rule(5)
    _, vol, g = mesh.element_geometry()
    vq = p2_field_at(mesh, v, lam)
    if shift is not None:
        vq = vq - shift[:, None, :]
    vg = np.einsum("eqd,eqbd->eqb", vq, p2_grads(lam, g))
    loc = vol[:, None, None] * np.einsum("q,qa,eqb->eab", w, p2_values(lam), vg)
    return _scatter(loc, mesh.tet2, mesh.tet2, (mesh.N2, mesh.N2))


def ksym(mesh, eta):
    """eta int (delta_cd grad zeta_b . grad zeta_a + d_c zeta_b d_d zeta_a)
    on interleaved velocity dofs (3 N2 x 3 N2)."""
    lam, w = tetra_rule(2)
    _, vol, g = mesh.element_geometry()
    dN = p2_grads(lam, g)
    lap = np.einsum("q,eqad,eqbd->eab", w, dN, dN)
    cross = np.einsum("q,eqbc,eqad->eacbd", w, dN, dN)
    loc = cross + lap[:, :, None, :, None] * np.eye(3)[None, None, :, None, :]
    loc = (eta * vol[:, None, None, None, None] * loc).reshape(mesh.E, 30, 30)
    dofs = vel_dofs(mesh)
    return _scatter(loc, dofs, dofs, (3 * mesh.N2, 3 * mesh.N2))


def divergence(mesh):
    """b_{q,(b,d)} = - int psi_q d_d zeta_b (pressure rows), N1 x 3 N2."""
    lam, w = tetra_rule(2)
    _, vol, g = mesh.element_geometry()
    dN = p2_grads(lam, g)
    loc = -vol[:, None, None, None] * np.einsum("q,qa,eqbd->eabd", w, lam, dN)
    return _scatter(loc.reshape(mesh.E, 4, 30), mesh.tet, vel_dofs(mesh), (mesh.N1, 3 * mesh.N2))


def load_p1(mesh, integrand, degree):
    lam, w = tetra_rule(degree)
    _, vol, _ = mesh.element_geometry()
    loc = vol[:, None] * np.einsum("q,eq,qa->ea", w, integrand(lam), lam)
    return _scatter_vec(loc, mesh.tet, mesh.N1)


def top_load_p1(mesh):
    """t_a = int_{Gamma_t} psi_a dS on z = lz: the top face of each cube is
    cut along its (0,0)-(1,1) diagonal by the Kuhn tetrahedra; a P1 hat
    integrates to |triangle| / 3 on each triangle of its vertex."""
    n = mesh.n
    out = np.zeros(mesh.N1)
    area = mesh.h[0] * mesh.h[1] / 2.0
    for j in range(n):
        for i in range(n):
            v = lambda a, b: int(mesh.id1(np.array([a, b, n])))   # noqa: E731
            for t in ((v(i, j), v(i + 1, j), v(i + 1, j + 1)), (v(i, j), v(i + 1, j + 1), v(i, j + 1))):
                for a in t:
                    out[a] += area / 3.0
    return out


def korteweg(mesh, Gt):
    """G_(a,c) = int sum_b G_cb d_b zeta_a, Gt per element (E,3,3)."""
    lam, w = tetra_rule(1)
    _, vol, g = mesh.element_geometry()
    loc = vol[:, None, None] * np.einsum("q,ecb,eqab->eac", w, Gt, p2_grads(lam, g))
    return _scatter_vec(loc.reshape(mesh.E, 30), vel_dofs(mesh), 3 * mesh.N2)


def velocity_dirichlet(A, bnd_nodes):
    mask = np.repeat(bnd_nodes, 3)
    out = (sp.diags((~mask).astype(float)) @ A @ sp.diags((~mask).astype(float)) + sp.diags(mask.astype(float)))
    out = out.tocsr()
    out.eliminate_zeros()
    out.sort_indices()
    return out


def zero_velocity_columns(B, bnd_nodes):
    out = (B @ sp.diags((~np.repeat(bnd_nodes, 3)).astype(float))).tocsr()
    out.eliminate_zeros()
    return out


def quad_points(mesh, lam):
    return np.einsum("qa,ead->eqd", lam, mesh.x1[mesh.tet])


def load_velocity(mesh, fn, degree):
    lam, w = tetra_rule(degree)
    _, vol, _ = mesh.element_geometry()
    X = quad_points(mesh, lam)
    F = np.stack(fn(X[..., 0], X[..., 1], X[..., 2]), axis=-1)           # (E,Q,3)
    loc = vol[:, None, None] * np.einsum("q,eqc,qa->eac", w, F, p2_values(lam))
    return _scatter_vec(loc.reshape(mesh.E, 30), vel_dofs(mesh), 3 * mesh.N2)


def l2_error_p1(mesh, uh, fn, degree=6):
    lam, w = tetra_rule(degree)
    _, vol, _ = mesh.element_geometry()
    X = quad_points(mesh, lam)
    d = p1_field_at(mesh, uh, lam) - fn(X[..., 0], X[..., 1], X[..., 2])
    return float(np.sqrt(np.sum(vol[:, None] * w[None] * d * d)))


def l2_error_velocity(mesh, vh, fn, degree=6):
    lam, w = tetra_rule(degree)
    _, vol, _ = mesh.element_geometry()
    X = quad_points(mesh, lam)
    d = p2_field_at(mesh, vh, lam) - np.stack(fn(X[..., 0], X[..., 1], X[..., 2]), axis=-1)
    return float(np.sqrt(np.sum(vol[:, None] * w[None] * np.sum(d * d, axis=-1))))


# ----------------------------------------------------------------------------
# transfers between nested Kuhn meshes
def _locate(nc, X):
    """X (N,3) in units of coarse cells -> element id of a containing Kuhn
    tetrahedron and its barycentric coordinates (N,4)."""
    cell = np.minimum(np.floor(X).astype(np.int64), nc - 1)
    loc = X - cell
    order = np.argsort(-loc, axis=1, kind="stable")              # sigma: decreasing coordinates
    code = order[:, 0] * 9 + order[:, 1] * 3 + order[:, 2]
    table = {p[0] * 9 + p[1] * 3 + p[2]: k for k, p in enumerate(PERMS)}
    perm = np.vectorize(table.get)(code)
    srt = np.take_along_axis(loc, order, axis=1)
    lam = np.stack([1 - srt[:, 0], srt[:, 0] - srt[:, 1], srt[:, 1] - srt[:, 2], srt[:, 2]], axis=1)
    cube = (cell[:, 2] * nc + cell[:, 1]) * nc + cell[:, 0]
    return 6 * cube + perm, lam


def prolongation_p1(coarse: Mesh3D):
    """Linear interpolation of coarse P1 functions at the fine (2 nc) nodes."""
    fine = Mesh3D(2 * coarse.n)
    e, lam = _locate(coarse.n, fine.lat1 / 2.0)
    rows = np.repeat(np.arange(fine.N1), 4)
    P = sp.coo_matrix((lam.ravel(), (rows, coarse.tet[e].ravel())), shape=(fine.N1, coarse.N1)).tocsr()
    P.sum_duplicates()
    P.eliminate_zeros()
    return P


def prolongation_p2(coarse: Mesh3D):
    """Quadratic interpolation of coarse P2 functions at the fine P2 nodes."""
    fine = Mesh3D(2 * coarse.n)
    e, lam = _locate(coarse.n, fine.lat2 / 4.0)
    rows = np.repeat(np.arange(fine.N2), 10)
    P = sp.coo_matrix((p2_values(lam).ravel(), (rows, coarse.tet2[e].ravel())),
                      shape=(fine.N2, coarse.N2)).tocsr()
    P.sum_duplicates()
    P.eliminate_zeros()
    return P


def prolongation_velocity(coarse: Mesh3D, fine: Mesh3D):
    P = prolongation_p2(coarse)
    P = (sp.diags((~fine.p2_boundary()).astype(float)) @ P @ sp.diags((~coarse.p2_boundary()).astype(float))).tocsr()
    P.eliminate_zeros()
    return sp.kron(P, sp.eye(3), format="csr")


def inject_p1(f, nf):
    F = f.reshape(nf + 1, nf + 1, nf + 1)
    return np.ascontiguousarray(F[::2, ::2, ::2]).ravel()


def inject_velocity(v, nf):
    m = 2 * nf + 1
    V = v.reshape(m, m, m, 3)
    return np.ascontiguousarray(V[::2, ::2, ::2, :]).ravel()


def level_sizes(n):
    sizes = [n]
    while sizes[-1] % 2 == 0 and sizes[-1] >= 4:
        sizes.append(sizes[-1] // 2)
    return sizes


# ----------------------------------------------------------------------------
# the model (Sec. 2-4) on a tetrahedral mesh
def potential_loads(mesh, phi, Phi):
    """int df/dphi_i psi (i = p, N, s, a) and int df/dPhi psi of
    eqn:appPotential, phi_a = 1 - sum phi (degree-7 integrands)."""
    out = []
    for k in range(5):
        def integrand(lam, k=k):
            pp, pn, ps = (p1_field_at(mesh, phi[i], lam) for i in range(3))
            return potential_partials(pp, pn, ps, 1.0 - pp - pn - ps, p1_field_at(mesh, Phi, lam))[k]
        out.append(load_p1(mesh, integrand, 7))
    return out


def mobility_at(mesh, phi_i, params, species):
    g = params["gamma"][species]
    if params["mobility_kind"] == 0:
        return lambda lam: np.full((mesh.E, lam.shape[0]), g)
    m0 = params["mobility_m0"]
    return lambda lam: g * (p1_field_at(mesh, phi_i, lam) * (1.0 - p1_field_at(mesh, phi_i, lam)) + m0)


class Forms3D:
    def __init__(self, mesh: Mesh3D, params):
        self.mesh = mesh
        self.params = params
        self.M = mass_p1(mesh)
        self.K = stiffness_p1(mesh)
        self.top = top_load_p1(mesh)
        self._vel = None

    def velocity_forms(self):
        if self._vel is None:
            m = self.mesh
            bnd = m.p2_boundary()
            M2 = mass_p2(m)
            self._vel = {"bnd": bnd, "M2": M2, "Mv": sp.kron(M2, sp.eye(3), format="csr"),
                         "Ksym": ksym(m, self.params["eta"]),
                         "B": zero_velocity_columns(divergence(m), bnd)}
        return self._vel


def ns_shift(mesh, state, params):
    return sum(params["alpha"][i] * p1_gradient(mesh, state["mu"][i]) for i in range(4))


def korteweg_tensor(mesh, state, params):
    phi = state["phi"]
    grads = [p1_gradient(mesh, phi[i]) for i in range(3)]
    grads.append(-(grads[0] + grads[1] + grads[2]))
    Gt = sum(params["beta"][i] * np.einsum("ec,ed->ecd", grads[i], grads[i]) for i in range(4))
    gv = p1_gradient(mesh, state["Phi_v"])
    return Gt + params["beta_v"] * np.einsum("ec,ed->ecd", gv, gv)


def ns_system(forms, state, params):
    mesh = forms.mesh
    vf = forms.velocity_forms()
    tau = params["tau"]
    shift = ns_shift(mesh, state, params)
    A = vf["Mv"] / tau + sp.kron(convection_p2(mesh, state["v"], shift), sp.eye(3), format="csr") + vf["Ksym"]
    A = velocity_dirichlet(A.tocsr(), vf["bnd"])
    rhs_v = vf["Mv"] @ state["v"] / tau + korteweg(mesh, korteweg_tensor(mesh, state, params))
    rhs_v[np.repeat(vf["bnd"], 3)] = 0.0
    Ap = (forms.M / tau + params["eta"] * forms.K + convection_p1(mesh, state["v"], shift)).tocsr()
    if mesh.top_free:
        Ap = p1_dirichlet(Ap, mesh.p1_top())       # PCD outflow condition on the open top
    return A, vf["B"], rhs_v, Ap, shift


def _direct(A, b):
    x = spla.spsolve(A.tocsc(), b)
    nb = float(np.linalg.norm(b))
    return x, {"iters": 0, "rel_residual": float(np.linalg.norm(b - A @ x)) / nb if nb else 0.0, "converged": True}


class Oracle3D:
    """One step of the model on the Kuhn mesh of n^3 cubes (see the module
    docstring); exact=True replaces every Krylov solve by sparse LU."""

    def __init__(self, n, params, exact=False):
        self.params = dict(params)
        self.exact = exact
        self.sizes = level_sizes(n)
        self.top_free = self.params.get("top_bc", 0) == 1
        self.meshes = [Mesh3D(s, top_free=self.top_free) for s in self.sizes]
        self.forms = [Forms3D(m, self.params) for m in self.meshes]
        self.P1 = [prolongation_p1(self.meshes[l + 1]) for l in range(len(self.sizes) - 1)]
        self.Pv = [prolongation_velocity(self.meshes[l + 1], self.meshes[l]) for l in range(len(self.sizes) - 1)]
        self._Kp = None

    @property
    def mesh(self):
        return self.meshes[0]

    def level_states(self, state):
        out = [state]
        for l in range(len(self.sizes) - 1):
            nf = self.sizes[l]
            s = out[-1]
            out.append({"v": inject_velocity(s["v"], nf), "mu": np.stack([inject_p1(m, nf) for m in s["mu"]]),
                        "phi": np.stack([inject_p1(f, nf) for f in s["phi"]])})
        return out

    def _mg(self, mats, prolongs, **kw):
        mg = MG(mats, prolongs, **kw)
        rtol = self.params.get("inner_rtol", 0.0)
        return mg if not rtol else (lambda b: mg.solve(b, rtol, self.params.get("inner_maxit", 20))[0])

    def step(self, state):
        p = self.params
        mesh, F = self.mesh, self.forms[0]
        tau = p["tau"]
        N1 = mesh.N1
        lst = self.level_states(state)
        convs = [convection_p1(f.mesh, s["v"]) for f, s in zip(self.forms, lst)]
        loads = potential_loads(mesh, state["phi"], state["Phi_v"])
        j = p["evap_rate"] * (state["phi"][2][mesh.top_reference_node()] - p["phi_s_inf"])
        beta = p["beta"]
        f = [loads[0], loads[1], loads[2] - beta[2] * j * F.top, loads[3] + beta[3] * j * F.top]
        new = {"phi": np.empty_like(state["phi"]), "mu": np.empty_like(state["mu"])}
        info = {}
        # Cahn-Hilliard, three species (eqn:CH_linear)
        for i, name in enumerate(("ch_p", "ch_N", "ch_s")):
            g, b = p["gamma"][i], p["beta"][i]
            L0 = (F.M + tau * convs[0]).tocsr()
            Kk = g * F.K if p["mobility_kind"] == 0 else weighted_stiffness_p1(
                mesh, mobility_at(mesh, state["phi"][i], p, i))
            c = tau * g / b
            A = sp.bmat([[L0, tau * Kk], [tau * g * F.K, -c * F.M]], format="csr")
            rhs = np.concatenate([F.M @ state["phi"][i], -c * f[i]])
            if self.exact:
                x, inf = _direct(A, rhs)
            else:
                a = math.sqrt(tau * g / b)
                mgL = self._mg([(fm.M + tau * C).tocsr() for fm, C in zip(self.forms, convs)], self.P1)
                X1 = [(tau * g * fm.K + a * fm.M).tocsr() for fm in self.forms]
                mgX1 = self._mg(X1, self.P1)
                if p["mobility_kind"] == 0:
                    mgX2 = mgX1
                else:
                    mgX2 = self._mg([(tau * weighted_stiffness_p1(fm.mesh, mobility_at(fm.mesh, s["phi"][i], p, i))
                                      + a * fm.M).tocsr() for fm, s in zip(self.forms, lst)], self.P1)

                def prec(r, mgL=mgL, mgX1=mgX1, mgX2=mgX2):
                    return np.concatenate([mgL(r[:N1]), mgX2(F.M @ mgX1(r[N1:]))])
                x, inf = fgmres(lambda y: A @ y, prec, rhs, p["rtol"], p["atol"], p["restart"], p["maxit"])
            new["phi"][i], new["mu"][i], info[name] = x[:N1], x[N1:], inf
        # Allen-Cahn
        Aac = (F.M + tau * p["delta_v"] * F.K + tau * convs[0]).tocsr()
        rac = F.M @ state["Phi_v"] - tau * p["gamma_v"] * loads[4]
        if p["ac_top_flux"]:
            rac = rac + tau * p["delta_v"] * j * F.top
        if self.exact:
            new["Phi_v"], info["ac"] = _direct(Aac, rac)
        else:
            mg = self._mg([(fm.M + tau * p["delta_v"] * fm.K + tau * C).tocsr() for fm, C in zip(self.forms, convs)],
                          self.P1)
            new["Phi_v"], info["ac"] = fgmres(lambda y: Aac @ y, mg, rac, p["rtol"], p["atol"], p["restart"], p["maxit"])
        # air potential (Sec. 5)
        phi_a = 1.0 - new["phi"].sum(axis=0)
        rmu = f[3] + beta[3] * (F.K @ phi_a)
        new["mu"][3], info["mu_a"] = _direct(F.M, rmu) if self.exact else pcg(F.M, rmu, 1.0 / F.M.diagonal(), rtol=1e-12)
        # Oseen (eqn:linearnav) with the pressure convection-diffusion preconditioner
        A, B, rhs_v, Ap, _ = ns_system(F, state, p)
        nv = A.shape[0]
        rhs = np.concatenate([rhs_v, np.zeros(N1)])
        m = F.M @ np.ones(N1)
        if self.exact and self.top_free:
            x, info["ns"] = _direct(sp.bmat([[A, B.T], [B, None]], format="csc"), rhs)
        elif self.exact:
            K = sp.bmat([[A, B.T, None], [B, None, sp.csr_matrix(m[:, None])],
                         [None, sp.csr_matrix(m[None, :]), None]], format="csc")
            x, info["ns"] = _direct(K, np.concatenate([rhs, [0.0]]))
            x = x[:-1]
        else:
            mats = [A]
            for l in range(1, len(self.sizes)):
                fm, s = self.forms[l], lst[l]
                vf = fm.velocity_forms()
                J2 = convection_p2(fm.mesh, s["v"], ns_shift(fm.mesh, s, p))
                mats.append(velocity_dirichlet((vf["Mv"] / tau + sp.kron(J2, sp.eye(3)) + vf["Ksym"]).tocsr(), vf["bnd"]))
            mgA = self._mg(mats, self.Pv, degree=VEL_SMOOTH_DEGREE, ratio=VEL_LO_RATIO)
            if self._Kp is None:
                if self.top_free:   # outflow: K_p with Dirichlet rows on the open top, non-singular
                    self._Kp = MG([p1_dirichlet(fm.K, fm.mesh.p1_top()) for fm in self.forms], self.P1,
                                  dense_coarse=True)
                else:
                    self._Kp = MG([fm.K for fm in self.forms], self.P1, singular=True, dense_coarse=True)
            kp = self._Kp if not p.get("inner_rtol", 0.0) else (
                lambda b: self._Kp.solve(b, p["inner_rtol"], p.get("inner_maxit", 20))[0])
            mdinv = 1.0 / F.M.diagonal()

            def prec(r):
                t = Ap @ kp(r[nv:])
                return np.concatenate([mgA(r[:nv]),
                                       chebyshev(lambda y: F.M @ y, mdinv, t, None, *MASS_CHEB_BOUNDS, MASS_CHEB_DEGREE)])

            def op(y):
                return np.concatenate([A @ y[:nv] + B.T @ y[nv:], B @ y[:nv]])
            rt, at = (p["ns_rtol"], p["ns_atol"]) if p.get("ns_rtol", 0.0) > 0 else (p["rtol"], p["atol"])
            x, info["ns"] = fgmres(op, prec, rhs, rt, at, p["restart"], p["maxit"])
        pr = x[nv:]
        # enclosed flow: pressure in L^2_0 (Sec. 3); open top: fixed by the do-nothing condition
        new["v"], new["p"] = x[:nv], pr if self.top_free else pr - (m @ pr) / m.sum()
        return new, info

    def diagnostics(self, state):
        F = self.forms[0]
        one = np.ones(self.mesh.N1)
        return {"mass": [float(one @ (F.M @ state["phi"][i])) for i in range(3)],
                "div": float(np.linalg.norm(F.velocity_forms()["B"] @ state["v"])),
                "p_mean": float(one @ (F.M @ state["p"]))}
