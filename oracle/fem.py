"""Element integrals and global assembly (oracle; TEST INFRASTRUCTURE).

Every form is integrated with a quadrature rule exact for its integrand
degree on affine triangles, element by element, and summed into a global
scipy.sparse matrix (duplicates added).  Forms follow the paper:
  M, K, C            Sec. 4 (CH / AC systems: mass, stiffness, convection)
  M_vel, J, K_sym, B Sec. 4, eqn:matrixns (entries j_mn, k_mn, b_mn)
  M_p, K_p, A_p      Sec. 4 (pressure mass, stiffness, convection-diffusion)
  G                  Sec. 3, eqn:weakns right-hand side  int G : grad u
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh
from .quadrature import triangle_rule, edge_rule


# ----------------------------------------------------------------------------
# basis functions on one element, at barycentric points lam (Q,3)
def p1_values(lam):
    return lam.copy()                                       # (Q,3)


def p2_values(lam):
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    return np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                     4 * l1 * l2, 4 * l0 * l2, 4 * l0 * l1], axis=1)  # (Q,6)


def p2_grads(lam, g):
    """Gradients of the six P2 basis functions: (E,Q,6,2) for barycentric
    gradients g (E,3,2)."""
    l0, l1, l2 = (lam[:, k][None, :, None] for k in range(3))
    g0, g1, g2 = (g[:, k][:, None, :] for k in range(3))
    return np.stack([(4 * l0 - 1) * g0, (4 * l1 - 1) * g1, (4 * l2 - 1) * g2,
                     4 * (l1 * g2 + l2 * g1), 4 * (l0 * g2 + l2 * g0),
                     4 * (l0 * g1 + l1 * g0)], axis=2)


def p2_field_at(mesh: Mesh, v, lam):
    """Velocity (interleaved 2*N2) at quadrature points: (E,Q,2)."""
    vn = v.reshape(-1, 2)[mesh.tri2]                        # (E,6,2)
    return np.einsum("qa,ead->eqd", p2_values(lam), vn)


def p1_field_at(mesh: Mesh, f, lam):
    return np.einsum("qa,ea->eq", lam, f[mesh.tri])


def p1_gradient(mesh: Mesh, f):
    """Piecewise-constant gradient of a P1 field: (E,2)."""
    _, _, g = mesh.element_geometry()
    return np.einsum("ea,ead->ed", f[mesh.tri], g)


# ----------------------------------------------------------------------------
def _scatter(local, rows, cols, shape):
    """Sum element matrices local (E,a,b) into a CSR matrix."""
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


def vel_dofs(mesh: Mesh):
    """Global velocity indices (E,12) ordered (node a, component c) -> 2*node+c."""
    return (2 * mesh.tri2[:, :, None] + np.arange(2)[None, None, :]).reshape(mesh.E, 12)


# ----------------------------------------------------------------------------
# P1 forms
def mass_p1(mesh: Mesh):
    """M_ab = int psi_a psi_b (Sec. 4)."""
    lam, w = triangle_rule(2)
    _, area, _ = mesh.element_geometry()
    phi = p1_values(lam)
    loc = area[:, None, None] * np.einsum("q,qa,qb->ab", w, phi, phi)[None]
    return _scatter(loc, mesh.tri, mesh.tri, (mesh.N1, mesh.N1))


def stiffness_p1(mesh: Mesh):
    """K_ab = int grad psi_a . grad psi_b (Sec. 4)."""
    _, area, g = mesh.element_geometry()
    loc = area[:, None, None] * np.einsum("ead,ebd->eab", g, g)
    return _scatter(loc, mesh.tri, mesh.tri, (mesh.N1, mesh.N1))


def weighted_stiffness_p1(mesh: Mesh, kappa_at):
    """K_kappa,ab = int kappa grad psi_a . grad psi_b, kappa given at the
    points of the degree-2 rule as an (E,Q) array (variable mobility)."""
    lam, w = triangle_rule(2)
    _, area, g = mesh.element_geometry()
    kap = kappa_at(lam)                                       # (E,Q)
    loc = (area * (kap @ w))[:, None, None] * np.einsum("ead,ebd->eab", g, g)
    return _scatter(loc, mesh.tri, mesh.tri, (mesh.N1, mesh.N1))


def convection_p1(mesh: Mesh, v, shift=None):
    """C_ab = int ((v - shift) . grad psi_b) psi_a with v a P2 velocity and
    shift a per-element constant vector (E,2) or None (Sec. 4: C; A_p)."""
    lam, w = triangle_rule(3)
    _, area, g = mesh.element_geometry()
    vq = p2_field_at(mesh, v, lam)                          # (E,Q,2)
    if shift is not None:
        vq = vq - shift[:, None, :]
    phi = p1_values(lam)                                    # (Q,3)
    vg = np.einsum("eqd,ebd->eqb", vq, g)                   # (E,Q,3)
    loc = area[:, None, None] * np.einsum("q,qa,eqb->eab", w, phi, vg)
    return _scatter(loc, mesh.tri, mesh.tri, (mesh.N1, mesh.N1))


# ----------------------------------------------------------------------------
# P2 / Taylor-Hood forms
def mass_p2(mesh: Mesh):
    """Scalar P2 mass int zeta_a zeta_b (N2 x N2)."""
    lam, w = triangle_rule(4)
    _, area, _ = mesh.element_geometry()
    N = p2_values(lam)
    loc = area[:, None, None] * np.einsum("q,qa,qb->ab", w, N, N)[None]
    return _scatter(loc, mesh.tri2, mesh.tri2, (mesh.N2, mesh.N2))


def convection_p2(mesh: Mesh, v, shift=None):
    """Scalar j_ab = int ((v - shift) . grad zeta_b) zeta_a (eqn:matrixns j_mn
    with w = rho v - sum alpha_i grad mu_i), N2 x N2."""
    lam, w = triangle_rule(5)
    _, area, g = mesh.element_geometry()
    vq = p2_field_at(mesh, v, lam)
    if shift is not None:
        vq = vq - shift[:, None, :]
    N = p2_values(lam)                                      # (Q,6)
    dN = p2_grads(lam, g)                                   # (E,Q,6,2)
    vg = np.einsum("eqd,eqbd->eqb", vq, dN)                 # (E,Q,6)
    loc = area[:, None, None] * np.einsum("q,qa,eqb->eab", w, N, vg)
    return _scatter(loc, mesh.tri2, mesh.tri2, (mesh.N2, mesh.N2))


def ksym(mesh: Mesh, eta: float):
    """k_{(a,c),(b,d)} = int 2 eta sym(zeta_b e_d) : sym(zeta_a e_c)
    = eta int (delta_cd grad zeta_b . grad zeta_a + d_c zeta_b d_d zeta_a)
    (eqn:matrixns k_mn), on interleaved velocity dofs (2N2 x 2N2)."""
    lam, w = triangle_rule(2)
    _, area, g = mesh.element_geometry()
    dN = p2_grads(lam, g)                                   # (E,Q,6,2)
    lap = np.einsum("q,eqad,eqbd->eab", w, dN, dN)          # (E,6,6)
    cross = np.einsum("q,eqbc,eqad->eacbd", w, dN, dN)      # (E,a,c,b,d) = d_c N_b d_d N_a
    loc = cross + lap[:, :, None, :, None] * np.eye(2)[None, None, :, None, :]
    loc = eta * area[:, None, None, None, None] * loc
    loc = loc.reshape(mesh.E, 12, 12)
    dofs = vel_dofs(mesh)
    return _scatter(loc, dofs, dofs, (2 * mesh.N2, 2 * mesh.N2))


def divergence(mesh: Mesh):
    """b_{q,(b,d)} = - int psi_q d_d zeta_b (eqn:matrixns b_mn, pressure rows),
    N1 x 2N2."""
    lam, w = triangle_rule(2)
    _, area, g = mesh.element_geometry()
    dN = p2_grads(lam, g)                                   # (E,Q,6,2)
    loc = -area[:, None, None, None] * np.einsum("q,qa,eqbd->eabd", w, p1_values(lam), dN)
    loc = loc.reshape(mesh.E, 3, 12)
    return _scatter(loc, mesh.tri, vel_dofs(mesh), (mesh.N1, 2 * mesh.N2))


# ----------------------------------------------------------------------------
# load vectors
def load_p1(mesh: Mesh, integrand, degree: int):
    """int g psi_a with g given at the quadrature points as integrand(lam)
    returning (E,Q)."""
    lam, w = triangle_rule(degree)
    _, area, _ = mesh.element_geometry()
    gq = integrand(lam)
    loc = area[:, None] * np.einsum("q,eq,qa->ea", w, gq, p1_values(lam))
    return _scatter_vec(loc, mesh.tri, mesh.N1)


def top_load_p1(mesh: Mesh):
    """t_a = int_{Gamma_t} psi_a ds on the top edge y = Ly."""
    s, w = edge_rule(1)
    n = mesh.n
    out = np.zeros(mesh.N1)
    for i in range(n):
        a, b = n * (n + 1) + i, n * (n + 1) + i + 1
        out[a] += mesh.hx * np.sum(w * (1 - s))
        out[b] += mesh.hx * np.sum(w * s)
    return out


def korteweg(mesh: Mesh, Gt):
    """G_{(a,c)} = int sum_b G_cb d_b zeta_a for a per-element constant
    tensor Gt (E,2,2) (eqn:weakns right-hand side)."""
    lam, w = triangle_rule(1)
    _, area, g = mesh.element_geometry()
    dN = p2_grads(lam, g)                                   # (E,Q,6,2)
    loc = area[:, None, None] * np.einsum("q,ecb,eqab->eac", w, Gt, dN)
    return _scatter_vec(loc.reshape(mesh.E, 12), vel_dofs(mesh), 2 * mesh.N2)


# ----------------------------------------------------------------------------
def velocity_dirichlet(A, bnd_nodes_mask):
    """No-slip (eqn:bc): keep boundary velocity dofs in the system as identity
    rows with zero coupling in both directions."""
    mask = np.repeat(bnd_nodes_mask, 2)
    Dint = sp.diags((~mask).astype(float))
    Db = sp.diags(mask.astype(float))
    out = (Dint @ A @ Dint + Db).tocsr()
    out.eliminate_zeros()
    out.sort_indices()
    return out


def p1_dirichlet(A, nodes_mask):
    """Homogeneous Dirichlet rows / columns on P1 nodes: identity rows, zero
    coupling in both directions (the outflow condition of the pressure
    convection-diffusion operators, Elman-Silvester-Wathen, cited in Sec. 4)."""
    Dint = sp.diags((~nodes_mask).astype(float))
    Db = sp.diags(nodes_mask.astype(float))
    out = (Dint @ A @ Dint + Db).tocsr()
    out.eliminate_zeros()
    out.sort_indices()
    return out


def zero_velocity_columns(B, bnd_nodes_mask):
    mask = np.repeat(bnd_nodes_mask, 2)
    out = (B @ sp.diags((~mask).astype(float))).tocsr()
    out.eliminate_zeros()
    return out


def quad_points(mesh: Mesh, lam):
    """Physical coordinates of barycentric points lam (Q,3) on every
    element: (E,Q,2)."""
    return np.einsum("qa,ead->eqd", lam, mesh.x1[mesh.tri])


def load_velocity(mesh: Mesh, fn, degree: int):
    """int f . (zeta_a e_c) for a vector function fn(x, y) -> (fx, fy)."""
    lam, w = triangle_rule(degree)
    _, area, _ = mesh.element_geometry()
    X = quad_points(mesh, lam)
    fx, fy = fn(X[..., 0], X[..., 1])
    F = np.stack([fx, fy], axis=-1)                         # (E,Q,2)
    loc = area[:, None, None] * np.einsum("q,eqc,qa->eac", w, F, p2_values(lam))
    return _scatter_vec(loc.reshape(mesh.E, 12), vel_dofs(mesh), 2 * mesh.N2)


def l2_error_p1(mesh: Mesh, uh, fn, degree: int = 8):
    lam, w = triangle_rule(degree)
    _, area, _ = mesh.element_geometry()
    X = quad_points(mesh, lam)
    d = p1_field_at(mesh, uh, lam) - fn(X[..., 0], X[..., 1])
    return float(np.sqrt(np.sum(area[:, None] * w[None] * d * d)))


def l2_error_velocity(mesh: Mesh, vh, fn, degree: int = 8):
    lam, w = triangle_rule(degree)
    _, area, _ = mesh.element_geometry()
    X = quad_points(mesh, lam)
    fx, fy = fn(X[..., 0], X[..., 1])
    d = p2_field_at(mesh, vh, lam) - np.stack([fx, fy], axis=-1)
    return float(np.sqrt(np.sum(area[:, None] * w[None] * np.sum(d * d, axis=-1))))


def convection_p1_wind(mesh: Mesh, wind):
    """C_ab = int (w . grad psi_b) psi_a with w a P1 vector field given at
    the vertices, (N1, 2) (the convection matrix C of Sec. 4 with a
    prescribed velocity; also on oracle.mesh.TriMesh)."""
    lam, w = triangle_rule(2)
    _, area, g = mesh.element_geometry()
    phi = p1_values(lam)                                    # (Q,3)
    wq = np.einsum("qk,ekd->eqd", phi, np.asarray(wind)[mesh.tri])   # (E,Q,2)
    vg = np.einsum("eqd,ebd->eqb", wq, g)                   # (E,Q,3)
    loc = area[:, None, None] * np.einsum("q,qa,eqb->eab", w, phi, vg)
    return _scatter(loc, mesh.tri, mesh.tri, (mesh.N1, mesh.N1))
