"""Discrete adjoint of the 3D step (oracle; TEST INFRASTRUCTURE: only tests/
use it).

The reverse sweep of oracle/adjoint.py on the Kuhn tetrahedra of
oracle/three_d.py: for every linear solve A(u^k, theta) x = b(u^k, theta) of
the step, y = A^{-T} xbar and ubar += (d b / d u)^T y - (d (A(u) x) / d u)^T y,
with the transposed Jacobian products of the state-dependent pieces written
for tetrahedra: the convection C(v) on P1 and J(w) on P2
(w = v - sum alpha_i grad mu_i), the potential loads (Hessian of
eqn:appPotential), the Korteweg load, the evaporation flux and, with the
concentration-dependent mobility, K_kappa(phi_i^k).  theta = (evaporation
rate, mobility scale gamma with gamma_i = gamma).  Objective
J = int |grad phi_p|^2 = phi_p^T K phi_p at the final time.  Enclosed flow or
the open top; the forward solves are the sparse-LU ones of
Oracle3D(exact=True), whose transposes are solved here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import three_d as t3
from .adjoint import A, N, P, S, V, hessian
from .quadrature import tetra_rule


def loads_vjp(mesh, phi, Phi, weights):
    """Gradient of sum_i weights[i]^T F_i (F_i = int g_i psi, g_i = df/dvar_i
    at phi_a = 1 - sum phi) with respect to (phi_p, phi_N, phi_s) and Phi_v."""
    lam, w = tetra_rule(7)
    _, vol, _ = mesh.element_geometry()
    pp, pn, ps = (t3.p1_field_at(mesh, phi[i], lam) for i in range(3))
    pa = 1.0 - pp - pn - ps
    H = hessian(pp, pn, ps, pa, t3.p1_field_at(mesh, Phi, lam))
    zq = [None if z is None else t3.p1_field_at(mesh, z, lam) for z in weights]

    def integrate(gq):
        return t3._scatter_vec(vol[:, None] * np.einsum("q,eq,qa->ea", w, gq, lam), mesh.tet, mesh.N1)

    phibar = np.zeros((3, mesh.N1))
    for j in (P, N, S):
        g = 0.0 * pp
        for i in range(5):
            if zq[i] is not None:
                g = g + (H[i][j] - H[i][A]) * zq[i]      # phi_a = 1 - sum phi
        phibar[j] = integrate(g)
    g = 0.0 * pp
    for i in range(5):
        if zq[i] is not None:
            g = g + H[i][V] * zq[i]
    return phibar, integrate(g)


def conv_p1_vjp(mesh, x, y):
    """d/dv of y^T C(v) x, C_ab = int (v . grad psi_b) psi_a: the velocity
    gradient (3 N2), int zeta_k (d_d x) y."""
    lam, w = tetra_rule(3)
    _, vol, g = mesh.element_geometry()
    gx = np.einsum("ea,ead->ed", x[mesh.tet], g)
    yq = t3.p1_field_at(mesh, y, lam)
    loc = vol[:, None, None] * np.einsum("q,qk,eq,ed->ekd", w, t3.p2_values(lam), yq, gx)
    return t3._scatter_vec(loc.reshape(mesh.E, 30), t3.vel_dofs(mesh), 3 * mesh.N2)


def conv_p2_vjp(mesh, x, y):
    """d/dw of y^T (J(w) (x) I) x for interleaved velocities x, y: the nodal
    gradient (3 N2), int zeta_k sum_c (d_d x_c) y_c, and the gradient with
    respect to a per-element constant shift s of w = v - s, (E,3)."""
    lam, w = tetra_rule(5)
    _, vol, g = mesh.element_geometry()
    dN = t3.p2_grads(lam, g)                                        # (E,Q,10,3)
    gradx = np.einsum("eqbd,ebc->eqcd", dN, x.reshape(-1, 3)[mesh.tet2])
    t = np.einsum("eqcd,eqc->eqd", gradx, t3.p2_field_at(mesh, y, lam))
    loc = vol[:, None, None] * np.einsum("q,qk,eqd->ekd", w, t3.p2_values(lam), t)
    out = t3._scatter_vec(loc.reshape(mesh.E, 30), t3.vel_dofs(mesh), 3 * mesh.N2)
    return out, -vol[:, None] * np.einsum("q,eqd->ed", w, t)


def korteweg_vjp(mesh, phi, Phi, y, params):
    """d/d(phi_p, phi_N, phi_s, Phi_v) of y^T G, G_(a,c) = int sum_b G_cb
    d_b zeta_a with G = sum_i beta_i grad phi_i (x) grad phi_i + beta_v
    grad Phi (x) grad Phi, phi_a = 1 - sum phi."""
    _, vol, g = mesh.element_geometry()
    lam, w = tetra_rule(1)
    dN = t3.p2_grads(lam, g)
    Y = vol[:, None, None] * np.einsum("q,eqab,eac->ecb", w, dN, y.reshape(-1, 3)[mesh.tet2])
    Ssym = Y + np.transpose(Y, (0, 2, 1))
    grads = [t3.p1_gradient(mesh, phi[i]) for i in range(3)]
    ga = -(grads[0] + grads[1] + grads[2])
    beta = params["beta"]

    def scatter(vec_e):
        return t3._scatter_vec(np.einsum("ed,emd->em", vec_e, g), mesh.tet, mesh.N1)

    phibar = np.stack([scatter(np.einsum("ecb,eb->ec", Ssym, beta[j] * grads[j] - beta[3] * ga))
                       for j in range(3)])
    return phibar, scatter(np.einsum("ecb,eb->ec", Ssym, params["beta_v"] * t3.p1_gradient(mesh, Phi)))


def wstiff_vjp(mesh, phi_i, gamma, x, y):
    """d/d phi_i of y^T K_kappa(phi_i) x, kappa = gamma (phi (1 - phi) + m0):
    int gamma (1 - 2 phi_h) psi_c grad x_h . grad y_h (degree 2, exact)."""
    lam, w = tetra_rule(2)
    _, vol, g = mesh.element_geometry()
    ph = t3.p1_field_at(mesh, phi_i, lam)
    dot = np.sum(np.einsum("ea,ead->ed", x[mesh.tet], g) * np.einsum("ea,ead->ed", y[mesh.tet], g), axis=1)
    loc = vol[:, None] * dot[:, None] * np.einsum("eq,q,qc->ec", gamma * (1.0 - 2.0 * ph), w, lam)
    return t3._scatter_vec(loc, mesh.tet, mesh.N1)


def _solve_T(M, rhs):
    return spla.spsolve(M.T.tocsc(), rhs)


def adjoint_step(o: t3.Oracle3D, st, new, lam):
    """One reverse step of the 3D step.  st: state at t_k, new: the forward
    output at t_{k+1}, lam: adjoint of the state at t_{k+1}.  Returns (adjoint
    at t_k, {"evap": .., "gamma": ..})."""
    p = o.params
    mesh, F = o.mesh, o.forms[0]
    tau, N1 = p["tau"], mesh.N1
    beta = p["beta"]
    bnd = np.repeat(mesh.p2_boundary(), 3)
    out = {"phi": np.zeros((3, N1)), "mu": np.zeros((4, N1)), "Phi_v": np.zeros(N1),
           "v": np.zeros(3 * mesh.N2), "p": np.zeros(N1)}
    lam_phi_new = lam["phi"].copy()
    jbar = gbar = 0.0
    top, ref = F.top, mesh.top_reference_node()
    loads = t3.potential_loads(mesh, st["phi"], st["Phi_v"])
    j = p["evap_rate"] * (st["phi"][2][ref] - p["phi_s_inf"])
    f = [loads[0], loads[1], loads[2] - beta[2] * j * top]
    C = t3.convection_p1(mesh, st["v"])
    lw = [None] * 5
    # Oseen: the transposed saddle point (with the zero-mean constraint for enclosed flow)
    Amat, B, _, _, _ = t3.ns_system(F, st, p)
    nv = Amat.shape[0]
    m = F.M @ np.ones(N1)
    lv = np.where(bnd, 0.0, lam["v"])
    if o.top_free:
        y = spla.spsolve(sp.bmat([[Amat.T, B.T], [B, None]], format="csc"), np.concatenate([lv, lam["p"]]))
    else:
        lp = lam["p"] - m * lam["p"].sum() / m.sum()     # transpose of the zero-mean shift
        K = sp.bmat([[Amat.T, B.T, None], [B, None, sp.csr_matrix(m[:, None])],
                     [None, sp.csr_matrix(m[None, :]), None]], format="csc")
        y = spla.spsolve(K, np.concatenate([lv, lp, [0.0]]))
    yv = y[:nv]
    out["v"] += F.velocity_forms()["Mv"] @ yv / tau
    kp, kv = korteweg_vjp(mesh, st["phi"], st["Phi_v"], yv, p)
    out["phi"] += kp
    out["Phi_v"] += kv
    wbar, sbar = conv_p2_vjp(mesh, np.where(bnd, 0.0, new["v"]), yv)
    out["v"] -= wbar
    _, _, gl = mesh.element_geometry()
    for i in range(4):                                    # d s / d mu_i = alpha_i grad psi
        out["mu"][i] += t3._scatter_vec(-p["alpha"][i] * np.einsum("ed,emd->em", sbar, gl), mesh.tet, N1)
    # air potential: M mu_a = f_a + beta_a K (1 - sum phi^{k+1}), f_a = F_a + beta_a j t
    z = spla.spsolve(F.M.tocsc(), lam["mu"][3])
    for i in range(3):
        lam_phi_new[i] -= beta[3] * (F.K @ z)
    lw[A] = z
    jbar += beta[3] * (top @ z)
    # Allen-Cahn
    Aac = (F.M + tau * p["delta_v"] * F.K + tau * C).tocsr()
    y = _solve_T(Aac, lam["Phi_v"])
    out["Phi_v"] += F.M @ y
    lw[V] = -tau * p["gamma_v"] * y
    out["v"] -= tau * conv_p1_vjp(mesh, new["Phi_v"], y)
    if p["ac_top_flux"]:
        jbar += tau * p["delta_v"] * (top @ y)
    # Cahn-Hilliard, three species
    for i in range(3):
        g_i, b_i = p["gamma"][i], beta[i]
        Kk = g_i * F.K if p["mobility_kind"] == 0 else t3.weighted_stiffness_p1(
            mesh, t3.mobility_at(mesh, st["phi"][i], p, i))
        c = tau * g_i / b_i
        Ach = sp.bmat([[F.M + tau * C, tau * Kk], [tau * g_i * F.K, -c * F.M]], format="csr")
        y = _solve_T(Ach, np.concatenate([lam_phi_new[i], lam["mu"][i]]))
        y1, y2 = y[:N1], y[N1:]
        out["phi"][i] += F.M @ y1
        lw[i] = -c * y2
        if i == 2:
            jbar += c * b_i * (top @ y2)                  # f_s = F_s - beta_s j t
        out["v"] -= tau * conv_p1_vjp(mesh, new["phi"][i], y1)
        mu_new = new["mu"][i]
        # d/dgamma_i of (b - A x); tau K_kappa is gamma_i times a gamma-free matrix
        db = -(tau / b_i) * f[i] @ y2
        dAx = (y1 @ (tau * (Kk @ mu_new)) / g_i
               + y2 @ (tau * (F.K @ new["phi"][i]) - (tau / b_i) * (F.M @ mu_new)))
        gbar += db - dAx
        if p["mobility_kind"] != 0:
            out["phi"][i] -= tau * wstiff_vjp(mesh, st["phi"][i], g_i, mu_new, y1)
    # potential loads and the evaporation flux
    lp_phi, lp_Phi = loads_vjp(mesh, st["phi"], st["Phi_v"], lw)
    out["phi"] += lp_phi
    out["Phi_v"] += lp_Phi
    evap_bar = jbar * (st["phi"][2][ref] - p["phi_s_inf"])
    out["phi"][2][ref] += jbar * p["evap_rate"]
    out["v"][bnd] = 0.0
    return out, {"evap": evap_bar, "gamma": gbar}


def objective(o: t3.Oracle3D, st):
    """J = int |grad phi_p|^2 = phi_p^T K phi_p."""
    return float(st["phi"][0] @ (o.forms[0].K @ st["phi"][0]))


def trajectory_gradient(n, params, st0, steps):
    """J after `steps` sparse-LU steps on the Kuhn mesh of n^3 cubes and its
    gradient with respect to the evaporation rate, the mobility scale and
    every field of the initial state."""
    o = t3.Oracle3D(n, params, exact=True)
    states = [st0]
    for _ in range(steps):
        states.append(o.step(states[-1])[0])
    J = objective(o, states[-1])
    lam = {k: np.zeros_like(np.asarray(v, dtype=float)) for k, v in st0.items()}
    lam["phi"][0] = 2.0 * (o.forms[0].K @ states[-1]["phi"][0])
    g_evap = g_gamma = 0.0
    for k in range(steps, 0, -1):
        lam, th = adjoint_step(o, states[k - 1], states[k], lam)
        g_evap += th["evap"]
        g_gamma += th["gamma"]
    return J, {"evap": g_evap, "gamma": g_gamma, "state0": lam}
