"""Discrete adjoint of the semi-implicit step (oracle; TEST INFRASTRUCTURE).

The step of oracle/step.py maps u^k = (phi_p, phi_N, phi_s, mu (4), Phi_v, v,
p) to u^{k+1} through linear solves A(u^k, theta) x = b(u^k, theta) (Sec. 4)
with theta = (evaporation rate, mobility scale gamma; gamma_i = gamma for all
three species).  For each solve, given the adjoint xbar of its solution x,
  y = A^{-T} xbar,   ubar += (d b / d u)^T y - (d (A(u) x) / d u)^T y,
which is the exact derivative of x = A^{-1} b.  The transposed Jacobian
products of the u-dependent pieces are written out here:
  convection C(v) on P1 and J(w) on P2 (w = v - sum alpha_i grad mu_i),
  the potential loads int df/dphi_i psi (Hessian of eqn:appPotential),
  the Korteweg load int G : grad u (G = sum beta_i grad phi_i (x) grad phi_i),
  the evaporation flux j_out = evap (phi_s^vap - phi_s^inf),
  the concentration-dependent mobility K_kappa(phi_i^k) of the first CH row
  (kappa = gamma_i (phi_i (1 - phi_i) + m0), Sec. 2.3 extension, lagged).
Objective of the adjoint check: J = int |grad phi_p|^2 = phi_p^T K phi_p at
the final time.  The pressure p^k does not enter the next step, and the
velocity is zero on the boundary, so those adjoint entries are zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, model
from .mesh import Mesh
from .quadrature import triangle_rule
from .step import Oracle

P, N, S, A, V = range(5)   # indices of (phi_p, phi_N, phi_s, phi_a, Phi_v)


def hessian(pp, pn, ps, pa, Phi):
    """Second partial derivatives H[i][j] of eqn:appPotential in the
    variables (phi_p, phi_N, phi_s, phi_a, Phi_v) (un-reduced)."""
    q = model.interp_p(Phi)
    dq = model.dinterp_p(Phi)
    ddq = 6.0 - 12.0 * Phi
    z = 0.0 * pp
    H = [[z] * 5 for _ in range(5)]
    H[P][P] = (1 - q) * 7.0 * pn**2 + 7.0 * q
    H[P][N] = H[N][P] = (1 - q) * 14.0 * pp * pn
    H[N][N] = (1 - q) * 7.0 * pp**2 + 7.0 * q
    H[S][S] = (1 - q) * 0.6 + 4.0 * q
    H[S][A] = H[A][S] = -(1 - q) * 10.0 + z
    H[A][A] = (1 - q) * 0.6 + 0.2 * q
    H[P][V] = H[V][P] = dq * 7.0 * pp * (1 - pn**2)
    H[N][V] = H[V][N] = dq * 7.0 * pn * (1 - pp**2)
    H[S][V] = H[V][S] = dq * (3.4 * ps + 10.0 * pa)
    H[A][V] = H[V][A] = dq * (10.0 * ps - 0.4 * pa)
    H[V][V] = ddq * (model.f_gas(pp, pn, ps, pa) - model.f_liquid(pp, pn, ps, pa))
    return H


def loads_vjp(mesh: Mesh, phi, Phi, weights):
    """Gradient of sum_i weights[i]^T F_i (F_i = int g_i psi, g_i = df/dvar_i
    at phi_a = 1 - sum phi, i over p, N, s, a, Phi_v) with respect to
    (phi_p, phi_N, phi_s) and Phi_v.  Returns (phibar (3,N1), Phibar (N1))."""
    lam, w = triangle_rule(7)
    _, area, _ = mesh.element_geometry()
    pp = fem.p1_field_at(mesh, phi[0], lam)
    pn = fem.p1_field_at(mesh, phi[1], lam)
    ps = fem.p1_field_at(mesh, phi[2], lam)
    pa = 1.0 - pp - pn - ps
    Ph = fem.p1_field_at(mesh, Phi, lam)
    H = hessian(pp, pn, ps, pa, Ph)
    zq = [None if z is None else fem.p1_field_at(mesh, z, lam) for z in weights]

    def integrate(gq):
        loc = area[:, None] * np.einsum("q,eq,qa->ea", w, gq, fem.p1_values(lam))
        out = np.zeros(mesh.N1)
        np.add.at(out, mesh.tri.ravel(), loc.ravel())
        return out

    phibar = np.zeros((3, mesh.N1))
    for j in (P, N, S):
        g = 0.0
        for i in range(5):
            if zq[i] is not None:
                g = g + (H[i][j] - H[i][A]) * zq[i]      # phi_a = 1 - sum phi
        phibar[j] = integrate(g + 0.0 * pp)
    g = 0.0
    for i in range(5):
        if zq[i] is not None:
            g = g + H[i][V] * zq[i]
    return phibar, integrate(g + 0.0 * pp)


def conv_p1_vjp(mesh: Mesh, x, y):
    """d/dv of y^T C(v) x, C_ab = int (v . grad psi_b) psi_a: returns the
    interleaved velocity gradient (2 N2): int zeta_k (d_d x) y."""
    lam, w = triangle_rule(3)
    _, area, g = mesh.element_geometry()
    gx = np.einsum("ea,ead->ed", x[mesh.tri], g)                    # (E,2)
    yq = fem.p1_field_at(mesh, y, lam)                              # (E,Q)
    Z = fem.p2_values(lam)                                          # (Q,6)
    loc = area[:, None, None] * np.einsum("q,qk,eq,ed->ekd", w, Z, yq, gx)
    out = np.zeros(2 * mesh.N2)
    np.add.at(out, fem.vel_dofs(mesh).ravel(), loc.reshape(mesh.E, 12).ravel())
    return out


def conv_p2_vjp(mesh: Mesh, x, y):
    """d/dw of y^T J(w) x (vector form, x and y interleaved velocities):
    returns (nodal gradient (2 N2) = int zeta_k sum_c (d_d x_c) y_c, and the
    per-element gradient with respect to a constant shift s of w = v - s,
    -int_T sum_c (d_d x_c) y_c, shape (E,2))."""
    lam, w = triangle_rule(5)
    _, area, g = mesh.element_geometry()
    dN = fem.p2_grads(lam, g)                                       # (E,Q,6,2)
    xn = x.reshape(-1, 2)[mesh.tri2]                                # (E,6,2) [node, comp]
    gradx = np.einsum("eqbd,ebc->eqcd", dN, xn)                     # d_d x_c at q
    yq = fem.p2_field_at(mesh, y, lam)                              # (E,Q,2)
    t = np.einsum("eqcd,eqc->eqd", gradx, yq)                       # sum_c d_d x_c y_c
    Z = fem.p2_values(lam)
    loc = area[:, None, None] * np.einsum("q,qk,eqd->ekd", w, Z, t)
    out = np.zeros(2 * mesh.N2)
    np.add.at(out, fem.vel_dofs(mesh).ravel(), loc.reshape(mesh.E, 12).ravel())
    sbar = -area[:, None] * np.einsum("q,eqd->ed", w, t)
    return out, sbar


def korteweg_vjp(mesh: Mesh, phi, Phi, y, params):
    """d/d(phi_p, phi_N, phi_s, Phi_v) of y^T G with G_(a,c) = int sum_b
    G_cb d_b zeta_a, G = sum_i beta_i grad phi_i (x) grad phi_i + beta_v grad
    Phi (x) grad Phi, phi_a = 1 - sum phi."""
    _, area, g = mesh.element_geometry()
    lam, w = triangle_rule(1)
    dN = fem.p2_grads(lam, g)                                       # (E,Q,6,2)
    yn = y.reshape(-1, 2)[mesh.tri2]                                # (E,6,2)
    Y = area[:, None, None] * np.einsum("q,eqab,eac->ecb", w, dN, yn)   # Y[c][b] = int d_b y_c
    Ssym = Y + np.transpose(Y, (0, 2, 1))
    grads = [fem.p1_gradient(mesh, phi[i]) for i in range(3)]
    ga = -(grads[0] + grads[1] + grads[2])
    gv = fem.p1_gradient(mesh, Phi)
    beta = params["beta"]

    def scatter(vec_e):                                             # (E,2) . grad psi_m
        loc = np.einsum("ed,emd->em", vec_e, g)
        out = np.zeros(mesh.N1)
        np.add.at(out, mesh.tri.ravel(), loc.ravel())
        return out

    phibar = np.zeros((3, mesh.N1))
    for j in range(3):
        phibar[j] = scatter(np.einsum("ecb,eb->ec", Ssym, beta[j] * grads[j] - beta[3] * ga))
    Phibar = scatter(np.einsum("ecb,eb->ec", Ssym, params["beta_v"] * gv))
    return phibar, Phibar


def wstiff_vjp(mesh: Mesh, phi_i, gamma, x, y):
    """d/d phi_i of y^T K_kappa(phi_i) x, kappa = gamma (phi (1 - phi) + m0):
    entry c = int gamma (1 - 2 phi_h) psi_c grad x_h . grad y_h (degree-2
    rule, exact: the integrand is quadratic on each triangle)."""
    lam, w = triangle_rule(2)
    _, area, g = mesh.element_geometry()
    ph = fem.p1_field_at(mesh, phi_i, lam)                        # (E,Q)
    gx = np.einsum("ea,ead->ed", x[mesh.tri], g)
    gy = np.einsum("ea,ead->ed", y[mesh.tri], g)
    dot = np.sum(gx * gy, axis=1)                                 # (E,)
    loc = area[:, None] * dot[:, None] * np.einsum("eq,q,qc->ec", gamma * (1.0 - 2.0 * ph), w, lam)
    out = np.zeros(mesh.N1)
    np.add.at(out, mesh.tri.ravel(), loc.ravel())
    return out


def _solve_T(A, rhs):
    return spla.spsolve(A.T.tocsc(), rhs)


def adjoint_step(o: Oracle, st, new, lam):
    """One reverse step.  st: state at t_k, new: state at t_{k+1} (forward
    outputs), lam: adjoint of the state at t_{k+1} (dict like a state).
    Returns (adjoint at t_k, {"evap": .., "gamma": ..})."""
    p = o.params
    mesh = o.mesh
    F = o.forms[0]
    tau = p["tau"]
    N1 = mesh.N1
    bnd = np.repeat(mesh.p2_boundary(), 2)
    out = {"phi": np.zeros((3, N1)), "mu": np.zeros((4, N1)), "Phi_v": np.zeros(N1),
           "v": np.zeros(2 * mesh.N2), "p": np.zeros(N1)}
    lam_phi_new = lam["phi"].copy()
    jbar = 0.0
    gbar = 0.0
    top = F.top
    ref = mesh.top_reference_node()
    loads = model.potential_loads(mesh, st["phi"], st["Phi_v"])
    f, f_v, j_out = model.ch_rhs_loads(mesh, st, p, loads, top)
    C = fem.convection_p1(mesh, st["v"])
    lw = [None] * 5                                   # adjoint weights of the load vectors

    # --- Navier-Stokes ------------------------------------------------------
    Amat, B, rhs_v, Ap, shift = model.ns_system(F, st, p)
    nv = Amat.shape[0]
    m = F.M @ np.ones(N1)
    lv = np.where(bnd, 0.0, lam["v"])
    if o.top_free:     # open top: non-singular saddle point, no pressure shift
        Kt = sp.bmat([[Amat.T, B.T], [B, None]], format="csc")
        y = spla.spsolve(Kt, np.concatenate([lv, lam["p"]]))
    else:
        lp = lam["p"] - m * lam["p"].sum() / m.sum()     # transpose of the zero-mean shift
        Kaug = sp.bmat([[Amat.T, B.T, None], [B, None, sp.csr_matrix(m[:, None])],
                        [None, sp.csr_matrix(m[None, :]), None]], format="csc")
        y = spla.spsolve(Kaug, np.concatenate([lv, lp, [0.0]]))
    yv = y[:nv]
    vf = F.velocity_forms()
    out["v"] += vf["Mv"] @ yv / tau
    kp, kv = korteweg_vjp(mesh, st["phi"], st["Phi_v"], yv, p)
    out["phi"] += kp
    out["Phi_v"] += kv
    xv = np.where(bnd, 0.0, new["v"])
    wbar, sbar = conv_p2_vjp(mesh, xv, yv)
    out["v"] -= wbar
    _, _, gl = mesh.element_geometry()
    for i in range(4):
        a = p["alpha"][i]
        loc = -a * np.einsum("ed,emd->em", sbar, gl)   # d s / d mu_i = alpha_i grad psi
        tmp = np.zeros(N1)
        np.add.at(tmp, mesh.tri.ravel(), loc.ravel())
        out["mu"][i] += tmp
    # --- air potential ------------------------------------------------------
    z = spla.spsolve(F.M.tocsc(), lam["mu"][3])
    for i in range(3):
        lam_phi_new[i] -= p["beta"][3] * (F.K @ z)
    lw[A] = z
    jbar += p["beta"][3] * (top @ z)
    # --- Allen-Cahn --------------------------------------------------------
    Aac, _ = model.ac_system(F, st, p, f_v, C, j_out)
    y = _solve_T(Aac, lam["Phi_v"])
    out["Phi_v"] += F.M @ y
    lw[V] = -tau * p["gamma_v"] * y
    out["v"] -= tau * conv_p1_vjp(mesh, new["Phi_v"], y)
    if p["ac_top_flux"]:
        jbar += tau * p["delta_v"] * (top @ y)
    # --- Cahn-Hilliard ------------------------------------------------------
    for i in range(3):
        Ach, _, _, Kk = model.ch_system(F, st, p, i, f[i], C)
        y = _solve_T(Ach, np.concatenate([lam_phi_new[i], lam["mu"][i]]))
        y1, y2 = y[:N1], y[N1:]
        g_i, b_i = p["gamma"][i], p["beta"][i]
        c = tau * g_i / b_i
        out["phi"][i] += F.M @ y1
        lw[i] = -c * y2
        if i == 2:
            jbar += c * b_i * (top @ y2)               # f_s = F_s - beta_s j t
        out["v"] -= tau * conv_p1_vjp(mesh, new["phi"][i], y1)
        mu_new = new["mu"][i]
        # d/dgamma_i of (b - A x), gamma_i = gamma (one mobility scale); the
        # first row's tau K_kappa is gamma_i times a gamma-free matrix in both
        # mobility laws
        db = -(tau / b_i) * f[i] @ y2
        dAx = (y1 @ (tau * (Kk @ mu_new)) / g_i
               + y2 @ (tau * (F.K @ new["phi"][i]) - (tau / b_i) * (F.M @ mu_new)))
        gbar += db - dAx
        if p["mobility_kind"] != 0:                    # K_kappa depends on phi_i^k
            out["phi"][i] -= tau * wstiff_vjp(mesh, st["phi"][i], g_i, mu_new, y1)
    # --- potential loads and evaporation flux ------------------------------
    lp_phi, lp_Phi = loads_vjp(mesh, st["phi"], st["Phi_v"], lw)
    out["phi"] += lp_phi
    out["Phi_v"] += lp_Phi
    evap_bar = jbar * (st["phi"][2][ref] - p["phi_s_inf"])
    out["phi"][2][ref] += jbar * p["evap_rate"]
    out["v"][bnd] = 0.0
    return out, {"evap": evap_bar, "gamma": gbar}


def objective(o: Oracle, st):
    """J = int |grad phi_p|^2 = phi_p^T K phi_p."""
    K = o.forms[0].K
    return float(st["phi"][0] @ (K @ st["phi"][0]))


def trajectory_gradient(n, params, st0, steps, checkpoint_every=0):
    """J after `steps` exact-solve steps and its gradient with respect to the
    evaporation rate, the mobility scale and the initial polymer field.
    checkpoint_every = k keeps only every k-th state and recomputes the
    others segment by segment (the gradient is identical)."""
    o = Oracle(n, params, exact=True)
    states = [st0]
    for _ in range(steps):
        states.append(o.step(states[-1])[0])
    J = objective(o, states[-1])
    keep = set(range(0, steps + 1, checkpoint_every)) if checkpoint_every else set(range(steps + 1))
    stored = {k: states[k] for k in keep}
    K = o.forms[0].K
    lam = {"phi": np.zeros_like(st0["phi"]), "mu": np.zeros_like(st0["mu"]),
           "Phi_v": np.zeros_like(st0["Phi_v"]), "v": np.zeros_like(st0["v"]), "p": np.zeros_like(st0["p"])}
    lam["phi"][0] = 2.0 * (K @ states[-1]["phi"][0])
    g_evap = g_gamma = 0.0
    k = steps
    while k > 0:
        k0 = max(c for c in stored if c < k)
        seg = [stored[k0]]
        for _ in range(k0, k):
            seg.append(o.step(seg[-1])[0])
        for kk in range(k, k0, -1):
            lam, th = adjoint_step(o, seg[kk - 1 - k0], seg[kk - k0], lam)
            g_evap += th["evap"]
            g_gamma += th["gamma"]
        k = k0
    return J, {"evap": g_evap, "gamma": g_gamma, "phi_p0": lam["phi"][0], "state0": lam}
