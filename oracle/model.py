"""Potential, right-hand sides and linear systems of one step (oracle; TEST
INFRASTRUCTURE).

Potential: the polynomial fit eqn:appPotential,
  f = (1 - p(Phi)) (3.5 phi_p^2 phi_N^2 + 0.3 phi_s^2 + 0.3 phi_a^2 - 10 phi_s phi_a)
    + p(Phi) (3.5 phi_p^2 + 3.5 phi_N^2 + 2 phi_s^2 + 0.1 phi_a^2),
  p(Phi) = Phi^2 (3 - 2 Phi)   (Sec. 2.2),
with partial derivatives taken before phi_a = 1 - phi_p - phi_N - phi_s is
substituted (Sec. 5 keeps mu_a as a separate field).

Solvent-air sub-model (Sec. 5.1, params["model"] = 1): only solvent and air,
the Flory-Huggins density of Sec. 2.2 with the polymer and NFA terms removed,
  f_liq = g(phi_s) / N_s + g(phi_a) / N_a + chi_sa phi_s phi_a,
  f_gas = g(phi_s) - phi_s ln phi_sat(s) + g(phi_a) - phi_a ln phi_sat(a),
where every phi ln phi is replaced by its Taylor polynomial g of degree 4 at
phi = 1/2 (Sec. 5), RT / V_0 = 1, and the same interpolation p(Phi).

Systems (Sec. 4):
  CH  eqn:CH_linear   [[M + tau C, tau K_gamma], [tau gamma K, -(tau gamma / beta) M]]
  AC                  (M + tau delta_v K + tau C) Phi = M Phi^k - tau gamma_v f_v^k
  NS  eqn:linearnav   [[A, B^T], [B, 0]],  A = (rho/tau) M + J + K_sym
All coefficients are taken at t_k (semi-implicit scheme, Sec. 3).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .mesh import Mesh
from .quadrature import triangle_rule

SPECIES = ("p", "N", "s", "a")


def interp_p(Phi):
    """p(Phi) = Phi^2 (3 - 2 Phi) (Sec. 2.2)."""
    return Phi * Phi * (3.0 - 2.0 * Phi)


def dinterp_p(Phi):
    return 6.0 * Phi * (1.0 - Phi)


def f_liquid(pp, pn, ps, pa):
    return 3.5 * pp**2 * pn**2 + 0.3 * ps**2 + 0.3 * pa**2 - 10.0 * ps * pa


def f_gas(pp, pn, ps, pa):
    return 3.5 * pp**2 + 3.5 * pn**2 + 2.0 * ps**2 + 0.1 * pa**2


# Taylor polynomial of x ln x at x = 1/2 to 4th order (Sec. 5):
# derivatives of x ln x at 1/2: value -ln2/2, then 1 - ln 2, 1/x = 2,
# -1/x^2 = -4, 2/x^3 = 16, divided by k!.
TAYLOR_XLNX = (-0.5 * np.log(2.0), 1.0 - np.log(2.0), 1.0, -2.0 / 3.0, 2.0 / 3.0)


def taylor_xlnx(x):
    d = x - 0.5
    c = TAYLOR_XLNX
    return c[0] + d * (c[1] + d * (c[2] + d * (c[3] + d * c[4])))


def dtaylor_xlnx(x):
    d = x - 0.5
    c = TAYLOR_XLNX
    return c[1] + d * (2.0 * c[2] + d * (3.0 * c[3] + d * 4.0 * c[4]))


def fh_liquid(ps, pa, prm):
    return taylor_xlnx(ps) / prm["n_s"] + taylor_xlnx(pa) / prm["n_a"] + prm["chi_sa"] * ps * pa


def fh_gas(ps, pa, prm):
    return (taylor_xlnx(ps) - ps * np.log(prm["phi_sat_s"]) + taylor_xlnx(pa) - pa * np.log(prm["phi_sat_a"]))


def fh_partials(ps, pa, Phi, prm):
    """(df/dphi_s, df/dphi_a, df/dPhi_v) of the solvent-air density."""
    q = interp_p(Phi)
    dq = dinterp_p(Phi)
    gs, ga = dtaylor_xlnx(ps), dtaylor_xlnx(pa)
    d_s = (1 - q) * (gs / prm["n_s"] + prm["chi_sa"] * pa) + q * (gs - np.log(prm["phi_sat_s"]))
    d_a = (1 - q) * (ga / prm["n_a"] + prm["chi_sa"] * ps) + q * (ga - np.log(prm["phi_sat_a"]))
    d_v = dq * (fh_gas(ps, pa, prm) - fh_liquid(ps, pa, prm))
    return d_s, d_a, d_v


def potential(pp, pn, ps, pa, Phi):
    """f of eqn:appPotential."""
    q = interp_p(Phi)
    return (1 - q) * f_liquid(pp, pn, ps, pa) + q * f_gas(pp, pn, ps, pa)


def free_energy(forms: Forms, state, params):
    """Parts of the discrete energy of a state (Sec. 2.2 free energy in its
    dimensionless form, beta_i and beta_v in place of eps_i^2 and lambda^2,
    plus the kinetic energy of the flow with rho = 1):
      local:    int f(phi_h, Phi_h) dx, f of eqn:appPotential (or the
                solvent-air density of Sec. 5.1), phi_a = 1 - sum phi;
                degree-7 integrand, exact rule;
      gradient: sum_i beta_i / 2 int |grad phi_i|^2 + beta_v / 2 int |grad Phi_v|^2
                = sum_i beta_i / 2 phi_i^T K phi_i + beta_v / 2 Phi^T K Phi;
      kinetic:  1/2 int |v_h|^2 dx = 1/2 v^T M_v v."""
    mesh = forms.mesh
    phi, Phi = state["phi"], state["Phi_v"]
    lam, w = triangle_rule(7)
    _, area, _ = mesh.element_geometry()
    pp, pn, ps = (fem.p1_field_at(mesh, phi[i], lam) for i in range(3))
    pa = 1.0 - pp - pn - ps
    Ph = fem.p1_field_at(mesh, Phi, lam)
    if params.get("model", 0) == 1:
        q = interp_p(Ph)
        fq = (1 - q) * fh_liquid(ps, pa, params) + q * fh_gas(ps, pa, params)
    else:
        fq = potential(pp, pn, ps, pa, Ph)
    local = float(np.sum(area[:, None] * w[None] * fq))
    K = forms.K
    fields = [phi[0], phi[1], phi[2], 1.0 - phi[0] - phi[1] - phi[2]]
    grad = sum(0.5 * params["beta"][i] * float(fields[i] @ (K @ fields[i])) for i in range(4))
    grad += 0.5 * params["beta_v"] * float(Phi @ (K @ Phi))
    v = state["v"]
    kinetic = 0.5 * float(v @ (forms.velocity_forms()["Mv"] @ v))
    return {"local": local, "gradient": grad, "kinetic": kinetic}


def potential_partials(pp, pn, ps, pa, Phi):
    """(df/dphi_p, df/dphi_N, df/dphi_s, df/dphi_a, df/dPhi_v) of
    eqn:appPotential, un-reduced partials."""
    q = interp_p(Phi)
    dq = dinterp_p(Phi)
    d_p = (1 - q) * 7.0 * pp * pn**2 + q * 7.0 * pp
    d_n = (1 - q) * 7.0 * pp**2 * pn + q * 7.0 * pn
    d_s = (1 - q) * (0.6 * ps - 10.0 * pa) + q * 4.0 * ps
    d_a = (1 - q) * (0.6 * pa - 10.0 * ps) + q * 0.2 * pa
    d_v = dq * (f_gas(pp, pn, ps, pa) - f_liquid(pp, pn, ps, pa))
    return d_p, d_n, d_s, d_a, d_v


def potential_loads(mesh: Mesh, phi, Phi, params=None):
    """Load vectors int df/dphi_i psi_m (i = p, N, s, a) and int df/dPhi psi_m
    with phi_a = 1 - sum phi (Sec. 5).  Integrand degree 7 in P1 fields.
    Solvent-air model: the polymer and NFA loads are zero."""
    solvent_air = params is not None and params.get("model", 0) == 1
    out = []
    for k in range(5):
        if solvent_air and k < 2:
            out.append(np.zeros(mesh.N1))
            continue

        def integrand(lam, k=k):
            pp = fem.p1_field_at(mesh, phi[0], lam)
            pn = fem.p1_field_at(mesh, phi[1], lam)
            ps = fem.p1_field_at(mesh, phi[2], lam)
            pa = 1.0 - pp - pn - ps
            Ph = fem.p1_field_at(mesh, Phi, lam)
            if solvent_air:
                return fh_partials(ps, pa, Ph, params)[k - 2]
            return potential_partials(pp, pn, ps, pa, Ph)[k]
        out.append(fem.load_p1(mesh, integrand, 7))
    return out


def evaporation_flux(mesh: Mesh, phi_s, params):
    """j_out = evap_rate (phi_s^vap - phi_s^inf), phi_s^vap = phi_s at the top
    reference point (Sec. 2.1; the Hertz-Knudsen constants are lumped into
    evap_rate)."""
    return params["evap_rate"] * (phi_s[mesh.top_reference_node()] - params["phi_s_inf"])


def ch_rhs_loads(mesh: Mesh, state, params, loads=None, top=None):
    """f_i^k (i = p, N, s, a) of eqn:airdisc: int df/dphi_i w - beta_i int_Gt
    (d phi_i/dn) w, with d phi_s/dn = j_out and d phi_a/dn = -j_out (eqn:bc)."""
    if loads is None:
        loads = potential_loads(mesh, state["phi"], state["Phi_v"], params)
    if top is None:
        top = fem.top_load_p1(mesh)
    j = evaporation_flux(mesh, state["phi"][2], params)
    beta = params["beta"]
    f = [loads[0].copy(), loads[1].copy(),
         loads[2] - beta[2] * j * top,
         loads[3] + beta[3] * j * top]
    return f, loads[4], j


# ----------------------------------------------------------------------------
def mobility_at(mesh: Mesh, phi_i, params, species: int):
    """Mobility kappa(x) at quadrature points: gamma_i (constant mobility,
    Sec. 2.3) or gamma_i (phi_i (1 - phi_i) + m0) (concentration-dependent
    mobility, lagged at t_k)."""
    g = params["gamma"][species]
    if params["mobility_kind"] == 0:
        return lambda lam: np.full((mesh.E, lam.shape[0]), g)
    m0 = params["mobility_m0"]

    def kap(lam):
        ph = fem.p1_field_at(mesh, phi_i, lam)
        return g * (ph * (1.0 - ph) + m0)
    return kap


class Forms:
    """Matrices of one mesh that do not depend on the state."""

    def __init__(self, mesh: Mesh, params):
        self.mesh = mesh
        self.M = fem.mass_p1(mesh)
        self.K = fem.stiffness_p1(mesh)
        self.top = fem.top_load_p1(mesh)
        self._vel = None
        self.params = params

    def velocity_forms(self):
        if self._vel is None:
            mesh = self.mesh
            bnd = mesh.p2_boundary()
            M2 = fem.mass_p2(mesh)
            Mv = sp.kron(M2, sp.eye(2), format="csr")
            Ks = fem.ksym(mesh, self.params["eta"])
            B = fem.zero_velocity_columns(fem.divergence(mesh), bnd)
            self._vel = {"bnd": bnd, "M2": M2, "Mv": Mv, "Ksym": Ks, "B": B}
        return self._vel


def ch_system(forms: Forms, state, params, species: int, f_i, C):
    """Matrix and right-hand side of eqn:CH_linear for one species.
    Row 2 is scaled by -tau gamma_i / beta_i as in the paper."""
    mesh = forms.mesh
    tau, g, b = params["tau"], params["gamma"][species], params["beta"][species]
    L = (forms.M + tau * C).tocsr()
    if params["mobility_kind"] == 0:
        Kk = g * forms.K
    else:
        Kk = fem.weighted_stiffness_p1(mesh, mobility_at(mesh, state["phi"][species], params, species))
    c = tau * g / b
    A = sp.bmat([[L, tau * Kk], [tau * g * forms.K, -c * forms.M]], format="csr")
    rhs = np.concatenate([forms.M @ state["phi"][species], -c * f_i])
    return A, rhs, L, Kk


def ac_system(forms: Forms, state, params, f_v, C, j_out):
    """(M + tau delta_v K + tau C) Phi^{k+1} = M Phi^k - tau gamma_v f_v^k
    (Sec. 4), plus, when ac_top_flux is set, the boundary term
    tau delta_v j_out int_Gt q of a flux delta_v dPhi/dn = delta_v j_out on the
    top boundary."""
    tau = params["tau"]
    A = (forms.M + tau * params["delta_v"] * forms.K + tau * C).tocsr()
    rhs = forms.M @ state["Phi_v"] - tau * params["gamma_v"] * f_v
    if params["ac_top_flux"]:
        rhs = rhs + tau * params["delta_v"] * j_out * forms.top
    return A, rhs


def ns_shift(mesh: Mesh, state, params):
    """Per-element constant sum_i alpha_i grad mu_i^k (eqn:matrixns w)."""
    g = np.zeros((mesh.E, 2))
    for i in range(4):
        g += params["alpha"][i] * fem.p1_gradient(mesh, state["mu"][i])
    return g


def korteweg_tensor(mesh: Mesh, state, params):
    """G = sum_i beta_i grad phi_i (x) grad phi_i + beta_v grad Phi (x) grad Phi
    (Sec. 3), phi_a = 1 - sum phi, per element."""
    phi = state["phi"]
    grads = [fem.p1_gradient(mesh, phi[i]) for i in range(3)]
    grads.append(-(grads[0] + grads[1] + grads[2]))
    Gt = np.zeros((mesh.E, 2, 2))
    for i in range(4):
        Gt += params["beta"][i] * np.einsum("ec,ed->ecd", grads[i], grads[i])
    gv = fem.p1_gradient(mesh, state["Phi_v"])
    Gt += params["beta_v"] * np.einsum("ec,ed->ecd", gv, gv)
    return Gt


def ns_system(forms: Forms, state, params):
    """Blocks and right-hand side of eqn:linearnav with rho = 1 (equal pure
    densities), no-slip velocity on the whole boundary (eqn:bc) or, on a
    top_free mesh, on the bottom and side walls with the do-nothing
    condition (2 eta eps(v) - p I) n = 0 on the top (natural in the weak
    form)."""
    mesh = forms.mesh
    vf = forms.velocity_forms()
    tau = params["tau"]
    shift = ns_shift(mesh, state, params)
    J2 = fem.convection_p2(mesh, state["v"], shift)
    A = vf["Mv"] / tau + sp.kron(J2, sp.eye(2), format="csr") + vf["Ksym"]
    A = fem.velocity_dirichlet(A.tocsr(), vf["bnd"])
    G = fem.korteweg(mesh, korteweg_tensor(mesh, state, params))
    rhs_v = vf["Mv"] @ state["v"] / tau + G
    rhs_v[np.repeat(vf["bnd"], 2)] = 0.0
    B = vf["B"]
    Ap = (forms.M / tau + params["eta"] * forms.K + fem.convection_p1(mesh, state["v"], shift)).tocsr()
    if mesh.top_free:
        Ap = fem.p1_dirichlet(Ap, mesh.p1_top())       # PCD outflow condition on the open top
    return A, B, rhs_v, Ap, shift
