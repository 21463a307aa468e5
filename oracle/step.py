"""One semi-implicit step of the CH / AC / NS model (oracle; TEST
INFRASTRUCTURE).

Order of work (Sec. 3 time scheme, Sec. 4 systems, Sec. 5 air recovery):
  1. potential loads f_i^k, f_v^k and the evaporation flux j_out at t_k;
  2. CH system eqn:CH_linear for polymer, NFA and solvent, FGMRES with
     diag(MG(M + tau C), X2^{-1} M X1^{-1}) where X = tau gamma K + sqrt(tau
     gamma / beta) M is the matching factor of eqn::schurCH;
  3. AC system, FGMRES with MG(M + tau delta_v K + tau C);
  4. phi_a^{k+1} = 1 - sum phi_i^{k+1}; M mu_a = f_a^k + beta_a K phi_a^{k+1}
     by Jacobi-PCG;
  5. Oseen system eqn:linearnav, FGMRES with diag(MG(A), M_p^{-1} A_p K_p^{-1})
     (pressure convection-diffusion); pressure shifted to zero mean.
All matrices use coefficients at t_k, so 2, 3 and 5 are independent.
Every MG(.) above is one V-cycle, or with params["inner_rtol"] > 0 the
V-cycle iteration MG.solve to that relative tolerance (Sec. 5 applies its
AMG preconditioners with a tolerance of 1e-4); M_p^{-1} stays the fixed
Chebyshev iteration.  With params["amg"] = 1 the MG of the AC block is the
smoothed aggregation of oracle.amg built from the fine AC matrix of the
step (Sec. 5 takes PyAMG for this block) instead of the geometric hierarchy.

Solvent-air sub-model (params["model"] = 1, Sec. 5.1): no polymer or NFA
(their fields stay zero and their CH systems are not solved), the
Taylor-expanded Flory-Huggins density of oracle.model, and the truncation
eqn:truncateCH of the new solvent fraction to [0, 1] before phi_a^{k+1} is
formed.
"""
from __future__ import annotations

import math
import time

import numpy as np
import scipy.sparse as sp

from . import fem
from .amg import SAHierarchy
from .krylov import chebyshev, fgmres, pcg
from .mesh import Mesh
from .mg import (MG, VEL_LO_RATIO, VEL_SMOOTH_DEGREE, inject_p1, inject_velocity, level_sizes, prolongation_p1,
                 prolongation_velocity)
from .model import (Forms, ac_system, ch_rhs_loads, ch_system, free_energy, mobility_at, ns_shift, ns_system,
                    potential_loads)

MASS_CHEB_DEGREE = 5
MASS_CHEB_BOUNDS = (0.5, 2.0)      # spectrum of D^{-1} M for P1 triangles (Wathen)


def _direct(A, b):
    """Sparse LU solve (used by the exact-solve mode of the oracle)."""
    import scipy.sparse.linalg as spla
    x = spla.spsolve(A.tocsc(), b)
    r = float(np.linalg.norm(b - A @ x))
    nb = float(np.linalg.norm(b))
    return x, {"iters": 0, "rel_residual": r / nb if nb else 0.0, "converged": True}


class Oracle:
    """exact=True replaces every Krylov solve by a sparse LU solve of the same
    system (finite-difference and adjoint checks need solves free of the
    stopping-rule error)."""

    def __init__(self, n: int, params: dict, lx: float = 1.0, ly: float = 1.0, exact: bool = False):
        self.exact = exact
        self.params = dict(params)
        self.sizes = level_sizes(n)
        self.top_free = self.params.get("top_bc", 0) == 1
        self.meshes = [Mesh(s, lx, ly, self.top_free) for s in self.sizes]
        self.forms = [Forms(m, self.params) for m in self.meshes]
        self.P1 = [prolongation_p1(self.meshes[l + 1]) for l in range(len(self.sizes) - 1)]
        self._Pv = None
        self._Kp = None

    @property
    def mesh(self) -> Mesh:
        return self.meshes[0]

    def Pv(self):
        if self._Pv is None:
            self._Pv = [prolongation_velocity(self.meshes[l + 1], self.meshes[l])
                        for l in range(len(self.sizes) - 1)]
        return self._Pv

    # ------------------------------------------------------------------
    def level_fields(self, state):
        """Velocity, potentials and phase fields injected to every level."""
        vs, mus, phis = [state["v"]], [state["mu"]], [state["phi"]]
        for l in range(len(self.sizes) - 1):
            nf = self.sizes[l]
            vs.append(inject_velocity(vs[-1], nf))
            mus.append(np.stack([inject_p1(m, nf) for m in mus[-1]]))
            phis.append(np.stack([inject_p1(f, nf) for f in phis[-1]]))
        return vs, mus, phis

    def level_states(self, state):
        vs, mus, phis = self.level_fields(state)
        return [{"v": vs[l], "mu": mus[l], "phi": phis[l]} for l in range(len(vs))]

    # ------------------------------------------------------------------
    def ch_preconditioner(self, species, lstates, convs):
        p = self.params
        tau, g, b = p["tau"], p["gamma"][species], p["beta"][species]
        a = math.sqrt(tau * g / b)
        L = [(f.M + tau * C).tocsr() for f, C in zip(self.forms, convs)]
        X1 = [(tau * g * f.K + a * f.M).tocsr() for f in self.forms]
        mgL = MG(L, self.P1)
        mgX1 = MG(X1, self.P1)
        if p["mobility_kind"] == 0:
            mgX2 = mgX1
        else:
            X2 = [(tau * fem.weighted_stiffness_p1(
                f.mesh, mobility_at(f.mesh, st["phi"][species], p, species)) + a * f.M).tocsr()
                for f, st in zip(self.forms, lstates)]
            mgX2 = MG(X2, self.P1)
        M = self.forms[0].M
        N = self.mesh.N1
        iL, iX1, iX2 = mgL.inner(p), mgX1.inner(p), mgX2.inner(p)

        def apply(r):
            z = np.empty_like(r)
            z[:N] = iL(r[:N])
            z[N:] = iX2(M @ iX1(r[N:]))
            return z
        return apply

    def solve_ch(self, state, species, f_i, lstates, convs):
        p = self.params
        A, rhs, _, _ = ch_system(self.forms[0], state, p, species, f_i, convs[0])
        if self.exact:
            x, info = _direct(A, rhs)
        else:
            prec = self.ch_preconditioner(species, lstates, convs)
            x, info = fgmres(lambda y: A @ y, prec, rhs, p["rtol"], p["atol"], p["restart"], p["maxit"])
        N = self.mesh.N1
        return x[:N], x[N:], info, (A, rhs)

    def solve_ac(self, state, f_v, j_out, convs):
        p = self.params
        A, rhs = ac_system(self.forms[0], state, p, f_v, convs[0], j_out)
        tau = p["tau"]
        if self.exact:
            x, info = _direct(A, rhs)
            return x, info, (A, rhs)
        mats = [(f.M + tau * p["delta_v"] * f.K + tau * C).tocsr() for f, C in zip(self.forms, convs)]
        if p.get("amg", 0) == 1:     # Sec. 5: algebraic multigrid of this block (oracle.amg)
            mg = SAHierarchy(mats[0]).mg
        else:
            mg = MG(mats, self.P1)
        x, info = fgmres(lambda y: A @ y, mg.inner(p), rhs, p["rtol"], p["atol"], p["restart"], p["maxit"])
        return x, info, (A, rhs)

    def solve_mu_a(self, f_a, phi_new):
        p = self.params
        F = self.forms[0]
        phi_a = 1.0 - phi_new[0] - phi_new[1] - phi_new[2]
        rhs = f_a + p["beta"][3] * (F.K @ phi_a)
        if self.exact:
            return _direct(F.M, rhs)
        x, info = pcg(F.M, rhs, 1.0 / F.M.diagonal(), rtol=1e-12)
        return x, info

    def ns_operator(self, A, B):
        nv = A.shape[0]

        def apply(y):
            out = np.empty_like(y)
            out[:nv] = A @ y[:nv] + B.T @ y[nv:]
            out[nv:] = B @ y[:nv]
            return out
        return apply

    def ns_preconditioner(self, A, Ap, lstates):
        p = self.params
        tau = p["tau"]
        mats = [A]
        for l in range(1, len(self.sizes)):
            f, st = self.forms[l], lstates[l]
            vf = f.velocity_forms()
            shift = ns_shift(f.mesh, st, p)
            J2 = fem.convection_p2(f.mesh, st["v"], shift)
            Al = vf["Mv"] / tau + sp.kron(J2, sp.eye(2), format="csr") + vf["Ksym"]
            mats.append(fem.velocity_dirichlet(Al.tocsr(), vf["bnd"]))
        mgA = MG(mats, self.Pv(), degree=VEL_SMOOTH_DEGREE, ratio=VEL_LO_RATIO)
        if self._Kp is None:
            if self.top_free:        # outflow: K_p with Dirichlet rows on the open top, non-singular
                self._Kp = MG([fem.p1_dirichlet(f.K, f.mesh.p1_top()) for f in self.forms], self.P1,
                              dense_coarse=True)
            else:
                self._Kp = MG([f.K for f in self.forms], self.P1, singular=True, dense_coarse=True)
        mgK = self._Kp
        iA, iK = mgA.inner(p), mgK.inner(p)
        Mp = self.forms[0].M
        mdinv = 1.0 / Mp.diagonal()
        lo, hi = MASS_CHEB_BOUNDS
        nv = A.shape[0]

        def apply(r):
            z = np.empty_like(r)
            z[:nv] = iA(r[:nv])
            t = Ap @ iK(r[nv:])
            z[nv:] = chebyshev(lambda y: Mp @ y, mdinv, t, None, lo, hi, MASS_CHEB_DEGREE)
            return z
        return apply

    def solve_ns(self, state, lstates):
        p = self.params
        A, B, rhs_v, Ap, _ = ns_system(self.forms[0], state, p)
        nv = A.shape[0]
        rhs = np.concatenate([rhs_v, np.zeros(self.mesh.N1)])
        if self.exact and self.top_free:
            x, info = _direct(sp.bmat([[A, B.T], [B, None]], format="csc"), rhs)
        elif self.exact:
            m = self.forms[0].M @ np.ones(self.mesh.N1)
            K = sp.bmat([[A, B.T, None], [B, None, sp.csr_matrix(m[:, None])],
                         [None, sp.csr_matrix(m[None, :]), None]], format="csc")
            x, info = _direct(K, np.concatenate([rhs, [0.0]]))
            x = x[:-1]
        else:
            prec = self.ns_preconditioner(A, Ap, lstates)
            # Sec. 5 stops the Oseen solve at tolerances of its own (ns_rtol > 0)
            rt, at = (p["ns_rtol"], p["ns_atol"]) if p.get("ns_rtol", 0.0) > 0 else (p["rtol"], p["atol"])
            x, info = fgmres(self.ns_operator(A, B), prec, rhs, rt, at, p["restart"], p["maxit"])
        v, pr = x[:nv], x[nv:]
        if not self.top_free:       # enclosed flow: pressure in L^2_0
            Mp = self.forms[0].M
            one = np.ones(self.mesh.N1)
            pr = pr - (one @ (Mp @ pr)) / (one @ (Mp @ one))
        return v, pr, info, (A, B, rhs)

    # ------------------------------------------------------------------
    def step(self, state, keep_systems=False):
        t0 = time.perf_counter()
        p = self.params
        mesh = self.mesh
        lstates = self.level_states(state)
        convs = [fem.convection_p1(f.mesh, st["v"]) for f, st in zip(self.forms, lstates)]
        loads = potential_loads(mesh, state["phi"], state["Phi_v"], p)
        f, f_v, j_out = ch_rhs_loads(mesh, state, p, loads, self.forms[0].top)
        new = {"phi": np.empty_like(state["phi"]), "mu": np.empty_like(state["mu"])}
        info, systems = {}, {}
        solvent_air = p.get("model", 0) == 1
        for i, name in enumerate(("ch_p", "ch_N", "ch_s")):
            if solvent_air and i < 2:
                new["phi"][i] = 0.0
                new["mu"][i] = 0.0
                info[name] = {"iters": 0, "rel_residual": 0.0, "converged": True}
                continue
            new["phi"][i], new["mu"][i], info[name], systems[name] = self.solve_ch(state, i, f[i], lstates, convs)
        if solvent_air:
            new["phi"][2] = np.clip(new["phi"][2], 0.0, 1.0)      # eqn:truncateCH
        new["Phi_v"], info["ac"], systems["ac"] = self.solve_ac(state, f_v, j_out, convs)
        new["mu"][3], info["mu_a"] = self.solve_mu_a(f[3], new["phi"])
        new["v"], new["p"], info["ns"], systems["ns"] = self.solve_ns(state, lstates)
        info["seconds"] = time.perf_counter() - t0
        info["j_out"] = j_out
        if keep_systems:
            info["systems"] = systems
        return new, info

    def diagnostics(self, state):
        """FP64 mass sums 1^T M phi_i (i = p, N, s, and the air fraction
        phi_a = 1 - sum phi), ||B v|| (discrete divergence), int p (Sec. 3,
        L^2_0 pressure) and the discrete energy (model.free_energy: local
        and gradient parts of the Sec. 2.2 free energy, kinetic energy)."""
        F = self.forms[0]
        vf = F.velocity_forms()
        one = np.ones(self.mesh.N1)
        phi_a = 1.0 - state["phi"][0] - state["phi"][1] - state["phi"][2]
        e = free_energy(F, state, self.params)
        return {
            "mass": [float(one @ (F.M @ state["phi"][i])) for i in range(3)],
            "mass_a": float(one @ (F.M @ phi_a)),
            "div": float(np.linalg.norm(vf["B"] @ state["v"])),
            "p_mean": float(one @ (F.M @ state["p"])),
            "energy": e["local"] + e["gradient"] + e["kinetic"],
            "energy_parts": e,
        }
