"""Step-level pins of the oracle: discrete mass conservation, divergence-free
velocity, agreement with sparse direct solves, energy decay in the
flow-free single-species case (CPU only)."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, model
from oracle.krylov import fgmres
from oracle.mesh import Mesh
from oracle.step import Oracle
from paper_2501_11767_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_sequence():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    keys = np.array([int(r[0]) for r in rows], dtype=np.uint64)
    out = inputs.splitmix64(keys)
    assert [format(int(v), "016x") for v in out] == [r[1] for r in rows]
    u = inputs.uniform_noise(7, 1, 100000)
    assert u.min() >= -0.01 and u.max() < 0.01 and abs(u.mean()) < 1e-4


@pytest.fixture(scope="module")
def two_steps():
    n = 16
    p = inputs.default_params()
    o = Oracle(n, p)
    s0 = inputs.initial_state(n, seed=3)
    s1, i1 = o.step(s0)
    s2, i2 = o.step(s1, keep_systems=True)
    return o, (s0, s1, s2), (i1, i2)


def test_all_solves_converge(two_steps):
    _, _, infos = two_steps
    for info in infos:
        for k in ("ch_p", "ch_N", "ch_s", "ac", "ns", "mu_a"):
            assert info[k]["converged"], (k, info[k])


def test_mass_conservation(two_steps):
    """1^T M phi_i^{k+1} = 1^T M phi_i^k: 1^T K = 0 and 1^T C(v) phi = -int phi
    div v = 0 for the discretely divergence-free v^k (P1 pressure space)."""
    o, states, _ = two_steps
    mass = [o.diagnostics(s)["mass"] for s in states]
    assert np.max(np.abs(states[1]["v"])) > 0          # the second step has flow
    for k in range(2):
        for i in range(3):
            assert abs(mass[k + 1][i] - mass[k][i]) <= 1e-8 * mass[k][i]


def test_divergence_free_and_mean_zero_pressure(two_steps):
    o, states, infos = two_steps
    A, B, rhs = infos[1]["systems"]["ns"]
    for s in states[1:]:
        d = o.diagnostics(s)
        assert d["div"] <= 1e-8 * np.linalg.norm(rhs)
        assert abs(d["p_mean"]) < 1e-14


def test_evaporation_flux_raises_vapour_at_top(two_steps):
    o, states, infos = two_steps
    assert infos[0]["j_out"] > 0
    top = o.mesh.p1_top()
    assert states[1]["Phi_v"][top].mean() > 0
    assert states[1]["Phi_v"][top].mean() > 10 * abs(states[1]["Phi_v"][~top]).mean()


def test_solves_agree_with_sparse_direct():
    """Each Krylov solution of a step, at rtol 1e-12, agrees with a sparse LU
    solve of the same system (dense-LU pin of the solver path)."""
    n = 8
    p = inputs.default_params()
    p["rtol"] = 1e-12
    o = Oracle(n, p)
    s0 = inputs.initial_state(n, seed=1)
    s1, _ = o.step(s0)
    s2, info = o.step(s1, keep_systems=True)
    N = o.mesh.N1
    for name, i in (("ch_p", 0), ("ch_N", 1), ("ch_s", 2)):
        A, rhs = info["systems"][name]
        x = spla.spsolve(A.tocsc(), rhs)
        got = np.concatenate([s2["phi"][i], s2["mu"][i]])
        assert np.linalg.norm(got - x) <= 1e-9 * np.linalg.norm(x)
    A, rhs = info["systems"]["ac"]
    x = spla.spsolve(A.tocsc(), rhs)
    assert np.linalg.norm(s2["Phi_v"] - x) <= 1e-9 * np.linalg.norm(x)
    A, B, rhs = info["systems"]["ns"]
    m = o.forms[0].M @ np.ones(N)
    K = sp.bmat([[A, B.T, None], [B, None, sp.csr_matrix(m[:, None])],
                 [None, sp.csr_matrix(m[None, :]), None]], format="csc")
    sol = spla.spsolve(K, np.concatenate([rhs, [0.0]]))
    nv = A.shape[0]
    assert np.linalg.norm(s2["v"] - sol[:nv]) <= 1e-9 * np.linalg.norm(sol[:nv])
    assert np.linalg.norm(s2["p"] - sol[nv:nv + N]) <= 1e-8 * np.linalg.norm(sol[nv:nv + N])
    # mu_a from the mass solve
    F = o.forms[0]
    phi_a = 1 - s2["phi"].sum(axis=0)
    f, _, _ = model.ch_rhs_loads(o.mesh, s1, p)
    mu_a = spla.spsolve(F.M.tocsc(), f[3] + p["beta"][3] * (F.K @ phi_a))
    assert np.linalg.norm(s2["mu"][3] - mu_a) <= 1e-10 * np.linalg.norm(mu_a)


def test_energy_decay_single_species_without_flow():
    """Special case: one CH field with the double-well F = (phi^2 - 1)^2 / 4,
    v = 0, no evaporation, small tau: the discrete energy
    int F(phi) + beta/2 |grad phi|^2 decreases monotonically."""
    n = 24
    mesh = Mesh(n)
    p = inputs.default_params()
    beta, tau = 1e-3, 1e-5
    p.update(beta=[beta] * 4, tau=tau, rtol=1e-11)
    forms = model.Forms(mesh, p)
    o = Oracle(n, p)
    st = inputs.initial_state(n, seed=5)
    phi = 0.5 * (st["phi"][0] - 0.3) / 0.01 * 0.05           # noise in [-0.05, 0.05]
    C = fem.convection_p1(mesh, st["v"])
    lstates = o.level_states(st)
    convs = [fem.convection_p1(f.mesh, s["v"]) for f, s in zip(o.forms, lstates)]
    prec = o.ch_preconditioner(0, lstates, convs)

    def energy(u):
        Fq = fem.load_p1(mesh, lambda lam: 0.25 * (fem.p1_field_at(mesh, u, lam) ** 2 - 1) ** 2, 8)
        return Fq.sum() + 0.5 * beta * u @ (forms.K @ u)
    E = [energy(phi)]
    for _ in range(15):
        f = fem.load_p1(mesh, lambda lam: fem.p1_field_at(mesh, phi, lam) ** 3 - fem.p1_field_at(mesh, phi, lam), 8)
        st["phi"][0] = phi
        A, rhs, _, _ = model.ch_system(forms, st, p, 0, f, C)
        x, info = fgmres(lambda y: A @ y, prec, rhs, p["rtol"], 0.0, 30, 600)
        assert info["converged"]
        phi = x[:mesh.N1]
        E.append(energy(phi))
    E = np.array(E)
    assert np.all(np.diff(E) < 0), E


def _trajectory(params, n=32, steps=8):
    o = Oracle(n, params)
    st = inputs.initial_state(n, seed=0)
    out = []
    for _ in range(steps):
        st, info = o.step(st)
        out.append((float(np.abs(st["v"]).max()), float(np.abs(st["phi"][0] - 0.3).max()),
                    all(info[k]["converged"] for k in ("ch_p", "ch_N", "ch_s", "ac", "ns"))))
    return out


def test_benchmark_parameter_reading_is_stable():
    """The 1024^2 benchmark's parameters (tau = 5e-4, eps = 0.005 read as the
    polymer / NFA gradient-energy coefficient, beta_s = 0.1, beta_a = 1) give
    a bounded trajectory of the semi-implicit scheme."""
    p = inputs.workload("film1024_mixed")["params"]
    traj = _trajectory(dict(p, precision=0))
    assert all(ok for _, _, ok in traj)
    assert max(v for v, _, _ in traj) < 0.1
    assert max(d for _, d, _ in traj) < 0.05


def test_all_species_eps_squared_reading_is_unstable():
    """beta_i = eps^2 for every species violates tau gamma lambda^2 < 8 beta
    for the solvent (lambda ~ 10.6) and the trajectory blows up within a few
    steps: the reason the benchmark does not use that reading."""
    p = dict(inputs.workload("film1024_mixed")["params"], precision=0, beta=[0.005 ** 2] * 4)
    traj = _trajectory(p, steps=5)
    assert traj[-1][0] > 1.0 or not traj[-1][2]
