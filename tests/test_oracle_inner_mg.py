"""Pins of the oracle's multigrid used as an inner solver with a tolerance
(Sec. 5: the block preconditioners apply their AMG to a relative tolerance of
1e-4).  MG.solve is the V-cycle iteration x <- x + V(b - A x) from x = 0;
these checks tie it to a sparse direct solve, to its own stopping rule and to
the single V-cycle it reduces to (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem
from oracle.mesh import Mesh
from oracle.mg import MG, VEL_LO_RATIO, VEL_SMOOTH_DEGREE, level_sizes, prolongation_p1, prolongation_velocity
from oracle.step import Oracle
from paper_2501_11767_gb300 import inputs


def _hier(n):
    sizes = level_sizes(n)
    meshes = [Mesh(s) for s in sizes]
    P1 = [prolongation_p1(meshes[l + 1]) for l in range(len(sizes) - 1)]
    return meshes, P1


def _conv_diff(meshes, tau=1e-2, seed=0):
    """M + tau K + tau C(v) on every level, v a smooth rotating field."""
    out = []
    for m in meshes:
        X, Y = m.x2[:, 0], m.x2[:, 1]
        v = np.stack([np.sin(np.pi * Y), -np.sin(np.pi * X)], axis=1).ravel()
        out.append((fem.mass_p1(m) + tau * fem.stiffness_p1(m) + tau * fem.convection_p1(m, v)).tocsr())
    return out


def test_one_cycle_cap_is_one_vcycle():
    meshes, P1 = _hier(16)
    mats = _conv_diff(meshes)
    mg = MG(mats, P1)
    b = np.random.default_rng(0).standard_normal(mats[0].shape[0])
    x, cycles = mg.solve(b, 1e-4, 1)
    assert cycles == 1
    assert np.array_equal(x, mg(b))
    # a zero tolerance on a zero right-hand side stops after the first cycle
    x0, c0 = mg.solve(np.zeros_like(b), 1e-4, 20)
    assert c0 == 1 and not np.any(x0)


@pytest.mark.parametrize("n", [8, 32])
def test_converges_to_the_direct_solve(n):
    """Nonsymmetric convection-diffusion: at a tight tolerance the iteration
    reaches the sparse LU solution."""
    meshes, P1 = _hier(n)
    mats = _conv_diff(meshes)
    mg = MG(mats, P1)
    b = np.random.default_rng(n).standard_normal(mats[0].shape[0])
    x, cycles = mg.solve(b, 1e-13, 200)
    ref = spla.spsolve(mats[0].tocsc(), b)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)
    assert cycles < 60


def test_stopping_rule_is_minimal():
    """The returned cycle count is the first at which ||b - A x|| <= rtol ||b||."""
    meshes, P1 = _hier(32)
    mats = _conv_diff(meshes)
    mg = MG(mats, P1)
    A = mats[0]
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    nb = np.linalg.norm(b)
    for rtol in (1e-2, 1e-4, 1e-6):
        x, k = mg.solve(b, rtol, 100)
        assert np.linalg.norm(b - A @ x) <= rtol * nb
        if k > 1:
            xp, kp = mg.solve(b, rtol, k - 1)
            assert kp == k - 1
            assert np.linalg.norm(b - A @ xp) > rtol * nb


def test_contraction_independent_of_mesh():
    """The V-cycle contracts the residual of the SPD matching factor by a
    factor that does not grow with n (geometric MG, P10)."""
    rates = []
    for n in (16, 32, 64):
        meshes, P1 = _hier(n)
        mats = [(1e-3 * fem.stiffness_p1(m) + 0.05 * fem.mass_p1(m)).tocsr() for m in meshes]
        mg = MG(mats, P1)
        A = mats[0]
        b = np.random.default_rng(n).standard_normal(A.shape[0])
        r_prev = None
        ratios = []
        for k in range(1, 6):
            x, _ = mg.solve(b, 0.0, k)
            r = np.linalg.norm(b - A @ x)
            if r_prev is not None:
                ratios.append(r / r_prev)
            r_prev = r
        rates.append(max(ratios))
    assert max(rates) < 0.3
    assert rates[-1] < 1.5 * rates[0] + 0.02


def test_singular_pressure_laplacian():
    """Pure-Neumann K_p: the iterate is mean-zero and solves K x = b - mean(b)."""
    meshes, P1 = _hier(16)
    mats = [fem.stiffness_p1(m).tocsr() for m in meshes]
    mg = MG(mats, P1, singular=True)
    b = np.random.default_rng(2).standard_normal(mats[0].shape[0]) + 3.0
    x, cycles = mg.solve(b, 1e-12, 200)
    bp = b - b.mean()
    assert abs(x.mean()) < 1e-12 * np.linalg.norm(x)
    assert np.linalg.norm(bp - mats[0] @ x) <= 1e-11 * np.linalg.norm(bp)


def test_velocity_hierarchy_converges():
    """The Taylor-Hood velocity operator (1/tau) M + K_sym with no-slip rows."""
    n = 16
    sizes = level_sizes(n)
    meshes = [Mesh(s) for s in sizes]
    Pv = [prolongation_velocity(meshes[l + 1], meshes[l]) for l in range(len(sizes) - 1)]
    mats = []
    for m in meshes:
        Mv = sp.kron(fem.mass_p2(m), sp.eye(2), format="csr")
        A = (Mv / 1e-3 + fem.ksym(m, 1.0)).tocsr()
        mats.append(fem.velocity_dirichlet(A, m.p2_boundary()))
    mg = MG(mats, Pv, degree=VEL_SMOOTH_DEGREE, ratio=VEL_LO_RATIO)
    b = np.random.default_rng(7).standard_normal(mats[0].shape[0])
    b[np.repeat(meshes[0].p2_boundary(), 2)] = 0.0
    x, cycles = mg.solve(b, 1e-12, 100)
    ref = spla.spsolve(mats[0].tocsc(), b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_step_with_inner_tolerance():
    """A whole step with inner_rtol = 1e-4: the same solution as the exact
    step (to the outer tolerance), and no more outer iterations than with
    one V-cycle per block."""
    n = 16
    p = inputs.default_params()
    p["rtol"] = 1e-10
    s0 = inputs.initial_state(n, seed=3)
    exact = Oracle(n, p, exact=True).step(s0)[0]
    one, info1 = Oracle(n, p).step(s0)[:2]
    pi = dict(p, inner_rtol=1e-4, inner_maxit=20)
    inner, info2 = Oracle(n, pi).step(s0)[:2]
    for key in ("phi", "mu", "Phi_v", "v"):
        a, e = np.ravel(inner[key]), np.ravel(exact[key])
        assert np.linalg.norm(a - e) <= 1e-6 * np.linalg.norm(e), key
    solves = [k for k, v in info1.items() if isinstance(v, dict)]
    assert {"ch_p", "ac", "ns"} <= set(solves)
    for name in solves:
        assert info2[name]["iters"] <= info1[name]["iters"], name


def test_paper_solver_settings():
    """Sec. 5's settings: CH / AC to rtol 1e-6 (atol 1e-8), the Oseen solve to
    rtol 1e-4 (atol 1e-8), AMG tolerance 1e-4.  Each solve stops at the first
    iterate meeting its own rule."""
    n = 16
    p = inputs.default_params()
    p.update(rtol=1e-6, atol=1e-8, ns_rtol=1e-4, ns_atol=1e-8, inner_rtol=1e-4, inner_maxit=20)
    o = Oracle(n, p)
    s0 = inputs.initial_state(n, seed=3)
    s1, info = o.step(s0)
    _, info2 = o.step(s1, keep_systems=True)[:2]
    tight = Oracle(n, dict(p, ns_rtol=0.0, rtol=1e-8, atol=0.0))
    _, info_t = tight.step(s1)[:2]
    systems = info2["systems"]
    for name, rt in (("ch_p", 1e-6), ("ch_N", 1e-6), ("ch_s", 1e-6), ("ac", 1e-6), ("ns", 1e-4)):
        b = systems[name][-1]
        nb = float(np.linalg.norm(b))
        assert info2[name]["converged"], name
        # ||b - A x|| <= max(rtol ||b||, atol), atol = 1e-8
        assert info2[name]["rel_residual"] * nb <= max(rt * nb, 1e-8) * (1 + 1e-9), name
    assert info2["ns"]["iters"] < info_t["ns"]["iters"]
