"""The hand-written adjoint on the GPU (chnss_adjoint_step) against the
oracle's discrete adjoint, against central finite differences of the GPU
forward, checkpoint invariance, and the torch.autograd.Function."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle.step import Oracle
from paper_2501_11767_gb300 import chnss, inputs
from paper_2501_11767_gb300 import adjoint as gadj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _params():
    p = inputs.default_params()
    p.update(alpha=[1e-2] * 4, evap_rate=0.5, rtol=1e-12)
    return p


@pytest.mark.parametrize("n", [8, 32])
def test_adjoint_step_matches_oracle(torch, n):
    """One adjoint step against the oracle's discrete adjoint (32 x 32 is the
    mesh of the adjoint workload's oracle check).  The oracle solves the
    transposed systems exactly (sparse LU), the GPU by FGMRES to 1e-12; the
    parameter gradients are sums of dot products that cancel, so at 32 x 32
    that tolerance reaches them at ~1e-8 relative (bound 1e-7, still far
    inside the 1e-5 of the finite-difference check)."""
    p = _params()
    o = Oracle(n, p, exact=True)
    s0 = inputs.initial_state(n, seed=4)
    sk = o.step(s0)[0]
    sk1 = o.step(sk)[0]
    rng = np.random.default_rng(1)
    lam = {k: rng.standard_normal(v.shape) for k, v in sk.items()}
    lam["v"][np.repeat(o.mesh.p2_boundary(), 2)] = 0.0
    ref, th = oadj.adjoint_step(o, sk, sk1, lam)
    ctx = chnss.Context(chnss.Mesh(n), p)
    out, grad, info, st = ctx.adjoint_step(*(chnss.state_to_device(x) for x in (sk, sk1, lam)))
    assert st == 0
    got = chnss.state_to_numpy(out)
    for key in ("phi", "mu", "Phi_v", "v"):
        assert rel(got[key], ref[key]) < 1e-8, key
    gtol = 1e-8 if n <= 8 else 1e-7
    assert grad[0] == pytest.approx(th["evap"], rel=gtol)
    assert grad[1] == pytest.approx(th["gamma"], rel=gtol)


def test_concurrent_adjoint_equals_serial(torch):
    """The three adjoint groups (NS, AC, air potential -> CH) overlap on their
    own streams; their contributions are summed in a fixed order, so the
    result is bitwise the one of the serial setting."""
    n = 24
    p = _params()
    o = Oracle(n, p)
    s0 = inputs.initial_state(n, seed=9)
    sk = o.step(s0)[0]
    sk1 = o.step(sk)[0]
    rng = np.random.default_rng(3)
    lam = {k: rng.standard_normal(v.shape) for k, v in sk.items()}
    lam["v"][np.repeat(o.mesh.p2_boundary(), 2)] = 0.0
    res = []
    for conc in (1, 0):
        ctx = chnss.Context(chnss.Mesh(n), p)
        ctx.set_step_concurrency(conc)
        out, grad, info, st = ctx.adjoint_step(*(chnss.state_to_device(x) for x in (sk, sk1, lam)))
        assert st == 0
        res.append((chnss.state_to_numpy(out), list(grad), [v["iters"] for v in info.values()]))
    (a, ga, ia), (b, gb, ib) = res
    assert ia == ib
    assert ga == gb
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key


@pytest.fixture(scope="module")
def trajectory(torch):
    n, steps = 16, 4
    p = _params()
    st0 = inputs.initial_state(n, seed=6)
    ctx = chnss.Context(chnss.Mesh(n), p)
    g = gadj.trajectory_gradient(ctx, chnss.state_to_device(st0), steps, checkpoint_every=2)
    return n, steps, p, st0, ctx, g


def test_trajectory_gradient_matches_oracle_adjoint(trajectory):
    n, steps, p, st0, ctx, g = trajectory
    J, ref = oadj.trajectory_gradient(n, p, st0, steps)
    assert g["J"] == pytest.approx(J, rel=1e-9)
    assert g["evap"] == pytest.approx(ref["evap"], rel=1e-6)
    assert g["gamma"] == pytest.approx(ref["gamma"], rel=1e-6)
    assert rel(g["adj0"]["phi"][0].cpu().numpy(), ref["phi_p0"]) < 1e-6


def test_trajectory_gradient_on_32_matches_oracle_adjoint(torch):
    """The checkpointed trajectory gradient on 32 x 32 (three steps,
    checkpoints every two) against the oracle's adjoint of the same
    trajectory: J, both parameter gradients and the initial polymer field's
    gradient."""
    n, steps = 32, 3
    p = _params()
    st0 = inputs.initial_state(n, seed=32)
    ctx = chnss.Context(chnss.Mesh(n), p)
    g = gadj.trajectory_gradient(ctx, chnss.state_to_device(st0), steps, checkpoint_every=2)
    J, ref = oadj.trajectory_gradient(n, p, st0, steps)
    assert g["J"] == pytest.approx(J, rel=1e-9)
    assert g["evap"] == pytest.approx(ref["evap"], rel=1e-6)
    assert g["gamma"] == pytest.approx(ref["gamma"], rel=1e-6)
    assert rel(g["adj0"]["phi"][0].cpu().numpy(), ref["phi_p0"]) < 1e-6


def test_trajectory_gradient_vs_central_differences(trajectory, torch):
    """Central differences of the GPU forward itself (relative step 1e-4, see
    the oracle test for why not 1e-6)."""
    n, steps, p, st0, ctx, g = trajectory
    mesh = ctx.mesh

    def J(prm, phi0=None):
        c = chnss.Context(mesh, prm)
        st = chnss.state_to_device(st0)
        if phi0 is not None:
            st["phi"][0].copy_(phi0)
        for _ in range(steps):
            st = c.step(st)[0]
        return c.objective(st["phi"][0])
    h = 1e-4 * p["evap_rate"]
    fd = (J(dict(p, evap_rate=p["evap_rate"] + h)) - J(dict(p, evap_rate=p["evap_rate"] - h))) / (2 * h)
    assert g["evap"] == pytest.approx(fd, rel=1e-5)
    h = 1e-4
    fd = (J(dict(p, gamma=[1 + h] * 3)) - J(dict(p, gamma=[1 - h] * 3))) / (2 * h)
    assert g["gamma"] == pytest.approx(fd, rel=1e-5)
    d = torch.as_tensor(np.random.default_rng(2).standard_normal(st0["phi"][0].shape) * 0.01,
                        dtype=torch.float64, device="cuda")
    base = torch.as_tensor(st0["phi"][0], dtype=torch.float64, device="cuda")
    fd = (J(p, base + h * d) - J(p, base - h * d)) / (2 * h)
    assert float((g["adj0"]["phi"][0] * d).sum()) == pytest.approx(fd, rel=1e-5)


def test_checkpointing_is_exact(trajectory):
    n, steps, p, st0, ctx, g = trajectory
    for k in (1, steps):
        g2 = gadj.trajectory_gradient(ctx, chnss.state_to_device(st0), steps, checkpoint_every=k)
        assert g2["J"] == g["J"] and g2["evap"] == g["evap"] and g2["gamma"] == g["gamma"]
        assert bool((g2["adj0"]["phi"][0] == g["adj0"]["phi"][0]).all())


def test_autograd_function(trajectory, torch):
    n, steps, p, st0, ctx, g = trajectory
    phi0 = torch.as_tensor(st0["phi"][0], dtype=torch.float64, device="cuda").requires_grad_(True)
    evap = torch.tensor(p["evap_rate"], dtype=torch.float64, requires_grad=True)
    gam = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    J = gadj.FilmGradient.apply(phi0, evap, gam, ctx.mesh, p, chnss.state_to_device(st0), steps, 2)
    J.backward()
    assert float(J) == pytest.approx(g["J"], rel=1e-12)
    assert float(evap.grad) == pytest.approx(g["evap"], rel=1e-10)
    assert float(gam.grad) == pytest.approx(g["gamma"], rel=1e-10)
    assert rel(phi0.grad.cpu().numpy(), g["adj0"]["phi"][0].cpu().numpy()) < 1e-10


def test_adjoint_step_variable_mobility(torch):
    """Concentration-dependent mobility: the transposed K_kappa and the
    derivative of K_kappa(phi_i^k) against the oracle's adjoint; the
    trajectory gradient against the oracle's."""
    n = 8
    p = dict(_params(), mobility_kind=1)
    o = Oracle(n, p, exact=True)
    sk = o.step(inputs.initial_state(n, seed=4))[0]
    sk1 = o.step(sk)[0]
    rng = np.random.default_rng(2)
    lam = {k: rng.standard_normal(v.shape) for k, v in sk.items()}
    lam["v"][np.repeat(o.mesh.p2_boundary(), 2)] = 0.0
    ref, th = oadj.adjoint_step(o, sk, sk1, lam)
    ctx = chnss.Context(chnss.Mesh(n), p)
    out, grad, info, st = ctx.adjoint_step(*(chnss.state_to_device(x) for x in (sk, sk1, lam)))
    assert st == 0
    got = chnss.state_to_numpy(out)
    for key in ("phi", "mu", "Phi_v", "v"):
        assert rel(got[key], ref[key]) < 1e-8, key
    assert grad[0] == pytest.approx(th["evap"], rel=1e-8)
    assert grad[1] == pytest.approx(th["gamma"], rel=1e-8)
    # a short trajectory (GPU forward at rtol 1e-12, exact oracle solves)
    steps = 3
    st0 = inputs.initial_state(n, seed=6)
    J, g = oadj.trajectory_gradient(n, p, st0, steps)
    gg = gadj.trajectory_gradient(chnss.Context(chnss.Mesh(n), p), chnss.state_to_device(st0), steps,
                                  checkpoint_every=2)
    assert gg["J"] == pytest.approx(J, rel=1e-8)
    assert gg["evap"] == pytest.approx(g["evap"], rel=1e-6)
    assert gg["gamma"] == pytest.approx(g["gamma"], rel=1e-6)


def test_adjoint_step_open_top(torch):
    """Open (do-nothing) top: the transposed saddle point without the
    pressure shift, free top velocities, against the oracle's adjoint."""
    n = 8
    p = dict(_params(), top_bc=1)
    o = Oracle(n, p, exact=True)
    sk = o.step(inputs.initial_state(n, seed=4))[0]
    sk1 = o.step(sk)[0]
    rng = np.random.default_rng(5)
    lam = {k: rng.standard_normal(v.shape) for k, v in sk.items()}
    lam["v"][np.repeat(o.mesh.p2_boundary(), 2)] = 0.0
    ref, th = oadj.adjoint_step(o, sk, sk1, lam)
    ctx = chnss.Context(chnss.Mesh(n, top_bc=1), p)
    out, grad, info, st = ctx.adjoint_step(*(chnss.state_to_device(x) for x in (sk, sk1, lam)))
    assert st == 0
    got = chnss.state_to_numpy(out)
    for key in ("phi", "mu", "Phi_v", "v"):
        assert rel(got[key], ref[key]) < 1e-8, key
    assert grad[0] == pytest.approx(th["evap"], rel=1e-8)
    assert grad[1] == pytest.approx(th["gamma"], rel=1e-8)
