"""The 3D adjoint on the GPU (chnss3_adjoint_step) against the oracle's
discrete adjoint of the 3D step (oracle/adjoint_three_d.py, sparse-LU
transposed solves), enclosed and open top, constant and concentration-
dependent mobility; the checkpointed trajectory gradient against the
oracle's and against central differences of the GPU forward."""
import numpy as np
import pytest

from oracle import adjoint_three_d as oadj
from oracle import three_d as t3
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


def _params(**kw):
    p = inputs.default_params()
    p.update(alpha=[1e-2] * 4, evap_rate=0.5, rtol=1e-12)
    p.update(kw)
    return p


def _moving_state(o, n, seed):
    """A state with an interior flow and potentials, so that the convection
    and shift derivatives are exercised from the first step."""
    st = {k: np.asarray(v, dtype=float).copy() for k, v in inputs.initial_state_3d(n, seed=seed).items()}
    rng = np.random.default_rng(seed)
    bnd = np.repeat(o.mesh.p2_boundary(), 3)
    st["v"] = np.where(bnd, 0.0, 0.5 * rng.standard_normal(st["v"].shape))
    st["mu"] = 0.1 * rng.standard_normal(st["mu"].shape)
    return st


CASES = {
    "enclosed": dict(),
    "mobility": dict(mobility_kind=1),
    "open_top": dict(top_bc=1),
    "large_alpha": dict(alpha=[2.0, 1.0, 0.5, 0.8]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_step_matches_oracle(torch, case):
    n = 4
    p = _params(**CASES[case])
    o = t3.Oracle3D(n, p, exact=True)
    sk = o.step(_moving_state(o, n, seed=3))[0]
    sk1 = o.step(sk)[0]
    rng = np.random.default_rng(7)
    lam = {k: rng.standard_normal(np.shape(v)) for k, v in sk.items()}
    lam["v"][np.repeat(o.mesh.p2_boundary(), 3)] = 0.0
    ref, th = oadj.adjoint_step(o, sk, sk1, lam)
    ctx = chnss.Context3(n, p)
    out, grad, info, st = ctx.adjoint_step(*(chnss.state_to_device(x) for x in (sk, sk1, lam)), check=False)
    assert st == 0, info
    for name, i in info.items():
        assert i["converged"], (name, i)
    got = chnss.state_to_numpy(out)
    for key in ("phi", "mu", "Phi_v", "v"):
        assert rel(got[key], ref[key]) < 1e-8, (case, key, rel(got[key], ref[key]))
    assert np.abs(got["p"]).max() == 0.0
    assert np.abs(got["v"][np.repeat(o.mesh.p2_boundary(), 3)]).max() == 0.0
    assert grad[0] == pytest.approx(th["evap"], rel=1e-8)
    assert grad[1] == pytest.approx(th["gamma"], rel=1e-8)


def test_concurrent_adjoint_equals_serial(torch):
    """The three adjoint groups overlap on their own streams; their
    contributions are summed in a fixed order, so the result is bitwise the
    one of the serial setting."""
    n = 8
    p = _params(mobility_kind=1)
    o = t3.Oracle3D(n, p)
    sk = o.step(_moving_state(o, n, seed=9))[0]
    sk1 = o.step(sk)[0]
    rng = np.random.default_rng(3)
    lam = {k: rng.standard_normal(np.shape(v)) for k, v in sk.items()}
    lam["v"][np.repeat(o.mesh.p2_boundary(), 3)] = 0.0
    res = []
    for conc in (True, False):
        ctx = chnss.Context3(n, p)
        ctx.set_step_concurrency(conc)
        out, grad, info, st = ctx.adjoint_step(*(chnss.state_to_device(x) for x in (sk, sk1, lam)))
        assert st == 0
        res.append((chnss.state_to_numpy(out), list(grad), [v["iters"] for v in info.values()]))
    (a, ga, ia), (b, gb, ib) = res
    assert ia == ib and ga == gb
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        assert np.array_equal(a[key], b[key]), key


def test_objective_matches_oracle(torch):
    n = 4
    p = _params()
    o = t3.Oracle3D(n, p)
    st = _moving_state(o, n, seed=5)
    ctx = chnss.Context3(n, p)
    dev = chnss.state_to_device(st)
    g = torch.zeros_like(dev["phi"][0])
    J = ctx.objective(dev["phi"][0], g)
    assert J == pytest.approx(oadj.objective(o, st), rel=1e-12)
    K = o.forms[0].K
    assert rel(g.cpu().numpy(), 2.0 * (K @ st["phi"][0])) < 1e-12


@pytest.fixture(scope="module")
def trajectory(torch):
    n, steps = 4, 3
    p = _params(mobility_kind=1)
    o = t3.Oracle3D(n, p)
    st0 = _moving_state(o, n, seed=11)
    ctx = chnss.Context3(n, p)
    g = gadj.trajectory_gradient(ctx, chnss.state_to_device(st0), steps, checkpoint_every=2)
    return n, steps, p, st0, g


def test_trajectory_gradient_matches_oracle_adjoint(trajectory):
    """Three GPU steps and their checkpointed reverse sweep against the
    oracle's (exact solves) on 4^3 cubes, concentration-dependent mobility."""
    n, steps, p, st0, g = trajectory
    J, ref = oadj.trajectory_gradient(n, p, st0, steps)
    assert g["J"] == pytest.approx(J, rel=1e-9)
    assert g["evap"] == pytest.approx(ref["evap"], rel=1e-6)
    assert g["gamma"] == pytest.approx(ref["gamma"], rel=1e-6)
    for key in ("phi", "Phi_v", "v", "mu"):
        assert rel(g["adj0"][key].cpu().numpy(), ref["state0"][key]) < 1e-6, key


def test_trajectory_gradient_vs_central_differences(trajectory, torch):
    """Central differences of the GPU forward itself (relative step 1e-4).
    On 4^3 cubes over three steps dJ/d(evap_rate) is ~6e-8: the difference
    quotient then resolves J changes of ~3e-12, where the 1e-12 Krylov
    tolerance of the forward solves shows, so that parameter is held to 1e-3
    (its 1e-6 agreement with the oracle's adjoint is the sharp check); the
    mobility scale and the initial polymer field to 1e-5."""
    n, steps, p, st0, g = trajectory

    def J(prm, phi0=None):
        c = chnss.Context3(n, prm)
        st = chnss.state_to_device(st0)
        if phi0 is not None:
            st["phi"][0].copy_(phi0)
        for _ in range(steps):
            st = c.step(st)[0]
        return c.objective(st["phi"][0])
    h = 1e-4 * p["evap_rate"]
    fd = (J(dict(p, evap_rate=p["evap_rate"] + h)) - J(dict(p, evap_rate=p["evap_rate"] - h))) / (2 * h)
    assert g["evap"] == pytest.approx(fd, rel=1e-3)
    h = 1e-4
    fd = (J(dict(p, gamma=[1 + h] * 3)) - J(dict(p, gamma=[1 - h] * 3))) / (2 * h)
    assert g["gamma"] == pytest.approx(fd, rel=1e-5)
    d = torch.as_tensor(np.random.default_rng(2).standard_normal(np.shape(st0["phi"][0])) * 0.01,
                        dtype=torch.float64, device="cuda")
    base = torch.as_tensor(st0["phi"][0], dtype=torch.float64, device="cuda")
    fd = (J(p, base + h * d) - J(p, base - h * d)) / (2 * h)
    assert float((g["adj0"]["phi"][0] * d).sum()) == pytest.approx(fd, rel=1e-5)


def test_adjoint_step_at_8(torch):
    """8^3 cubes (a three-level hierarchy, 4,913 velocity nodes): the
    transposed solves converge and the result matches the oracle's adjoint
    (whose sparse-LU solves take ~20 s here; 16^3 would take minutes)."""
    n = 8
    p = _params()
    o = t3.Oracle3D(n, p, exact=True)
    sk = o.step(_moving_state(o, n, seed=8))[0]
    sk1 = o.step(sk)[0]
    rng = np.random.default_rng(8)
    lam = {k: rng.standard_normal(np.shape(v)) for k, v in sk.items()}
    lam["v"][np.repeat(o.mesh.p2_boundary(), 3)] = 0.0
    ref, th = oadj.adjoint_step(o, sk, sk1, lam)
    ctx = chnss.Context3(n, p)
    out, grad, info, st = ctx.adjoint_step(*(chnss.state_to_device(x) for x in (sk, sk1, lam)))
    assert st == 0
    got = chnss.state_to_numpy(out)
    for key in ("phi", "mu", "Phi_v", "v"):
        assert rel(got[key], ref[key]) < 1e-8, key
    assert grad[0] == pytest.approx(th["evap"], rel=1e-7)
    assert grad[1] == pytest.approx(th["gamma"], rel=1e-7)


def test_adjoint_argument_checks(torch):
    ctx = chnss.Context3(2, _params())
    st = ctx.new_state()
    bad = dict(st, v=None)
    with pytest.raises(chnss.ChnssError):
        ctx.adjoint_step(st, st, bad)
