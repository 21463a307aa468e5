"""The 3D oracle adjoint (oracle/adjoint_three_d.py) against central
differences of the 3D oracle step itself (sparse-LU solves, two steps on the
Kuhn mesh of 2^3 cubes): the evaporation rate, the mobility scale and every
field of the initial state, enclosed and open top, constant and
concentration-dependent mobility (CPU only)."""
import numpy as np
import pytest

from oracle import adjoint_three_d as adj
from oracle import three_d as t3
from paper_2501_11767_gb300 import inputs

N, STEPS = 2, 2


def _setup(alpha=(1e-2,) * 4, **kw):
    p = inputs.default_params()
    p.update(alpha=list(alpha), gamma=[1.0] * 3)
    p.update(kw)
    st0 = {k: np.asarray(v, dtype=float).copy() for k, v in inputs.initial_state_3d(N, seed=1).items()}
    o = t3.Oracle3D(N, p, exact=True)
    s = o.step(st0)[0]
    rng = np.random.default_rng(5)
    bnd = np.repeat(o.mesh.p2_boundary(), 3)
    s["v"] = np.where(bnd, 0.0, rng.standard_normal(s["v"].shape))   # a flow that the steps convect
    s["mu"] = 0.1 * rng.standard_normal(s["mu"].shape)
    J, g = adj.trajectory_gradient(N, p, s, STEPS)
    return p, s, J, g, bnd, rng


def _J(p, st):
    o = t3.Oracle3D(N, p, exact=True)
    for _ in range(STEPS):
        st = o.step(st)[0]
    return adj.objective(o, st)


def _fd_param(p, s, key, rel=1e-3):
    if key == "evap":
        h = rel * p["evap_rate"]
        return (_J(dict(p, evap_rate=p["evap_rate"] + h), s) - _J(dict(p, evap_rate=p["evap_rate"] - h), s)) / (2 * h)
    h = rel
    return (_J(dict(p, gamma=[1 + h] * 3), s) - _J(dict(p, gamma=[1 - h] * 3), s)) / (2 * h)


def _fd_field(p, s, key, D, h):
    return (_J(p, dict(s, **{key: s[key] + h * D})) - _J(p, dict(s, **{key: s[key] - h * D}))) / (2 * h)


@pytest.mark.parametrize("kw", [dict(), dict(mobility_kind=1), dict(top_bc=1), dict(top_bc=1, mobility_kind=1)])
def test_parameter_gradients(kw):
    p, s, J, g, _, _ = _setup(**kw)
    assert J > 0
    for key in ("evap", "gamma"):
        fd = _fd_param(p, s, key)
        assert g[key] == pytest.approx(fd, rel=1e-5), (key, g[key], fd)


@pytest.mark.parametrize("kw", [dict(), dict(mobility_kind=1, top_bc=1)])
def test_initial_state_gradient(kw):
    """Directional derivatives along random directions, field by field (the
    velocity on interior nodes; the pressure does not enter the next step)."""
    p, s, _, g, bnd, rng = _setup(**kw)
    for key, h in (("phi", 1e-5), ("Phi_v", 1e-5), ("v", 1e-4)):
        D = rng.standard_normal(np.shape(s[key]))
        if key == "v":
            D[bnd] = 0.0
        fd = _fd_field(p, s, key, D, h)
        assert float(np.sum(g["state0"][key] * D)) == pytest.approx(fd, rel=1e-5), key
    assert np.abs(g["state0"]["p"]).max() == 0.0


def test_potential_gradient_through_the_convective_shift():
    """mu^k enters only through the shift alpha_i grad mu_i of the Oseen
    convection; with alpha = 1e-8 of the workloads its effect is below the
    finite-difference noise, so it is checked with large alpha_i."""
    p, s, _, g, _, rng = _setup(alpha=(20.0, 10.0, 5.0, 8.0))
    D = rng.standard_normal(s["mu"].shape)
    fd = _fd_field(p, s, "mu", D, 1e-3)
    assert float(np.sum(g["state0"]["mu"] * D)) == pytest.approx(fd, rel=1e-5)
