"""Pins of the oracle's discrete adjoint: every transposed-Jacobian product
against a directional finite difference of the forward function it
differentiates, and the gradient of J = int |grad phi_p|^2 after several
exact-solve steps against central finite differences (CPU only)."""
import numpy as np
import pytest

from oracle import adjoint, fem, model
from oracle.mesh import Mesh
from paper_2501_11767_gb300 import inputs


def _fd(fun, x, d, h=1e-6):
    return (fun(x + h * d) - fun(x - h * d)) / (2 * h)


def test_hessian_by_finite_differences():
    rng = np.random.default_rng(7)
    for pt in rng.uniform(0.05, 0.6, size=(15, 5)):
        H = adjoint.hessian(*pt)
        for j in range(5):
            e = np.zeros(5)
            e[j] = 1.0
            fd = _fd(lambda x: np.array(model.potential_partials(*x)), pt, e)
            for i in range(5):
                assert H[i][j] == pytest.approx(fd[i], rel=1e-6, abs=1e-8)


@pytest.fixture(scope="module")
def fields():
    n = 6
    mesh = Mesh(n)
    rng = np.random.default_rng(3)
    st = inputs.initial_state(n, seed=2)
    st["Phi_v"] = 0.2 + 0.1 * rng.random(mesh.N1)
    st["v"] = 0.1 * rng.standard_normal(2 * mesh.N2)
    st["v"][np.repeat(mesh.p2_boundary(), 2)] = 0.0
    return mesh, st, rng


def test_conv_p1_vjp(fields):
    mesh, st, rng = fields
    x, y = rng.standard_normal(mesh.N1), rng.standard_normal(mesh.N1)
    dv = rng.standard_normal(2 * mesh.N2)
    fd = _fd(lambda v: y @ (fem.convection_p1(mesh, v) @ x), st["v"], dv)
    assert adjoint.conv_p1_vjp(mesh, x, y) @ dv == pytest.approx(fd, rel=1e-7)


def test_conv_p2_vjp_nodes_and_shift(fields):
    mesh, st, rng = fields
    x, y = rng.standard_normal(2 * mesh.N2), rng.standard_normal(2 * mesh.N2)
    shift = rng.standard_normal((mesh.E, 2))
    import scipy.sparse as sp

    def yJx(v, s):
        J = sp.kron(fem.convection_p2(mesh, v, s), sp.eye(2))
        return y @ (J @ x)
    wbar, sbar = adjoint.conv_p2_vjp(mesh, x, y)
    dv = rng.standard_normal(2 * mesh.N2)
    assert wbar @ dv == pytest.approx(_fd(lambda v: yJx(v, shift), st["v"], dv), rel=1e-7)
    ds = rng.standard_normal((mesh.E, 2))
    fd = (yJx(st["v"], shift + 1e-6 * ds) - yJx(st["v"], shift - 1e-6 * ds)) / 2e-6
    assert np.sum(sbar * ds) == pytest.approx(fd, rel=1e-7)


def test_loads_vjp(fields):
    mesh, st, rng = fields
    wts = [rng.standard_normal(mesh.N1) for _ in range(5)]

    def total(phi, Phi):
        L = model.potential_loads(mesh, phi, Phi)
        return sum(w @ l for w, l in zip(wts, L))
    pb, Pb = adjoint.loads_vjp(mesh, st["phi"], st["Phi_v"], wts)
    dphi = rng.standard_normal(st["phi"].shape)
    dPhi = rng.standard_normal(mesh.N1)
    fd = _fd(lambda t: total(st["phi"] + t * dphi, st["Phi_v"] + t * dPhi), 0.0, 1.0)
    assert np.sum(pb * dphi) + Pb @ dPhi == pytest.approx(fd, rel=1e-6)


def test_korteweg_vjp(fields):
    mesh, st, rng = fields
    params = inputs.default_params()
    y = rng.standard_normal(2 * mesh.N2)

    def yG(phi, Phi):
        s = dict(st, phi=phi, Phi_v=Phi)
        return y @ fem.korteweg(mesh, model.korteweg_tensor(mesh, s, params))
    pb, Pb = adjoint.korteweg_vjp(mesh, st["phi"], st["Phi_v"], y, params)
    dphi = rng.standard_normal(st["phi"].shape)
    dPhi = rng.standard_normal(mesh.N1)
    fd = _fd(lambda t: yG(st["phi"] + t * dphi, st["Phi_v"] + t * dPhi), 0.0, 1.0)
    assert np.sum(pb * dphi) + Pb @ dPhi == pytest.approx(fd, rel=1e-6)


def test_wstiff_vjp(fields):
    mesh, st, rng = fields
    params = dict(inputs.default_params(), mobility_kind=1)
    x, y = rng.standard_normal(mesh.N1), rng.standard_normal(mesh.N1)

    def yKx(phi):
        K = fem.weighted_stiffness_p1(mesh, model.mobility_at(mesh, phi, params, 1))
        return y @ (K @ x)
    d = rng.standard_normal(mesh.N1)
    fd = _fd(lambda t: yKx(st["phi"][1] + t * d), 0.0, 1.0)
    g = adjoint.wstiff_vjp(mesh, st["phi"][1], params["gamma"][1], x, y)
    assert g @ d == pytest.approx(fd, rel=1e-7)


def _J(n, params, st0, steps):
    from oracle.step import Oracle
    o = Oracle(n, params, exact=True)
    st = st0
    for _ in range(steps):
        st = o.step(st)[0]
    return adjoint.objective(o, st)


@pytest.fixture(scope="module", params=[(0, 0), (1, 0), (0, 1)],
                ids=["constant_mobility", "variable_mobility", "open_top"])
def gradient_case(request):
    n, steps = 8, 3
    mobility, top = request.param
    params = inputs.default_params()
    # every coupling visible
    params.update(alpha=[1e-2] * 4, evap_rate=0.5, mobility_kind=mobility, top_bc=top)
    st0 = inputs.initial_state(n, seed=11)
    J, g = adjoint.trajectory_gradient(n, params, st0, steps)
    return n, steps, params, st0, J, g


def test_adjoint_gradient_vs_central_differences(gradient_case):
    """Relative step 1e-4: J ~ 1e-4 here and dJ/d(evap) ~ 3e-7, so at a step
    of 1e-6 the round-off of J (exact sparse-LU solves) already moves the
    difference quotient by ~1e-4 relative; at 1e-4 the quotient agrees with
    the adjoint to ~4e-7 and the O(h^2) truncation is still negligible."""
    n, steps, params, st0, J, g = gradient_case
    h = 1e-4 * params["evap_rate"]
    up = dict(params, evap_rate=params["evap_rate"] + h)
    dn = dict(params, evap_rate=params["evap_rate"] - h)
    fd = (_J(n, up, st0, steps) - _J(n, dn, st0, steps)) / (2 * h)
    assert g["evap"] == pytest.approx(fd, rel=1e-5)
    h = 1e-4
    up = dict(params, gamma=[1 + h] * 3)
    dn = dict(params, gamma=[1 - h] * 3)
    fd = (_J(n, up, st0, steps) - _J(n, dn, st0, steps)) / (2 * h)
    assert g["gamma"] == pytest.approx(fd, rel=1e-5)
    d = np.random.default_rng(5).standard_normal(st0["phi"][0].shape) * 0.01
    h = 1e-4

    def Jphi(t):
        s = {k: v.copy() for k, v in st0.items()}
        s["phi"][0] = st0["phi"][0] + t * d
        return _J(n, params, s, steps)
    fd = (Jphi(h) - Jphi(-h)) / (2 * h)
    assert g["phi_p0"] @ d == pytest.approx(fd, rel=1e-5)


def test_checkpointing_gives_the_same_gradient(gradient_case):
    n, steps, params, st0, J, g = gradient_case
    J2, g2 = adjoint.trajectory_gradient(n, params, st0, steps, checkpoint_every=2)
    assert J2 == J
    assert g2["evap"] == pytest.approx(g["evap"], rel=1e-12)
    assert np.allclose(g2["phi_p0"], g["phi_p0"], rtol=1e-12, atol=1e-14)
