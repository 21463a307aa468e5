"""Pins of the solvent-air sub-model (Sec. 5.1) in the oracle: the
Taylor-expanded Flory-Huggins density, its partial derivatives, and one step
(truncation, absent species, exact-solve agreement)."""
import numpy as np
import pytest

from oracle import model
from oracle.step import Oracle
from paper_2501_11767_gb300 import inputs


def test_taylor_polynomial_of_xlnx_has_fifth_order_error():
    """x ln x - T4(x) = g^(5)(1/2) d^5 / 5! + O(d^6) with g^(5)(x) = -6 / x^4:
    the ratio tends to -96/120 = -0.8 only if all five coefficients are right."""
    for d in (1e-2, 5e-3, 2.5e-3):
        for sgn in (1.0, -1.0):
            x = 0.5 + sgn * d
            ratio = (x * np.log(x) - model.taylor_xlnx(x)) / (sgn * d) ** 5
            assert ratio == pytest.approx(-0.8, rel=0.05)
    # the derivative polynomial is the derivative of the polynomial
    x = np.linspace(-0.2, 1.2, 29)
    h = 1e-6
    fd = (model.taylor_xlnx(x + h) - model.taylor_xlnx(x - h)) / (2 * h)
    assert np.allclose(model.dtaylor_xlnx(x), fd, rtol=1e-8, atol=1e-8)


def test_flory_huggins_partials_match_finite_differences():
    prm = dict(inputs.solvent_air_params(), chi_sa=0.7, n_s=1.0, n_a=2.0)
    rng = np.random.default_rng(3)
    ps, pa, Ph = rng.uniform(0.0, 1.0, (3, 40))

    def f(ps, pa, Ph):
        q = model.interp_p(Ph)
        return (1 - q) * model.fh_liquid(ps, pa, prm) + q * model.fh_gas(ps, pa, prm)
    h = 1e-6
    d_s, d_a, d_v = model.fh_partials(ps, pa, Ph, prm)
    assert np.allclose(d_s, (f(ps + h, pa, Ph) - f(ps - h, pa, Ph)) / (2 * h), rtol=1e-7, atol=1e-7)
    assert np.allclose(d_a, (f(ps, pa + h, Ph) - f(ps, pa - h, Ph)) / (2 * h), rtol=1e-7, atol=1e-7)
    assert np.allclose(d_v, (f(ps, pa, Ph + h) - f(ps, pa, Ph - h)) / (2 * h), rtol=1e-7, atol=1e-7)


def test_gas_phase_favours_solvent_leaving():
    """In the gas phase (Phi_v = 1) the vaporisation term -phi_s ln phi_sat(s)
    = 13.8 phi_s raises the solvent potential by ln(1e6) over the liquid."""
    prm = inputs.solvent_air_params()
    ds_liq = model.fh_partials(np.array([0.3]), np.array([0.7]), np.array([0.0]), prm)[0]
    ds_gas = model.fh_partials(np.array([0.3]), np.array([0.7]), np.array([1.0]), prm)[0]
    assert (ds_gas - ds_liq)[0] == pytest.approx(np.log(1e6), rel=1e-12)


@pytest.fixture(scope="module")
def one_step():
    n = 8
    p = inputs.solvent_air_params()
    st0 = inputs.initial_state_solvent_air(n, seed=2)
    o = Oracle(n, dict(p, rtol=1e-12))
    ox = Oracle(n, p, exact=True)
    return st0, o.step(st0)[0], ox.step(st0)[0]


def test_step_truncates_and_keeps_absent_species_zero(one_step):
    st0, new, _ = one_step
    assert new["phi"][2].min() >= 0.0 and new["phi"][2].max() <= 1.0
    assert not np.any(new["phi"][:2]) and not np.any(new["mu"][:2])
    assert st0["phi"][2].max() > 1.0          # the start exceeds 1: the clip acts


def test_step_krylov_solves_match_sparse_lu(one_step):
    _, new, exact = one_step
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        a, b = np.ravel(new[key]), np.ravel(exact[key])
        assert np.linalg.norm(a - b) <= 1e-8 * max(np.linalg.norm(b), 1.0), key
