"""chnss_diagnostics against the oracle's diagnostics: mass sums of the four
species, ||B v||, int p and the energy parts (Sec. 2.2 free energy, kinetic
energy), in FP64 through the C ABI."""
import numpy as np
import pytest

from oracle.step import Oracle
from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12     # FP64 sums of O(1) quantities in different orders


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _random_state(n, seed):
    """Fields with every diagnostic O(1): phase fields near the film values,
    Phi_v across [0, 1], a velocity that is not divergence-free (zero on the
    walls), a pressure with non-zero mean."""
    g = np.random.default_rng(seed)
    st = inputs.initial_state(n, seed=seed)
    N1, N2 = (n + 1) ** 2, (2 * n + 1) ** 2
    st["phi"] = np.stack([0.3 + 0.1 * g.standard_normal(N1), 0.3 + 0.1 * g.standard_normal(N1),
                          0.4 + 0.05 * g.standard_normal(N1)])
    st["Phi_v"] = g.uniform(0.0, 1.0, N1)
    v = g.standard_normal((N2, 2))
    lat = np.stack(np.meshgrid(np.arange(2 * n + 1), np.arange(2 * n + 1), indexing="xy"), -1).reshape(-1, 2)
    wall = np.any((lat == 0) | (lat == 2 * n), axis=1)
    v[wall] = 0.0
    st["v"] = v.ravel()
    st["p"] = 0.5 + g.standard_normal(N1)
    return st


def _check(got, ref, where):
    for i in range(3):
        assert got["mass"][i] == pytest.approx(ref["mass"][i], rel=TOL), (where, i)
    assert got["mass_a"] == pytest.approx(ref["mass_a"], rel=TOL, abs=TOL), where
    assert got["div"] == pytest.approx(ref["div"], rel=TOL), where
    assert got["p_mean"] == pytest.approx(ref["p_mean"], rel=TOL), where
    for k in ("local", "gradient", "kinetic"):
        assert got["energy_parts"][k] == pytest.approx(ref["energy_parts"][k], rel=TOL), (where, k)
    assert got["energy"] == pytest.approx(ref["energy"], rel=TOL), where


@pytest.mark.parametrize("n", [32, 20])
def test_diagnostics_match_oracle(torch, n):
    p = inputs.default_params()
    o = Oracle(n, p)
    ctx = chnss.Context(chnss.Mesh(n), p)
    st = _random_state(n, seed=n)
    got = ctx.diagnostics(chnss.state_to_device(st))
    _check(got, o.diagnostics(st), n)


def test_diagnostics_solvent_air_density(torch):
    n = 16
    p = inputs.solvent_air_params()
    o = Oracle(n, p)
    ctx = chnss.Context(chnss.Mesh(n), p)
    st = _random_state(n, seed=5)
    st["phi"][:2] = 0.0
    st["phi"][2] = np.clip(st["phi"][2] + 0.3, 0.0, 1.0)
    _check(ctx.diagnostics(chnss.state_to_device(st)), o.diagnostics(st), "solvent-air")


def test_diagnostics_of_a_step_and_determinism(torch):
    """After a step of the enclosed film the velocity is discretely
    divergence-free to the solve tolerance, the pressure has zero mean and
    every species' mass is conserved; two calls agree bitwise."""
    n = 32
    p = inputs.default_params()
    o = Oracle(n, p)
    ctx = chnss.Context(chnss.Mesh(n), p)
    st0 = inputs.initial_state(n, seed=3)
    d0 = ctx.diagnostics(chnss.state_to_device(st0))
    out, _, status = ctx.step(chnss.state_to_device(st0))
    assert status == 0
    d1 = ctx.diagnostics(out)
    assert d1 == ctx.diagnostics(out)
    ref = o.diagnostics(chnss.state_to_numpy(out))
    for i in range(3):
        assert d1["mass"][i] == pytest.approx(ref["mass"][i], rel=TOL)
        assert abs(d1["mass"][i] - d0["mass"][i]) <= 1e-9 * abs(d0["mass"][i]), i
    assert d1["div"] <= 1e-8 and ref["div"] <= 1e-8
    assert abs(d1["p_mean"]) <= 1e-12
    assert d1["energy_parts"]["kinetic"] > 0.0
