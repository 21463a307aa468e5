"""The solvent-air sub-model (Sec. 5.1) on the GPU against the oracle:
Taylor-expanded Flory-Huggins loads, only the solvent CH system solved, the
truncation to [0, 1], then AC, air potential and NS."""
import numpy as np
import pytest

from oracle.step import Oracle
from solve_compare import compare_solves
from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu
SOLVE_TOL = 1e-9


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n", [32, 20])
def test_solvent_air_steps_match_oracle(torch, n):
    p = inputs.solvent_air_params()
    o = Oracle(n, p)
    ctx = chnss.Context(chnss.Mesh(n), p)
    st = inputs.initial_state_solvent_air(n, seed=n)
    for k in range(2):
        ref, rinfo = o.step(st)
        out, info, status = ctx.step(chnss.state_to_device(st))
        assert status == 0
        got = chnss.state_to_numpy(out)
        assert info["ch_p"]["iters"] == 0 and info["ch_N"]["iters"] == 0
        assert not np.any(got["phi"][:2]) and not np.any(got["mu"][:2])
        assert got["phi"][2].min() >= 0.0 and got["phi"][2].max() <= 1.0
        compare_solves(got, info, ref, rinfo, st, p, lambda q: Oracle(n, q), names=("ch_s", "ac", "ns"), where=k)
        assert rel(got["mu"][3], ref["mu"][3]) <= SOLVE_TOL
        st = ref


def test_solvent_air_mixed_precision(torch):
    n = 32
    p = inputs.solvent_air_params()
    o = Oracle(n, dict(p, rtol=1e-12))
    ctx = chnss.Context(chnss.Mesh(n), dict(p, precision=1, rtol=1e-10))
    st = inputs.initial_state_solvent_air(n, seed=3)
    ref, _ = o.step(st)
    out, info, status = ctx.step(chnss.state_to_device(st))
    assert status == 0
    got = chnss.state_to_numpy(out)
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        assert rel(got[key], ref[key]) <= 1e-6, key


def test_solvent_air_has_no_adjoint(torch):
    n = 8
    p = inputs.solvent_air_params()
    ctx = chnss.Context(chnss.Mesh(n), p)
    st = chnss.state_to_device(inputs.initial_state_solvent_air(n))
    with pytest.raises(chnss.ChnssError) as e:
        ctx.adjoint_step(st, st, st)
    assert e.value.status == 1
