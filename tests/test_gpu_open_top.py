"""Open (do-nothing) top boundary on the GPU against the oracle: velocity
masks and transfers without the top edge, Dirichlet outflow rows in the
pressure convection-diffusion preconditioner, no pressure shift."""
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
def test_open_top_steps_match_oracle(torch, n):
    p = dict(inputs.default_params(), top_bc=1)
    o = Oracle(n, p)
    ctx = chnss.Context(chnss.Mesh(n, top_bc=1), p)
    st = inputs.initial_state(n, seed=n + 1)
    for k in range(2):
        ref, rinfo = o.step(st)
        out, info, status = ctx.step(chnss.state_to_device(st))
        assert status == 0
        got = chnss.state_to_numpy(out)
        compare_solves(got, info, ref, rinfo, st, p, lambda q: Oracle(n, q), where=k)
        st = ref
    # flow through the open top, zero on the walls
    mesh = o.mesh
    top = np.repeat((mesh.lat2[:, 1] == 2 * n) & ~mesh.p2_boundary(), 2)
    assert np.abs(got["v"][top]).max() > 0.0
    assert not got["v"][np.repeat(mesh.p2_boundary(), 2)].any()


def test_open_top_mixed_precision(torch):
    n = 32
    p = dict(inputs.default_params(), top_bc=1)
    o = Oracle(n, dict(p, rtol=1e-12))
    mesh = chnss.Mesh(n, top_bc=1)
    ctx = chnss.Context(mesh, dict(p, precision=1, rtol=1e-10))
    st = inputs.initial_state(n, seed=9)
    ref, _ = o.step(st)
    out, info, status = ctx.step(chnss.state_to_device(st))
    assert status == 0
    got = chnss.state_to_numpy(out)
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        assert rel(got[key], ref[key]) <= 1e-6, key
