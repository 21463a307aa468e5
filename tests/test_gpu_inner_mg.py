"""Multigrid blocks as inner solves to a relative tolerance (inner_rtol > 0;
Sec. 5 applies its AMG preconditioners with a tolerance of 1e-4).  On the GPU
each loop of V-cycles is a conditional WHILE node of the captured
preconditioner graph; the oracle is MG.solve.  Per-solve parity as for the
single V-cycle (relative L2 <= 1e-9 when the Krylov iteration counts agree,
counts within +-1), the open top, variable mobility, both reduced
precisions, concurrency and the adjoint."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle.step import Oracle
from solve_compare import compare_solves
from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-9
MIXED_TOL = 1e-6


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
    p.update(inner_rtol=1e-4, inner_maxit=20)
    p.update(kw)
    return p


def _compare(torch, n, params, seed, steps=2, top_bc=0):
    o = Oracle(n, params)
    ctx = chnss.Context(chnss.Mesh(n, top_bc=top_bc), params)
    st = inputs.initial_state(n, seed=seed)
    for k in range(steps):
        ref, rinfo = o.step(st)
        out, info, status = ctx.step(chnss.state_to_device(st))
        torch.cuda.synchronize()
        assert status == 0
        got = chnss.state_to_numpy(out)
        compare_solves(got, info, ref, rinfo, st, params, lambda q: Oracle(n, q), where=k)
        assert rel(got["mu"][3], ref["mu"][3]) <= SOLVE_TOL
        st = ref
    return ctx


@pytest.mark.parametrize("n", [32, 20])
def test_inner_step_matches_oracle(torch, n):
    """n = 20 ends on an odd coarsest mesh (5)."""
    _compare(torch, n, _params(), seed=n)


def test_inner_tight_tolerance_and_cap(torch):
    """A tight inner tolerance (many V-cycles, cap reached in some blocks)
    and a cap of one V-cycle (the plain preconditioner's iterates)."""
    _compare(torch, 16, _params(inner_rtol=1e-9, inner_maxit=6), seed=2, steps=1)
    p1 = _params(inner_maxit=1)
    n = 16
    st = chnss.state_to_device(inputs.initial_state(n, seed=3))
    a, ia, _ = chnss.Context(chnss.Mesh(n), p1).step(st)
    b, ib, _ = chnss.Context(chnss.Mesh(n), dict(p1, inner_rtol=0.0)).step(st)
    for name in ia:
        assert ia[name]["iters"] == ib[name]["iters"], name
    for key in ("phi", "mu", "Phi_v", "v", "p"):
        assert rel(chnss.state_to_numpy(a)[key], chnss.state_to_numpy(b)[key]) <= 1e-12, key


def test_inner_open_top(torch):
    """Open top: K_p with Dirichlet outflow rows (non-singular)."""
    _compare(torch, 16, _params(top_bc=1), seed=5, top_bc=1)


def test_inner_variable_mobility(torch):
    """Per-species X2 = tau K_kappa + a M, each its own inner solve."""
    _compare(torch, 16, _params(mobility_kind=1, beta=inputs.film_betas(0.01)), seed=4)


@pytest.mark.parametrize("precision", [1, 2])
def test_inner_mixed_precision(torch, precision):
    """FP32 (and BF16-stored velocity) inner loops inside FP64 FGMRES: at an
    outer tolerance of 1e-10 the step stays within 1e-6 of the oracle solved
    to 1e-12."""
    n = 32
    p = _params()
    o = Oracle(n, dict(p, rtol=1e-12))
    ctx = chnss.Context(chnss.Mesh(n), dict(p, precision=precision, rtol=1e-10))
    st = inputs.initial_state(n, seed=7)
    for _ in range(2):
        ref, _ = o.step(st)
        out, info, status = ctx.step(chnss.state_to_device(st))
        assert status == 0
        got = chnss.state_to_numpy(out)
        for key in ("phi", "mu", "Phi_v", "v", "p"):
            assert rel(got[key], ref[key]) <= MIXED_TOL, key
        st = ref


def test_inner_concurrent_equals_serial(torch):
    n = 32
    p = _params(precision=1)
    st = chnss.state_to_device(inputs.initial_state(n, seed=12))
    conc = chnss.Context(chnss.Mesh(n), p)
    ser = chnss.Context(chnss.Mesh(n), p)
    ser.set_step_concurrency(False)
    a, b = st, st
    for _ in range(2):
        a, ia, _ = conc.step(a)
        b, ib, _ = ser.step(b)
        for k in a:
            assert bool((a[k] == b[k]).all()), k
        assert all(ia[k]["iters"] == ib[k]["iters"] for k in ia)


def test_inner_fewer_outer_iterations(torch):
    """More accurate blocks: no solve needs more outer iterations."""
    n = 64
    st = chnss.state_to_device(inputs.initial_state(n, seed=8))
    _, i1, _ = chnss.Context(chnss.Mesh(n), inputs.default_params()).step(st)
    _, i2, _ = chnss.Context(chnss.Mesh(n), _params()).step(st)
    for name in ("ch_p", "ch_N", "ch_s", "ac", "ns"):
        assert i2[name]["iters"] <= i1[name]["iters"], (name, i1[name], i2[name])


def test_inner_adjoint_matches_oracle(torch):
    """The transposed solves of the adjoint step use the same preconditioner."""
    n = 8
    p = _params(alpha=[1e-2] * 4, evap_rate=0.5, rtol=1e-12)
    o = Oracle(n, p, exact=True)
    sk = o.step(inputs.initial_state(n, seed=4))[0]
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
    assert grad[0] == pytest.approx(th["evap"], rel=1e-8)
    assert grad[1] == pytest.approx(th["gamma"], rel=1e-8)


@pytest.mark.parametrize("bad", [dict(inner_rtol=-1e-4), dict(inner_rtol=1.0), dict(inner_maxit=0),
                                 dict(inner_maxit=1001)])
def test_inner_parameter_errors(torch, bad):
    with pytest.raises(chnss.ChnssError):
        chnss.Context(chnss.Mesh(8), _params(**bad))


def test_paper_solver_settings_match_oracle(torch):
    """Sec. 5's settings: CH / AC to rtol 1e-6 (atol 1e-8), the Oseen solve to
    its own rtol 1e-4 (atol 1e-8), inner multigrid to 1e-4."""
    p = _params(rtol=1e-6, atol=1e-8, ns_rtol=1e-4, ns_atol=1e-8)
    ctx = _compare(torch, 32, p, seed=6)
    with pytest.raises(chnss.ChnssError):
        chnss.Context(chnss.Mesh(8), _params(ns_rtol=1.5))
