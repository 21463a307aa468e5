"""The one-graph step (chnss_set_step_mode 1): the whole semi-implicit step
recorded as a CUDA graph whose Krylov loops are conditional nodes, replayed
with one launch.  It runs the same kernels in the same order as the
host-driven step, so states and iteration counts must be equal bitwise, for
every model variant, over several steps (the graph cache keeps two state
pairs), in a batch, and with failures reported instead of hanging."""
import numpy as np
import pytest

from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _equal(a, b):
    return all(bool((a[k] == b[k]).all()) for k in a)


def _run(n, params, init, steps, mode, top_bc=0, concurrent=True):
    mesh = chnss.Mesh(n, top_bc=top_bc)
    ctx = chnss.Context(mesh, params)
    ctx.set_step_concurrency(concurrent)
    ctx.set_step_mode(mode)
    a = chnss.state_to_device(init)
    b = ctx.new_state()
    infos = []
    for _ in range(steps):
        _, info, st = ctx.step(a, b)
        assert st == 0
        infos.append(info)
        a, b = b, a
    return a, infos


CASES = {
    "fp64": (32, dict(inputs.default_params()), "film", 0),
    "mixed": (32, dict(inputs.default_params(), precision=1, ortho=1), "film", 0),
    "bf16": (20, dict(inputs.default_params(), precision=2, ortho=1), "film", 0),
    "mobility": (16, dict(inputs.default_params(), mobility_kind=1, beta=inputs.film_betas(0.01)), "film", 0),
    "open_top": (16, dict(inputs.default_params(), top_bc=1), "film", 1),
    "solvent_air": (16, dict(inputs.solvent_air_params()), "solvent_air", 0),
    "inner_mg": (16, dict(inputs.default_params(), inner_rtol=1e-4, inner_maxit=20), "film", 0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_graph_step_equals_host_step(torch, case):
    n, p, init, top_bc = CASES[case]
    st0 = (inputs.initial_state_solvent_air if init == "solvent_air" else inputs.initial_state)(n, seed=21)
    host, ih = _run(n, p, st0, 3, 0, top_bc)
    graph, ig = _run(n, p, st0, 3, 1, top_bc)
    assert _equal(host, graph), case
    for a, b in zip(ih, ig):
        for k in a:
            assert a[k]["iters"] == b[k]["iters"] and a[k]["converged"] == b[k]["converged"], (case, k, a[k], b[k])
            assert a[k]["rel_residual"] == b[k]["rel_residual"], (case, k)


def test_graph_step_serial_branches(torch):
    """With the solve groups one after the other the recorded graph has no
    parallel branches; still the same result."""
    n, p = 16, dict(inputs.default_params(), precision=1, ortho=1)
    st0 = inputs.initial_state(n, seed=4)
    host, _ = _run(n, p, st0, 2, 0, concurrent=False)
    graph, _ = _run(n, p, st0, 2, 1, concurrent=False)
    assert _equal(host, graph)


@pytest.mark.parametrize("batch_mode", [0, 1])
def test_graph_batched_steps_equal_single_steps(torch, batch_mode):
    """Both batch modes (a graph launch per instance; one graph launch for
    the whole batch) give every instance bitwise its single steps."""
    inst = [(16, 0.1), (20, 0.3), (32, 0.05)]
    ref, ctxs, cur = [], [], []
    for i, (n, evap) in enumerate(inst):
        p = dict(inputs.default_params(), evap_rate=evap, precision=1, ortho=1)
        st0 = inputs.initial_state(n, seed=30 + i)
        ref.append(_run(n, p, st0, 2, 0))
        c = chnss.Context(chnss.Mesh(n), p, stream=torch.cuda.Stream())
        c.set_step_mode(1)
        ctxs.append(c)
        cur.append(chnss.state_to_device(st0))
    chnss.set_batch_mode(batch_mode)
    try:
        before = chnss.batch_stats()
        for _ in range(2):
            cur, recs, st = chnss.step_batched(ctxs, cur)
            assert st == 0
        after = chnss.batch_stats()
    finally:
        chnss.set_batch_mode(0)
    key = "one_graph" if batch_mode == 1 else "per_instance"
    assert after[key] == before[key] + 2, (before, after)   # the chosen path ran on both calls
    for (s_ref, i_ref), s_b, rec in zip(ref, cur, recs):
        assert _equal(s_b, s_ref)
        for k in rec:
            assert rec[k]["iters"] == i_ref[-1][k]["iters"], k


def test_graph_step_reports_nonconvergence(torch):
    """maxit = 2: every FGMRES loop of the graph stops after two iterations
    and the step returns CHNSS_ERR_NOCONV, like the host-driven step."""
    n = 16
    p = dict(inputs.default_params(), maxit=2, restart=2)
    res = {}
    for mode in (0, 1):
        ctx = chnss.Context(chnss.Mesh(n), p)
        ctx.set_step_mode(mode)
        out, info, st = ctx.step(chnss.state_to_device(inputs.initial_state(n, seed=2)), check=False)
        res[mode] = (st, info, chnss.state_to_numpy(out))
    assert res[0][0] == res[1][0] == 4                       # CHNSS_ERR_NOCONV
    for k in ("ch_p", "ac", "ns"):
        assert res[1][1][k]["iters"] == 2 and not res[1][1][k]["converged"]
    assert _equal(res[0][2], res[1][2])


def test_graph_mode_argument_checks(torch):
    ctx = chnss.Context(chnss.Mesh(8), dict(inputs.default_params(), restart=40))
    with pytest.raises(chnss.ChnssError):
        ctx.set_step_mode(1)                                 # restart > 31
    with pytest.raises(chnss.ChnssError):
        ctx.set_step_mode(2)
