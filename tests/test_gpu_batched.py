"""Batched stepping of independent instances (chnss_step_batched) and the
SpMV launch-shape autotuner (chnss_autotune): both must leave the
arithmetic untouched, so their results are compared bit for bit with plain
chnss_step calls, and one instance against the oracle."""
import numpy as np
import pytest

from oracle.step import Oracle
from solve_compare import compare_solves
from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _same(a: dict, b: dict) -> bool:
    return all(bool((a[k] == b[k]).all()) for k in a)


def _instances():
    """A small sweep: several mesh sizes and evaporation rates, both precisions."""
    out = []
    for i, (n, evap, prec) in enumerate([(16, 0.05, 0), (32, 0.3, 0), (24, 0.5, 1), (32, 0.1, 1), (16, 0.2, 0)]):
        p = inputs.default_params()
        p.update(evap_rate=evap, precision=prec)
        out.append((n, p, inputs.initial_state(n, seed=100 + i)))
    return out


def test_batched_step_is_bitwise_the_single_step(torch):
    inst = _instances()
    meshes = {n: chnss.Mesh(n) for n in {n for n, _, _ in inst}}
    ref = []
    for n, p, st0 in inst:
        c = chnss.Context(meshes[n], p)
        s1, info1, _ = c.step(chnss.state_to_device(st0))
        s2, info2, _ = c.step(s1)
        ref.append((s2, info2))
    torch.cuda.synchronize()
    ctxs = [chnss.Context(meshes[n], p, stream=torch.cuda.Stream()) for n, p, _ in inst]
    cur = [chnss.state_to_device(st0) for _, _, st0 in inst]
    for _ in range(2):
        cur, recs, st = chnss.step_batched(ctxs, cur, max_threads=3)
        assert st == 0
    for (s_ref, info_ref), s_b, rec in zip(ref, cur, recs):
        assert _same(s_b, s_ref)
        for k in chnss.SYSTEM_NAMES:
            assert rec[k]["iters"] == info_ref[k]["iters"], k


def test_batched_instance_matches_oracle(torch):
    n, p, st0 = _instances()[1]
    ctxs = [chnss.Context(chnss.Mesh(n), p, stream=torch.cuda.Stream())]
    out, recs, _ = chnss.step_batched(ctxs, [chnss.state_to_device(st0)])
    ref, oinfo = Oracle(n, p).step(st0)
    got = chnss.state_to_numpy(out[0])
    compare_solves(got, recs[0], ref, oinfo, st0, p, lambda q: Oracle(n, q))


def test_batched_rejects_a_repeated_context(torch):
    n, p, st0 = _instances()[0]
    c = chnss.Context(chnss.Mesh(n), p)
    s = chnss.state_to_device(st0)
    with pytest.raises(chnss.ChnssError) as e:
        chnss.step_batched([c, c], [s, s])
    assert e.value.status == 1


def test_autotune_keeps_results_bitwise(torch):
    n = 64
    p = inputs.default_params()
    p["precision"] = 1
    st0 = chnss.state_to_device(inputs.initial_state(n, seed=9))
    mesh = chnss.Mesh(n)
    c = chnss.Context(mesh, p)
    before, info_b, _ = c.step(st0)
    t = c.autotune()
    assert t["block_p1"] in t["candidates"] and t["block_p2"] in t["candidates"]
    assert all(ms > 0 for ms in t["ms_p1"] + t["ms_p2"])
    after, info_a, _ = c.step(st0)
    assert _same(before, after)
    assert all(info_a[k]["iters"] == info_b[k]["iters"] for k in chnss.SYSTEM_NAMES)
    # a fresh context on the tuned mesh captures the tuned shapes
    c2 = chnss.Context(mesh, p)
    again, _, _ = c2.step(st0)
    assert _same(again, before)


@pytest.mark.parametrize("blocks", [(128, 512), (512, 128), (512, 512), (128, 128)])
def test_every_launch_shape_gives_the_same_step(torch, blocks):
    """Every SELL kernel (MG sweeps, transfers, the CH and Oseen operators,
    B and B^T) must cover all slices for any threads-per-block; a forward
    and an adjoint step are compared bit for bit with the default shape."""
    n = 48
    p = inputs.default_params()
    p.update(alpha=[1e-2] * 4, evap_rate=0.5)
    st0 = chnss.state_to_device(inputs.initial_state(n, seed=3))
    lam = {k: torch.randn_like(v) * 0.1 for k, v in st0.items()}
    mesh = chnss.Mesh(n)

    def run():
        c = chnss.Context(mesh, p)
        s1, info, _ = c.step(st0)
        adj, grad, _, _ = c.adjoint_step(st0, s1, lam)
        return s1, adj, grad, info

    ref = run()
    c = chnss.Context(mesh, p)
    c.set_spmv_block(*blocks)
    got = run()
    c.set_spmv_block(256, 256)
    assert _same(got[0], ref[0])
    assert all(bool((got[1][k] == ref[1][k]).all()) for k in ("phi", "mu", "Phi_v", "v"))
    assert got[2] == ref[2]
    with pytest.raises(chnss.ChnssError):
        c.set_spmv_block(96, 256)


def test_autotune_needs_an_assembled_context(torch):
    c = chnss.Context(chnss.Mesh(16), inputs.default_params())
    with pytest.raises(chnss.ChnssError) as e:
        c.autotune()
    assert e.value.status == 8
