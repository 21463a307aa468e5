"""chnss_mass_solve_noalloc: the mass-matrix solve for callers that cannot
allocate device memory at the call (their memory is reserved up front by
their own pool, or they may not pay cudaMalloc's implicit synchronisation).
Its output must match the allocating path, chnss_solve(CHNSS_SYS_MU_A, rhs),
on consecutive calls that reuse the library's fixed scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
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


def _rhs(torch, n1, seed):
    g = np.random.default_rng(seed)
    return torch.as_tensor(g.standard_normal(n1), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n", [32, 256])          # 256: N1 = 66049, the array's exact fit
def test_noalloc_mass_solve_matches_allocating_solve(torch, n):
    ctx = chnss.Context(chnss.Mesh(n), inputs.default_params())
    ctx.assemble(chnss.state_to_device(inputs.initial_state(n)))
    for call, seed in enumerate((11, 12)):          # two calls in a row share the scratch array
        b = _rhs(torch, ctx.mesh.N1, seed)
        ref, rinfo, st_ref = ctx.solve(chnss.SYS_MU_A, rhs=b)
        x = torch.full_like(b, np.nan)              # stale output must not matter
        got, info, st = ctx.mass_solve_noalloc(b, x)
        torch.cuda.synchronize()
        assert st == 0 and st_ref == 0
        assert info["converged"] and info["iters"] == rinfo["iters"], (call, info, rinfo)
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(g - r) <= 1e-12 * np.linalg.norm(r), call


def test_noalloc_mass_solve_in_place(torch):
    """rhs == x_out: the right-hand side is read before the iterate is
    cleared, so an in-place solve gives the out-of-place result."""
    n = 32
    ctx = chnss.Context(chnss.Mesh(n), inputs.default_params())
    ctx.assemble(chnss.state_to_device(inputs.initial_state(n)))
    b = _rhs(torch, ctx.mesh.N1, 13)
    ref, rinfo, _ = ctx.mass_solve_noalloc(b, torch.empty_like(b))
    inplace = b.clone()
    got, info, st = ctx.mass_solve_noalloc(inplace, inplace)
    torch.cuda.synchronize()
    assert st == 0 and info["converged"] and info["iters"] == rinfo["iters"]
    assert torch.equal(got, ref)
    # partly overlapping arrays are refused before any work
    buf = torch.zeros(ctx.mesh.N1 + 8, dtype=torch.float64, device="cuda")
    with pytest.raises(chnss.ChnssError) as e:
        ctx.mass_solve_noalloc(buf[:ctx.mesh.N1], buf[8:])
    assert e.value.status == 1 and "overlap" in str(e.value)


# 272 = 17 * 2^4 is the smallest mesh above 256 x 256 that the library builds
# (258 ... 270 coarsen to more than 25 x 25 cells and are refused at creation)
@pytest.mark.parametrize("n", [272, 512])
def test_noalloc_mass_solve_rejects_large_meshes(torch, n):
    ctx = chnss.Context(chnss.Mesh(n), inputs.default_params())
    b = torch.ones(ctx.mesh.N1, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(chnss.ChnssError) as e:
        ctx.mass_solve_noalloc(b, x)
    assert e.value.status == 1 and "256 x 256" in str(e.value)
