"""GPU smoothed-aggregation AMG (chnss_amg_*) against the oracle
(oracle/amg.py), through the C ABI: per level the aggregates (bit-exact:
integer work), the patterns of A_l and P_l (exact), their values and the
spectral bounds (FP64 rounding order only), one V-cycle, and the
SA-preconditioned FGMRES solve (iterate against iterate).  Inputs: seeded
unstructured triangulations of the unit square (the meshes SA is for) and
the Cahn-Hilliard block M + tau C(v) assembled by the library itself for a
step of the thin-film model."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg, fem
from oracle.krylov import fgmres
from oracle.mesh import TriMesh
from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu

VAL_TOL = 1e-13       # level values: FP64, only the summation order may differ
CYCLE_TOL = 1e-11     # one V-cycle (FP64 hierarchy)
SOLVE_TOL = 1e-9      # per solve, as the step's parity tests


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _unstructured(n, seed=0, tau=1.0, wind=None):
    x, tri = inputs.unstructured_square(n, seed)
    m = TriMesh(x, tri)
    A = fem.mass_p1(m) + tau * fem.stiffness_p1(m)
    if wind is not None:
        A = A + tau * fem.convection_p1_wind(m, np.tile(wind, (m.N1, 1)))
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A


def _step_block(n, params=None):
    """L = M + tau C(v) of a thin-film step (export of the assembled matrix)."""
    ctx = chnss.Context(chnss.Mesh(n), params or inputs.default_params())
    st = inputs.initial_state(n, seed=4)
    # a non-zero velocity so that C(v) is present: a swirl on the P2 nodes
    N2 = (2 * n + 1) ** 2
    g = np.linspace(0.0, 1.0, 2 * n + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    v = np.stack([np.sin(np.pi * X) * np.cos(np.pi * Y), -np.cos(np.pi * X) * np.sin(np.pi * Y)], axis=-1)
    st["v"] = 0.5 * v.reshape(N2, 2).ravel()
    ctx.assemble(chnss.state_to_device(st))
    rp, col, val = ctx.export_csr(0)
    A = sp.csr_matrix((val, col, rp), shape=(len(rp) - 1, len(rp) - 1))
    A.sort_indices()
    return A


def _device(torch, A):
    return (torch.as_tensor(A.indptr.astype(np.int32), device="cuda"),
            torch.as_tensor(A.indices.astype(np.int32), device="cuda"),
            torch.as_tensor(A.data, dtype=torch.float64, device="cuda"))


def _compare_hierarchy(h, H):
    levels = h.levels()
    assert len(levels) == len(H.mats), (levels, [m.shape for m in H.mats])
    for l, Al in enumerate(H.mats):
        got = h.export_level(l)
        assert np.array_equal(got["a_rowptr"], Al.indptr) and np.array_equal(got["a_col"], Al.indices), l
        scale = np.abs(Al.data).max()
        assert np.abs(got["a_val"] - Al.data).max() <= VAL_TOL * scale, l
        assert abs(got["hi"] - H.his[l]) <= 1e-12 * H.his[l], (l, got["hi"], H.his[l])
        if l < len(H.mats) - 1:
            assert np.array_equal(got["agg"], H.aggs[l]), l           # integer work: bit-exact
            P = H.prolongs[l]
            assert np.array_equal(got["p_rowptr"], P.indptr) and np.array_equal(got["p_col"], P.indices), l
            assert np.abs(got["p_val"] - P.data).max() <= VAL_TOL * np.abs(P.data).max(), l


CASES = [("unstructured24", lambda: _unstructured(24, seed=1)),
         ("unstructured64_convection", lambda: _unstructured(64, seed=2, tau=0.05, wind=(2.0, 1.0))),
         ("unstructured160", lambda: _unstructured(160, seed=3)),        # 25 921 rows: several scan chunks
         ("ch_block_64", lambda: _step_block(64))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_hierarchy_matches_oracle(torch, name, make):
    A = make()
    H = amg.SAHierarchy(A)
    h = chnss.Amg(*_device(torch, A))
    _compare_hierarchy(h, H)


@pytest.mark.parametrize("name,make", CASES[:2] + CASES[3:], ids=[c[0] for c in CASES[:2] + CASES[3:]])
def test_vcycle_matches_oracle(torch, name, make):
    A = make()
    H = amg.SAHierarchy(A)
    b = np.cos(np.arange(A.shape[0]) * 0.731) + 0.2
    for precision, tol in ((0, CYCLE_TOL), (1, 2e-5)):
        h = chnss.Amg(*_device(torch, A), precision=precision)
        x = h.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
        want = H(b)
        err = np.linalg.norm(x - want) / np.linalg.norm(want)
        assert err <= tol, (precision, err)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_solve_matches_oracle(torch, name, make):
    A = make()
    H = amg.SAHierarchy(A)
    b = np.sin(np.arange(A.shape[0]) * 0.37) + 0.5
    h = chnss.Amg(*_device(torch, A))
    x, info, st = h.solve(torch.as_tensor(b, device="cuda"), rtol=1e-8)
    assert st == 0 and info["converged"]
    x = x.cpu().numpy()
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    ref, rinfo = fgmres(lambda y: A @ y, H, b, rtol=1e-8, restart=30, maxit=500)
    assert abs(info["iters"] - rinfo["iters"]) <= 1, (info, rinfo)
    if info["iters"] != rinfo["iters"]:         # the oracle's iterate at the GPU's count
        ref, _ = fgmres(lambda y: A @ y, H, b, rtol=0.0, atol=0.0, restart=30, maxit=info["iters"])
    assert np.linalg.norm(x - ref) <= SOLVE_TOL * np.linalg.norm(ref), info


def test_mixed_precision_solve_reaches_the_residual(torch):
    A = _unstructured(96, seed=5, tau=0.05, wind=(1.0, -2.0))
    b = np.sin(np.arange(A.shape[0]) * 0.11)
    h64 = chnss.Amg(*_device(torch, A), precision=0)
    h32 = chnss.Amg(*_device(torch, A), precision=1)
    bt = torch.as_tensor(b, device="cuda")
    x64, i64, _ = h64.solve(bt, rtol=1e-10)
    x32, i32, _ = h32.solve(bt, rtol=1e-10)
    assert i32["converged"] and i32["iters"] <= i64["iters"] + 2, (i64, i32)
    x = x32.cpu().numpy()
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)


def test_update_equals_fresh_setup_and_is_deterministic(torch):
    """chnss_amg_update on new values (same pattern) gives bitwise the
    hierarchy and V-cycle of a handle created with those values."""
    A1 = _unstructured(48, seed=6, tau=0.05, wind=(1.0, 0.0))
    A2 = _unstructured(48, seed=6, tau=0.2, wind=(-0.5, 1.5))
    assert np.array_equal(A1.indices, A2.indices)
    rp, col, v1 = _device(torch, A1)
    v2 = torch.as_tensor(A2.data, dtype=torch.float64, device="cuda")
    h = chnss.Amg(rp, col, v1)
    h.update(v2)
    fresh = chnss.Amg(rp, col, v2)
    again = chnss.Amg(rp, col, v2)
    b = torch.as_tensor(np.cos(np.arange(A1.shape[0]) * 0.3), device="cuda")
    xs = [g.vcycle(b) for g in (h, fresh, again)]
    assert torch.equal(xs[0], xs[1]) and torch.equal(xs[1], xs[2])
    for l in range(len(h.levels())):
        a, c = h.export_level(l), fresh.export_level(l)
        for k in a:
            assert np.array_equal(a[k], c[k]), (l, k)


def test_refuses_bad_patterns(torch):
    A = _unstructured(8, seed=0)
    rp, col, val = _device(torch, A)
    # a structurally unsymmetric pattern: drop one off-diagonal entry
    B = A.tolil()
    i, j = 3, int(A.indices[A.indptr[3]] if A.indices[A.indptr[3]] != 3 else A.indices[A.indptr[3] + 1])
    B[i, j] = 0.0
    B = sp.csr_matrix(B)
    B.eliminate_zeros()
    with pytest.raises(chnss.ChnssError) as e:
        chnss.Amg(*_device(torch, B))
    assert e.value.status == 1 and "symmetric" in str(e.value)
    # a missing diagonal
    C = A.tolil()
    C[5, 5] = 0.0
    C = sp.csr_matrix(C)
    C.eliminate_zeros()
    with pytest.raises(chnss.ChnssError) as e:
        chnss.Amg(*_device(torch, C))
    assert e.value.status == 1 and "diagonal" in str(e.value)
    # unsorted columns in a row
    col2 = col.clone()
    r0, r1 = int(A.indptr[4]), int(A.indptr[5])
    col2[r0:r1] = col2[r0:r1].flip(0)
    with pytest.raises(chnss.ChnssError) as e:
        chnss.Amg(rp, col2, val)
    assert e.value.status == 1 and "sorted" in str(e.value)


def test_full_size_ch_block_matches_oracle(torch):
    """The bench's size: the 1024^2 CH block M + tau C(v) (1 050 625 rows).
    The oracle's own setup is cheap enough here (numpy rounds, one Python
    pass per aggregation rule), so every level, one V-cycle and the
    SA-preconditioned solve are compared at the tolerances of the small
    cases.  Parameters of the 1024^2 workload (tau = 5e-4): with tau = 1e-3
    the swirl's cell Courant number tau |v| / h reaches 0.5 and the SA
    V-cycle with its Chebyshev-Jacobi smoother no longer preconditions the
    block (the oracle's FGMRES, too, is at 1e-2 after 120 iterations)."""
    A = _step_block(1024, inputs.workload("film1024_mixed")["params"])
    H = amg.SAHierarchy(A)
    h = chnss.Amg(*_device(torch, A))
    _compare_hierarchy(h, H)
    b = np.cos(np.arange(A.shape[0]) * 0.731) + 0.2
    x = h.vcycle(torch.as_tensor(b, device="cuda")).cpu().numpy()
    want = H(b)
    assert np.linalg.norm(x - want) <= CYCLE_TOL * np.linalg.norm(want)
    xs, info, st = h.solve(torch.as_tensor(b, device="cuda"), rtol=1e-8)
    ref, rinfo = fgmres(lambda y: A @ y, H, b, rtol=1e-8, restart=30, maxit=500)
    assert st == 0 and abs(info["iters"] - rinfo["iters"]) <= 1, (info, rinfo)
    if info["iters"] != rinfo["iters"]:
        ref, _ = fgmres(lambda y: A @ y, H, b, rtol=0.0, atol=0.0, restart=30, maxit=info["iters"])
    assert np.linalg.norm(xs.cpu().numpy() - ref) <= SOLVE_TOL * np.linalg.norm(ref), info


@pytest.mark.parametrize("n", [32, 64])
def test_step_with_sa_ac_block_matches_oracle(torch, n):
    """params amg = 1: the Allen-Cahn block's multigrid is the device smoothed
    aggregation of the assembled AC matrix, set up again in every step
    (Sec. 5 takes PyAMG for this block).  Every solve of two FP64 steps
    against the oracle step with the same option (oracle.amg for that block)."""
    from oracle.step import Oracle
    from solve_compare import compare_solves
    p = dict(inputs.default_params(), amg=1)
    o = Oracle(n, p)
    ctx = chnss.Context(chnss.Mesh(n), p)
    st = inputs.initial_state(n, seed=2)
    for k in range(2):
        ref, rinfo = o.step(st)
        out, info, status = ctx.step(chnss.state_to_device(st))
        torch.cuda.synchronize()
        assert status == 0
        compare_solves(chnss.state_to_numpy(out), info, ref, rinfo, st, p, lambda q: Oracle(n, q), where=k)
        st = ref


def test_step_with_sa_ac_block_graph_and_mixed(torch):
    """The same option in FP32 hierarchies with double-FP32 Gram-Schmidt: the
    one-graph step (the SA re-setup recorded with the assembly) equals the
    host-driven step bitwise, and every solve meets its stopping rule."""
    n = 64
    p = dict(inputs.default_params(), amg=1, precision=1, ortho=1)
    st0 = chnss.state_to_device(inputs.initial_state(n, seed=3))
    outs = []
    for mode in (0, 1):
        ctx = chnss.Context(chnss.Mesh(n), p)
        ctx.set_step_mode(mode)
        a = {k: v.clone() for k, v in st0.items()}
        for _ in range(2):
            a, info, status = ctx.step(a)
            assert status == 0 and all(info[k]["converged"] for k in info), info
        torch.cuda.synchronize()
        outs.append(a)
    for k in outs[0]:
        assert torch.equal(outs[0][k], outs[1][k]), k
