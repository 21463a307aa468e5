"""The Gram-Schmidt kernels of FGMRES (classical Gram-Schmidt applied twice)
in FP64 and in double-FP32 arithmetic (ortho = 1: every value a pair of
FP32 numbers, Dekker's exact product and Knuth's two-sum), through
chnss_debug_cgs2 on adversarial vectors, and whole steps with ortho = 1
against the oracle (whose Gram-Schmidt is FP64)."""
import math

import numpy as np
import pytest

from oracle.step import Oracle
from solve_compare import compare_solves, rel
from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _two_prod(a, b):
    """Exact products a * b = p + e of FP64 arrays (Dekker's splitting)."""
    c = 134217729.0                      # 2^27 + 1
    def split(x):
        t = c * x
        hi = t - (t - x)
        return hi, x - hi
    ah, al = split(a)
    bh, bl = split(b)
    p = a * b
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_dot(a, b):
    p, e = _two_prod(a, b)
    return math.fsum(np.concatenate([p, e]).tolist())


def _adversarial(n, k, seed):
    """k orthonormal vectors with entries over twelve orders of magnitude, and
    a w that is 1e8 times a combination of them plus an O(1) remainder
    orthogonal to them: pass 1 cancels eight digits, pass 2 must clean up."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((n, k)) * np.exp(g.uniform(-6, 6, (n, 1)) * np.log(10))
    Q, _ = np.linalg.qr(A)
    V = np.ascontiguousarray(Q.T)
    r = g.standard_normal(n) * np.exp(g.uniform(-3, 3, n) * np.log(10))
    r -= V.T @ (V @ r)
    r -= V.T @ (V @ r)
    w = 1e8 * (V.T @ g.standard_normal(k)) + r
    return V, w


@pytest.mark.parametrize("n,k", [(400_003, 7), (400_003, 31), (1_001, 16)])
def test_gram_schmidt_dots_and_basis_vector(torch, n, k):
    V, w = _adversarial(n, k, seed=n + k)
    ld = n + (n % 2)
    Vd = torch.zeros((k, ld), dtype=torch.float64, device="cuda")
    Vd[:, :n] = torch.as_tensor(V, device="cuda")
    wd = torch.as_tensor(w, device="cuda")
    scale = [math.fsum(np.abs(V[j] * w).tolist()) for j in range(k)]
    exact = np.array([exact_dot(V[j], w) for j in range(k)])
    out, h_norm2 = {}, []
    for arith in (0, 1):
        h1, h2, nrm2, vout = chnss.debug_cgs2(Vd, wd, arith)
        v = vout.cpu().numpy()
        # pass-1 dots against exact sums, relative to sum |v_i w_i|
        err = np.max(np.abs(h1 - exact) / np.array(scale))
        assert err <= 1e-13, (arith, err)
        # the next basis vector is unit and orthogonal to V
        assert abs(np.linalg.norm(v) - 1.0) <= 1e-12, arith
        assert np.max(np.abs(V @ v)) <= 1e-12, arith
        out[arith] = (h1, h2, v)
        h_norm2.append(nrm2)
    # the two arithmetics agree on the result: the dots to their rounding
    # level, the basis vector to the rounding of w - V h1 (relative u ||w||)
    # magnified by the cancellation ||w|| / ||w'|| (1e8 here), u = 2^-48 for
    # the pairs
    assert np.max(np.abs(out[0][0] - out[1][0]) / np.array(scale)) <= 1e-13
    cancel = np.linalg.norm(w) / math.sqrt(h_norm2[0])
    assert rel(out[1][2], out[0][2]) <= 64 * 2.0 ** -48 * cancel, (rel(out[1][2], out[0][2]), cancel)


def test_gram_schmidt_input_checks(torch):
    V = torch.zeros((40, 8), dtype=torch.float64, device="cuda")
    w = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(chnss.ChnssError):
        chnss.debug_cgs2(V, w, 1)                      # k = 40 > 31
    with pytest.raises(chnss.ChnssError):
        chnss.debug_cgs2(V[:4], w, 2)                  # unknown arithmetic


@pytest.mark.parametrize("n", [32, 20])
def test_step_with_double_fp32_gram_schmidt_matches_oracle(torch, n):
    """FP64 preconditioners and operators, Gram-Schmidt in double-FP32: every
    solve within 1e-9 of the FP64 oracle and iterations within one."""
    p = dict(inputs.default_params(), ortho=1)
    o = Oracle(n, dict(p, ortho=0))
    ctx = chnss.Context(chnss.Mesh(n), p)
    st = inputs.initial_state(n, seed=n + 7)
    for k in range(2):
        ref, rinfo = o.step(st)
        out, info, status = ctx.step(chnss.state_to_device(st))
        assert status == 0
        got = chnss.state_to_numpy(out)
        compare_solves(got, info, ref, rinfo, st, p, lambda q: Oracle(n, q), where=(n, k))
        assert rel(got["mu"][3], ref["mu"][3]) <= 1e-9
        st = ref


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_step_with_double_fp32_gram_schmidt(torch, precision):
    """The mixed-precision gates with ortho = 1: the 1e-8 relative residual is
    reached, and with the outer FGMRES at 1e-10 the step is within 1e-6 of the
    oracle (solved to 1e-12)."""
    n = 32
    params = dict(inputs.default_params(), ortho=1)
    o = Oracle(n, dict(params, rtol=1e-12))
    ctx8 = chnss.Context(chnss.Mesh(n), dict(params, precision=precision))
    ctx10 = chnss.Context(chnss.Mesh(n), dict(params, precision=precision, rtol=1e-10))
    st = inputs.initial_state(n, seed=15)
    for _ in range(2):
        ref, _ = o.step(st)
        dev = chnss.state_to_device(st)
        out8, info8, st8 = ctx8.step(dev)
        out10, _, st10 = ctx10.step(dev)
        assert st8 == 0 and st10 == 0
        for name, i in info8.items():
            if name != "mu_a":
                assert i["converged"] and i["rel_residual"] <= 1e-8, (name, i)
        g10 = chnss.state_to_numpy(out10)
        for key in ("phi", "mu", "Phi_v", "v", "p"):
            assert rel(g10[key], ref[key]) <= 1e-6, key
        st = ref


def test_three_d_step_with_double_fp32_gram_schmidt(torch):
    from oracle import three_d as t3
    n = 4
    p = dict(inputs.default_params(), alpha=[1e-2] * 4, ortho=1)
    o = t3.Oracle3D(n, dict(p, ortho=0))
    ctx = chnss.Context3(n, p)
    st = inputs.initial_state_3d(n, seed=1)
    ref, rinfo = o.step(st)
    out, info, status = ctx.step(chnss.state_to_device(st))
    assert status == 0
    compare_solves(chnss.state_to_numpy(out), info, ref, rinfo, st, p, lambda q: t3.Oracle3D(n, q))
