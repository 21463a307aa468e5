"""The SELL-C-sigma SpMV kernels one by one (chnss_debug_spmv, the same
dispatch as the solvers): scalar rows, 2x2 and 3x3 blocks, FP64 / FP32 /
BF16 values, the four epilogues (plain, residual, add, Chebyshev step),
against a numpy FP64 product of the same (rounded) inputs.  The random
patterns are chosen to reach every launch form: one thread per row (short
rows or many slices), several warps per slice (few slices of wide rows, up
to 32 warps), a ragged last slice, empty rows."""
import numpy as np
import pytest

from paper_2501_11767_gb300 import chnss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _pattern(rng, n, lo, hi, empty=0.0):
    """n rows, each with a random number of distinct ascending columns in
    [lo, hi] (some rows empty with probability `empty`), square."""
    rows = []
    for i in range(n):
        k = 0 if rng.random() < empty else int(rng.integers(lo, hi + 1))
        # distinct columns near the diagonal (a banded mesh-like pattern) for long
        # patterns, anywhere for short ones
        pool = n if n <= 4096 else min(n, 512)
        c = rng.choice(pool, size=min(k, pool), replace=False)
        if pool < n:
            c = (c + max(0, min(i - pool // 2, n - pool)))
        rows.append(np.sort(c))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    return rowptr, np.concatenate(rows).astype(np.int32) if rowptr[-1] else np.zeros(0, np.int32)


def _round(a, precision, torch, values=False):
    if precision == 0:
        return a
    t = torch.as_tensor(a, dtype=torch.float32)
    if precision == 2 and values:
        t = t.to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def _dense_blocks(rowptr, col, val, bs, n):
    """The block matrix as a scipy CSR over the n * bs interleaved dofs."""
    import scipy.sparse as sp
    node = np.repeat(np.arange(n), np.diff(rowptr))
    rows, cols, vals = [], [], []
    for r in range(bs):
        for d in range(bs):
            rows.append(node * bs + r)
            cols.append(col.astype(np.int64) * bs + d)
            vals.append(val[:, r * bs + d])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n * bs, n * bs))


CASES = {
    # name: (nodes, min entries, max entries, fraction of empty rows)
    "short_rows": (3001, 1, 8, 0.05),       # scalar: rows of at most 8 entries
    "medium_rows": (2083, 9, 11, 0.0),      # scalar one-thread-per-row form
    "wide_few_slices": (97, 20, 90, 0.1),   # few slices of wide rows: many warps per slice
    "wide_many": (12001, 12, 30, 0.02),     # wide rows, hundreds of slices
    "very_wide": (400, 256, 380, 0.0),      # 13 slices of 256+ entries: up to 32 warps per slice
    "narrow_many": (240001, 4, 15, 0.0),    # more slices than one wave of warps: one thread per row
}


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_spmv_matches_numpy(torch, layout, case):
    n, lo, hi, empty = CASES[case]
    bs = (1, 2, 3)[layout]
    rng = np.random.default_rng(100 * layout + sorted(CASES).index(case))
    rowptr, col = _pattern(rng, n, lo, hi, empty)
    nnz = len(col)
    val = rng.standard_normal((nnz, bs * bs)) * np.exp(rng.uniform(-2, 2, (nnz, 1)))
    x, b, w = (rng.standard_normal(n * bs) for _ in range(3))
    dinv = 1.0 / (1.0 + rng.random(n * bs))
    coef = np.array([0.7, -0.3, 1.3])
    y0 = rng.standard_normal(n * bs)
    seen = set()
    for precision in (0, 1, 2):
        vr = _round(val, precision, torch, values=True)
        xr, br, wr, dr, yr = (_round(a, precision, torch) for a in (x, b, w, dinv, y0))
        A = _dense_blocks(rowptr, col, vr, bs, n)
        Ax = A @ xr
        scale = abs(A) @ abs(xr) + 1e-300                       # sum |a_ij x_j| per row
        # FP64: a few roundings of the row sum; FP32 vectors and sums: 2^-24 per term
        tol = 1e-13 if precision == 0 else 64 * 2.0 ** -24 * max(hi, 1) * bs
        for mode in range(4):
            got, k = chnss.debug_spmv(layout, precision, mode, rowptr, col, val, x, b=b,
                                      w=w if mode == 3 else None, dinv=dinv, coef=coef, y=y0)
            seen.add(k)
            if mode == 0:
                want, sc = Ax, scale
            elif mode == 1:
                want, sc = br - Ax, scale + abs(br)
            elif mode == 2:
                want, sc = yr + Ax, scale + abs(yr)
            else:
                want = coef[0] * xr + coef[1] * wr + coef[2] * dr * (br - Ax)
                sc = abs(coef[0] * xr) + abs(coef[1] * wr) + abs(coef[2] * dr) * (abs(br) + scale)
            err = np.max(np.abs(got - want) / sc)
            assert err <= tol, (layout, case, precision, mode, k, err)
    if case in ("wide_few_slices", "very_wide"):
        assert max(seen) > 1, seen            # the several-warps-per-slice forms ran
    if case == "very_wide" and layout == 0:
        assert seen == {32}, seen
    if case in ("short_rows", "medium_rows") and layout == 0 or case == "narrow_many":
        assert seen == {1}, seen


def test_spmv_argument_checks(torch):
    rowptr, col = np.array([0, 1, 2]), np.array([0, 1])
    val, x = np.ones(2), np.ones(2)
    with pytest.raises(chnss.ChnssError):
        chnss.debug_spmv(3, 0, 0, rowptr, col, val, x)           # unknown layout
    with pytest.raises(chnss.ChnssError):
        chnss.debug_spmv(0, 0, 3, rowptr, col, val, x, b=x)      # Chebyshev without dinv / coef
    with pytest.raises(chnss.ChnssError):
        chnss.debug_spmv(0, 0, 0, rowptr, np.array([0, 5]), val, x)   # column out of range
