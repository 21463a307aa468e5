"""Smoothed-aggregation algebraic multigrid (oracle; TEST INFRASTRUCTURE).

Sec. 5 of the paper approximates its block inverses with PyAMG's algebraic
multigrid: smoothed aggregation (SA) for the nonsymmetric Cahn-Hilliard
blocks M + tau C, and SA for every Navier-Stokes block of the 3D runs.
This module restates the SA setup of Vanek, Mandel and Brezina (Computing
56, 1996) for a scalar operator with the constant near-null space, with
the parallel aggregation of Bell, Dalton and Olson (SIAM J. Sci. Comput. 34,
2012), one level at a time:

  1. strength graph: i != j are joined when |a_ij| or |a_ji| is at least
     theta sqrt(|a_ii a_jj|) (symmetrised, so the graph is undirected);
     theta = 0 (PyAMG's symmetric strength default) joins every pair with a
     stored entry;
  2. roots: a maximal independent set of distance 2 in that graph, built in
     synchronous rounds.  Node i carries the key (state, priority, i),
     state 0 removed < 1 undecided < 2 root, priority the 30 leading bits of
     SplitMix64 output number (level << 32) + i.  Each round every node
     takes the largest key over its closed neighbourhood, twice (so over
     distance 2); an undecided node whose result is its own key becomes a
     root, one whose result belongs to a root is removed;
  3. aggregates: the roots in increasing node order are aggregates 0, 1, ...;
     pass 1: every other node adjacent to a root joins the adjacent root of
     largest (priority, index); pass 2: every node still alone joins the
     pass-1 neighbour of largest (priority, index);
  4. tentative prolongator T[i, agg(i)] = 1 / sqrt(|agg(i)|);
  5. smoothed prolongator P = T - omega D^-1 (A T), omega = 4 / (3 hi), hi
     the level's bound of the spectral radius of D^-1 A: the smaller of the
     Gershgorin bound max_i sum_j |a_ij| / |a_ii| and 1.1 times the estimate
     of POWER_STEPS power iterations from a +-1 start vector (SplitMix64
     output number ((level + 64) << 32) + i decides the sign of entry i);
     the Gershgorin bound alone overestimates the coarse operators' radius
     by about half, which would leave part of their spectrum unsmoothed;
  6. Galerkin coarse operator A_c = P^T (A P).
P and A_c keep every structurally non-zero entry (the pattern of the
products of the patterns), so that a value that cancels to zero in one
rounding order is still stored.  Levels are added while a level has more
than COARSE_ROWS rows and aggregation shrinks it, up to MAX_LEVELS levels.
The cycle is the V-cycle of oracle.mg.MG with these operators and
prolongations (Chebyshev-Jacobi smoothing on [hi / 4, hi] with the same
per-level hi, restriction P^T).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from paper_2501_11767_gb300.inputs import splitmix64

from .mg import MG

COARSE_ROWS = 64
MAX_LEVELS = 12
POWER_STEPS = 10
POWER_SAFETY = 1.1
STATE_REMOVED, STATE_UNDECIDED, STATE_ROOT = 0, 1, 2


def _csr(A) -> sp.csr_matrix:
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sort_indices()
    return A


def strength_graph(A, theta: float = 0.0) -> sp.csr_matrix:
    """Boolean pattern (no diagonal) of the symmetrised strength graph.
    A must be square with a stored diagonal and a structurally symmetric
    pattern."""
    A = _csr(A)
    n = A.shape[0]
    d = A.diagonal()
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    cols = A.indices
    vals = np.abs(A.data)
    # |a_ji| at the position of a_ij
    AT = _csr(A.T)
    if not np.array_equal(AT.indptr, A.indptr) or not np.array_equal(AT.indices, A.indices):
        raise ValueError("the pattern of A must be structurally symmetric")
    valsT = np.abs(AT.data)
    bound = theta * np.sqrt(np.abs(d[rows] * d[cols]))
    keep = (rows != cols) & ((vals >= bound) | (valsT >= bound))
    S = sp.csr_matrix((np.ones(int(keep.sum())), (rows[keep], cols[keep])), shape=(n, n))
    S.sort_indices()
    return S


def priorities(n: int, level: int) -> np.ndarray:
    """The 30-bit priority of node i < n on a level (uint64 array)."""
    keys = (np.uint64(level) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
    return splitmix64(keys) >> np.uint64(34)


def mis2(S, level: int = 0):
    """Roots (bool array) of a maximal distance-2 independent set of the
    graph S, and the number of rounds taken."""
    S = sp.csr_matrix(S)
    n = S.shape[0]
    closed = (S + sp.identity(n, format="csr")).tocsr()
    closed.sort_indices()
    ptr, nb = closed.indptr, closed.indices
    idx = np.arange(n, dtype=np.uint64)
    base = (priorities(n, level) << np.uint64(32)) | idx
    state = np.full(n, STATE_UNDECIDED, dtype=np.uint64)
    rounds = 0
    while np.any(state == STATE_UNDECIDED):
        key = (state << np.uint64(62)) | base
        m1 = np.maximum.reduceat(key[nb], ptr[:-1])
        m2 = np.maximum.reduceat(m1[nb], ptr[:-1])
        und = state == STATE_UNDECIDED
        new = state.copy()
        new[und & (m2 == key)] = STATE_ROOT
        new[und & (m2 != key) & ((m2 >> np.uint64(62)) == STATE_ROOT)] = STATE_REMOVED
        state = new
        rounds += 1
    return state == STATE_ROOT, rounds


def aggregate(S, level: int = 0):
    """Aggregate index of every node (int array) and the aggregate count."""
    S = sp.csr_matrix(S)
    n = S.shape[0]
    roots, _ = mis2(S, level)
    base = (priorities(n, level) << np.uint64(32)) | np.arange(n, dtype=np.uint64)
    agg = np.full(n, -1, dtype=np.int64)
    agg[roots] = np.arange(int(roots.sum()))
    ptr, nb = S.indptr, S.indices
    first = agg.copy()
    for i in range(n):                              # pass 1: adjacent roots
        if roots[i]:
            continue
        cand = [j for j in nb[ptr[i]:ptr[i + 1]] if roots[j]]
        if cand:
            first[i] = agg[max(cand, key=lambda j: base[j])]
    second = first.copy()
    for i in range(n):                              # pass 2: pass-1 neighbours
        if first[i] >= 0:
            continue
        cand = [j for j in nb[ptr[i]:ptr[i + 1]] if first[j] >= 0]
        if not cand:
            raise RuntimeError("node %d is not within distance 2 of a root" % i)
        second[i] = first[max(cand, key=lambda j: base[j])]
    return second, int(roots.sum())


def tentative(agg, nagg: int) -> sp.csr_matrix:
    """T[i, agg(i)] = 1 / sqrt(|agg(i)|): orthonormal columns, T sqrt(sizes) = 1."""
    n = agg.shape[0]
    size = np.bincount(agg, minlength=nagg).astype(np.float64)
    t = 1.0 / np.sqrt(size[agg])
    return sp.csr_matrix((t, (np.arange(n), agg)), shape=(n, nagg))


def _on_pattern(values, pattern) -> sp.csr_matrix:
    """values (sparse) read at every position of pattern (sparse), zero where
    values has no entry: keeps structurally non-zero but cancelled entries."""
    pattern = sp.csr_matrix(pattern)
    pattern.sort_indices()
    rows = np.repeat(np.arange(pattern.shape[0]), np.diff(pattern.indptr))
    v = np.asarray(sp.csr_matrix(values)[rows, pattern.indices]).ravel()
    return sp.csr_matrix((v, pattern.indices.copy(), pattern.indptr.copy()), shape=pattern.shape)


def _ones(A) -> sp.csr_matrix:
    B = sp.csr_matrix(A, copy=True)
    B.data[:] = 1.0
    return B


def gershgorin(A) -> float:
    """hi = max_i sum_j |a_ij| / |a_ii| (bounds the spectrum of D^-1 A)."""
    A = _csr(A)
    return float(np.max(np.asarray(abs(A).sum(axis=1)).ravel() / np.abs(A.diagonal())))


def spectral_bound(A, level: int) -> float:
    """min(Gershgorin bound, POWER_SAFETY * power estimate) of rho(D^-1 A):
    x = x0 / ||x0||, then POWER_STEPS times y = D^-1 (A x), x = y / ||y||;
    the estimate is the last ||y||."""
    A = _csr(A)
    n = A.shape[0]
    dinv = 1.0 / A.diagonal()
    keys = (np.uint64(level + 64) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
    x = np.where((splitmix64(keys) >> np.uint64(63)) == 1, 1.0, -1.0)
    x = x / np.sqrt(x @ x)
    nrm = 0.0
    for _ in range(POWER_STEPS):
        y = dinv * (A @ x)
        nrm = np.sqrt(y @ y)
        x = y / nrm
    return min(gershgorin(A), POWER_SAFETY * float(nrm))


def smoothed_prolongator(A, agg, nagg: int, hi: float = None) -> sp.csr_matrix:
    """P = T - omega D^-1 (A T), omega = 4 / (3 hi), on the structural pattern
    of A T (hi: the Gershgorin bound unless given)."""
    A = _csr(A)
    T = tentative(agg, nagg)
    omega = 4.0 / (3.0 * (gershgorin(A) if hi is None else hi))
    s = omega * (1.0 / A.diagonal())
    AT = A @ T
    P = T - sp.diags(s) @ AT
    return _on_pattern(P, _ones(A) @ _ones(T))


def galerkin(A, P) -> sp.csr_matrix:
    """A_c = P^T (A P) on the structural pattern of the product."""
    A = _csr(A)
    P = _csr(P)
    AP = A @ P
    Ac = _csr(P.T) @ AP
    return _on_pattern(Ac, _ones(P).T @ (_ones(A) @ _ones(P)))


class SAHierarchy:
    """The SA levels of a square matrix A: mats[l] (CSR, FP64), prolongs[l]
    (level l+1 -> l), aggs[l] (aggregate of every node of level l), his[l]
    (spectral bound of D^-1 A_l: prolongator smoothing and smoother)."""

    def __init__(self, A, theta: float = 0.0, coarse_rows: int = COARSE_ROWS, max_levels: int = MAX_LEVELS):
        A = _csr(A)
        self.mats, self.prolongs, self.aggs = [A], [], []
        self.his = [spectral_bound(A, 0)]
        while A.shape[0] > coarse_rows and len(self.mats) < max_levels:
            level = len(self.mats) - 1
            S = strength_graph(A, theta)
            agg, nagg = aggregate(S, level)
            if nagg >= A.shape[0]:
                break
            P = smoothed_prolongator(A, agg, nagg, self.his[level])
            A = galerkin(A, P)
            self.aggs.append(agg)
            self.prolongs.append(P)
            self.mats.append(A)
            self.his.append(spectral_bound(A, level + 1))
        self.mg = MG(self.mats, self.prolongs, his=self.his)

    def __call__(self, b):
        """One V-cycle (oracle.mg.MG) applied to b."""
        return self.mg(b)
