"""Pins of the smoothed-aggregation oracle (oracle/amg.py) against what the
method and the mathematics fix: the distance-2 independent set checked by
brute-force graph distances, the aggregation rules, the orthonormal
tentative prolongator, a hand-derived smoothed prolongator of the 1D
Laplacian, the Galerkin product against dense algebra, and mesh-robust
preconditioning on unstructured meshes (which a planted sign mistake in the
prolongator smoothing breaks)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

from oracle import amg, fem
from oracle.krylov import fgmres
from oracle.mesh import TriMesh
from paper_2501_11767_gb300 import inputs


def _mesh(n, seed=0):
    x, tri = inputs.unstructured_square(n, seed)
    return TriMesh(x, tri)


def _operator(n, seed=0, tau=1e-2, wind=None):
    m = _mesh(n, seed)
    A = fem.mass_p1(m) + tau * fem.stiffness_p1(m)
    if wind is not None:
        A = A + tau * fem.convection_p1_wind(m, np.tile(wind, (m.N1, 1)))
    return sp.csr_matrix(A), m


def _graphs():
    out = {}
    A, _ = _operator(10, seed=3)
    out["unstructured"] = amg.strength_graph(A)
    n = 50
    path = sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")
    out["path"] = path
    g = sp.kron(sp.identity(8), sp.diags([1.0, 1.0], [-1, 1], shape=(8, 8))) + \
        sp.kron(sp.diags([1.0, 1.0], [-1, 1], shape=(8, 8)), sp.identity(8))
    out["grid"] = sp.csr_matrix(g)
    # two components and three isolated nodes
    iso = sp.block_diag([path[:7, :7], sp.csr_matrix((3, 3)), out["grid"][:20, :20]], format="csr")
    out["isolated"] = iso
    return out


@pytest.mark.parametrize("name", ["unstructured", "path", "grid", "isolated"])
def test_mis2_independent_and_maximal_by_brute_force(name):
    S = _graphs()[name]
    roots, rounds = amg.mis2(S, level=1)
    D = shortest_path(S, unweighted=True, directed=False)
    r = np.flatnonzero(roots)
    assert len(r) > 0 and rounds >= 1
    # independence: roots at graph distance >= 3 from each other
    sub = D[np.ix_(r, r)]
    np.fill_diagonal(sub, np.inf)
    assert sub.min() >= 3
    # maximality: every other node within distance 2 of a root
    assert np.all(D[:, r].min(axis=1) <= 2)


@pytest.mark.parametrize("name", ["unstructured", "path", "grid", "isolated"])
def test_aggregation_rules(name):
    S = _graphs()[name]
    n = S.shape[0]
    agg, nagg = amg.aggregate(S, level=0)
    roots, _ = amg.mis2(S, level=0)
    D = shortest_path(S, unweighted=True, directed=False)
    base = (amg.priorities(n, 0) << np.uint64(32)) | np.arange(n, dtype=np.uint64)
    assert agg.min() >= 0 and agg.max() == nagg - 1
    r = np.flatnonzero(roots)
    assert np.array_equal(agg[r], np.arange(nagg))            # roots numbered in node order
    for i in range(n):
        root = r[agg[i]]
        assert D[i, root] <= 2                                 # member within distance 2 of its root
        adj_roots = [j for j in S.indices[S.indptr[i]:S.indptr[i + 1]] if roots[j]]
        if not roots[i] and adj_roots:                         # pass 1: largest adjacent root
            assert root == max(adj_roots, key=lambda j: base[j])


def test_tentative_prolongator_orthonormal():
    A, _ = _operator(12)
    agg, nagg = amg.aggregate(amg.strength_graph(A))
    T = amg.tentative(agg, nagg)
    assert np.allclose((T.T @ T).toarray(), np.eye(nagg), atol=1e-15)
    sizes = np.bincount(agg, minlength=nagg)
    assert np.allclose(T @ np.sqrt(sizes), 1.0, atol=1e-15)


def test_smoothed_prolongator_1d_closed_form():
    """A = tridiag(-1, 2, -1) on 9 nodes, aggregates {0,1,2}, {3,4,5}, {6,7,8}:
    hi = 2 (interior rows), omega = 2/3, omega / a_ii = 1/3, t = 1/sqrt(3).
    (A T) has t at the aggregate ends, 0 in the middle, -t across an
    aggregate boundary, so P = T - (A T) / 3 is the piecewise-linear
    interpolation t * [2/3, 1, 2/3] with t/3 overlaps (derived by hand)."""
    n = 9
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    agg = np.repeat(np.arange(3), 3)
    P = amg.smoothed_prolongator(A, agg, 3).toarray()
    t = 1.0 / np.sqrt(3.0)
    want = t * np.array([[2 / 3, 0, 0], [1, 0, 0], [2 / 3, 1 / 3, 0],
                         [1 / 3, 2 / 3, 0], [0, 1, 0], [0, 2 / 3, 1 / 3],
                         [0, 1 / 3, 2 / 3], [0, 0, 1], [0, 0, 2 / 3]])
    assert np.allclose(P, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("wind", [None, (1.0, -0.5)])
def test_galerkin_product_against_dense_algebra(wind):
    A, _ = _operator(12, seed=5, tau=0.05, wind=wind)
    agg, nagg = amg.aggregate(amg.strength_graph(A))
    P = amg.smoothed_prolongator(A, agg, nagg)
    Ac = amg.galerkin(A, P)
    dense = P.toarray().T @ A.toarray() @ P.toarray()
    assert np.allclose(Ac.toarray(), dense, rtol=0, atol=1e-14 * abs(dense).max())
    # every non-zero of the dense product lies in the stored pattern
    mask = np.zeros(dense.shape, bool)
    mask[np.repeat(np.arange(nagg), np.diff(Ac.indptr)), Ac.indices] = True
    assert not np.any((dense != 0) & ~mask)


def test_constants_preserved_by_prolongation():
    """For a Neumann Laplacian (A 1 = 0) the smoothed prolongator still maps
    T^T 1 to the constant vector, and the coarse operator annihilates it."""
    m = _mesh(10, seed=2)
    K = sp.csr_matrix(fem.stiffness_p1(m))
    agg, nagg = amg.aggregate(amg.strength_graph(K))
    P = amg.smoothed_prolongator(K, agg, nagg)
    c = np.sqrt(np.bincount(agg, minlength=nagg).astype(float))
    assert np.allclose(P @ c, 1.0, atol=1e-12)
    Kc = amg.galerkin(K, P)
    assert np.abs(Kc @ c).max() <= 1e-12 * abs(Kc).max()


def _sa_iterations(n, seed=0, wind=None, tau=1.0):
    A, _ = _operator(n, seed=seed, tau=tau, wind=wind)
    H = amg.SAHierarchy(A)
    b = np.sin(np.arange(A.shape[0]) * 0.37) + 0.5
    x, info = fgmres(lambda y: A @ y, H, b, rtol=1e-8, restart=30, maxit=200)
    assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * 1.0001
    return info["iters"], H


def test_sa_preconditioner_mesh_robust_on_unstructured_meshes():
    """M + K on unstructured meshes (stiffness-dominated: the condition
    number grows like h^-2): SA-preconditioned FGMRES iterations grow by a
    few from 16^2 to 64^2 meshes (13, 17, 19: cheap degree-2 smoothing and
    ~10:1 aggregates) while the hierarchy deepens; a dropped or sign-flipped
    prolongator smoothing (below) takes 57 or 122 at 64^2."""
    its, levels = [], []
    for n in (16, 32, 64):
        it, H = _sa_iterations(n)
        its.append(it)
        levels.append(len(H.mats))
        assert H.mats[-1].shape[0] <= amg.COARSE_ROWS
        assert all(H.mats[l + 1].shape[0] < H.mats[l].shape[0] / 3 for l in range(len(H.mats) - 1))
    assert levels[0] < levels[-1]
    assert max(its) <= 22 and its[-1] <= its[0] + 8, its


def test_sa_nonsymmetric_convection_block():
    """M + tau (K + C(w)), the CH block shape of Sec. 4 with a prescribed wind."""
    it16, _ = _sa_iterations(16, wind=(2.0, 1.0), tau=0.05)
    it48, _ = _sa_iterations(48, wind=(2.0, 1.0), tau=0.05)
    assert it48 <= 16 and it48 <= it16 + 4, (it16, it48)


def _flipped(A, agg, nagg, hi=None):
    A = sp.csr_matrix(A)
    T = amg.tentative(agg, nagg)
    return sp.csr_matrix(T + sp.diags((4.0 / (3.0 * hi)) / A.diagonal()) @ (A @ T))


def _unsmoothed(A, agg, nagg, hi=None):
    return amg.tentative(agg, nagg)


@pytest.mark.parametrize("mistake", [_flipped, _unsmoothed])
def test_planted_mistake_in_smoothing_breaks_robustness(monkeypatch, mistake):
    """P = T + omega D^-1 A T (a sign flip), or P = T (the smoothing step
    dropped), must fail the iteration bound at 64^2."""
    good, _ = _sa_iterations(64)
    monkeypatch.setattr(amg, "smoothed_prolongator", mistake)
    bad, _ = _sa_iterations(64)
    assert bad > 2 * good, (good, bad)


def test_spectral_bound_against_eigenvalues():
    """The smoothing bound lies between rho(D^-1 A) / 1.05 and min(Gershgorin,
    1.1 rho) on the fine and the coarse operators (dense eigenvalues)."""
    A, _ = _operator(24, seed=4, tau=1.0)
    H = amg.SAHierarchy(A, coarse_rows=40)
    assert len(H.mats) >= 3
    for l, Al in enumerate(H.mats):
        rho = np.abs(np.linalg.eigvals(Al.toarray() / Al.diagonal()[:, None])).max()
        assert rho / 1.05 <= H.his[l] <= min(amg.gershgorin(Al), 1.1 * rho) * (1 + 1e-12), (l, rho, H.his[l])


@pytest.mark.parametrize("n,seed", [(8, 0), (33, 7), (64, 11)])
def test_unstructured_mesh_generator_is_a_valid_triangulation(n, seed):
    """The seeded unstructured meshes the SA tests run on: counter-clockwise
    triangles of positive area tiling the unit square, boundary nodes on the
    boundary, every interior edge shared by exactly two triangles."""
    x, tri = inputs.unstructured_square(n, seed)
    assert x.shape == ((n + 1) ** 2, 2) and tri.shape == (2 * n * n, 3)
    X = x[tri]
    area = 0.5 * ((X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1])
                  - (X[:, 2, 0] - X[:, 0, 0]) * (X[:, 1, 1] - X[:, 0, 1]))
    assert area.min() > 0.0 and abs(area.sum() - 1.0) < 1e-12
    i, j = np.arange(n + 1)[None, :].repeat(n + 1, 0).ravel(), np.arange(n + 1)[:, None].repeat(n + 1, 1).ravel()
    bnd = (i == 0) | (i == n) | (j == 0) | (j == n)
    assert np.allclose(x[bnd], np.stack([i[bnd] / n, j[bnd] / n], axis=1), atol=1e-15, rtol=0)
    edges = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    _, counts = np.unique(edges, axis=0, return_counts=True)
    assert counts.max() == 2 and (counts == 1).sum() == 4 * n       # boundary edges once
    flips = [tuple(sorted(t)) for t in tri[0::2]]
    assert len(set(flips)) == n * n                                     # both diagonals occur below
    m = TriMesh(x, tri)
    assert abs(fem.mass_p1(m).sum() - 1.0) < 1e-12


def test_oracle_step_option_puts_sa_on_the_ac_block():
    """params amg = 1 in the oracle step: the AC solve is preconditioned by
    oracle.amg and still meets its stopping rule; its result agrees with the
    exact AC solve within the Krylov tolerance's reach, and the other solves
    are untouched (same iteration counts as the geometric step)."""
    from oracle.step import Oracle
    n = 24
    p = inputs.default_params()
    st = inputs.initial_state(n, seed=5)
    geo, gi = Oracle(n, p).step(st)
    sa, si = Oracle(n, dict(p, amg=1)).step(st)
    exact, _ = Oracle(n, p, exact=True).step(st)
    assert si["ac"]["converged"] and si["ac"]["rel_residual"] <= p["rtol"]
    e = np.linalg.norm(sa["Phi_v"] - exact["Phi_v"]) / np.linalg.norm(exact["Phi_v"])
    assert e <= 1e-6, e
    for k in ("ch_p", "ch_N", "ch_s", "mu_a", "ns"):
        assert si[k]["iters"] == gi[k]["iters"], k
        assert np.array_equal(sa["v"], geo["v"]) and np.array_equal(sa["phi"], geo["phi"])
