"""The library's 3D (Kuhn tetrahedra) setup on the host against the 3D
oracle: every element operator the 3D device step uses (mass, stiffness,
P1 and P2 convection with the PCD shift, the symmetric-gradient form, the
divergence, the potential and Korteweg loads, the top-face load) and the
nested transfers, entry by entry.  No device is needed: the operators are
built by chnss3_host_operator from the same __host__ __device__ element
functions as the device kernels (CPU).  Also the weighted stiffness of the
concentration-dependent mobility."""
import numpy as np
import pytest

from oracle import three_d as t3
from paper_2501_11767_gb300 import chnss, inputs

N = 4


def _params():
    p = inputs.default_params()
    p.update(alpha=[1e-2, 2e-2, 3e-2, 4e-2], eta=1.3, beta=[0.01, 0.02, 0.1, 1.0], beta_v=0.7)
    return p


@pytest.fixture(scope="module")
def case():
    mesh = t3.Mesh3D(N)
    rng = np.random.default_rng(0)
    st = inputs.initial_state_3d(N, seed=3)
    st["Phi_v"] = 0.3 + 0.2 * rng.random(mesh.N1)
    st["mu"] = rng.standard_normal((4, mesh.N1))
    st["v"] = 0.1 * rng.standard_normal(3 * mesh.N2)
    st = {k: np.ascontiguousarray(v) for k, v in st.items()}
    return mesh, st, _params()


def _same(A, B, rel=1e-12):
    A, B = A.tocsr(), B.tocsr()
    assert A.shape == B.shape
    D = abs(A - B)
    scale = abs(B).max()
    assert (D.max() if D.nnz else 0.0) <= rel * scale


def test_p1_operators(case):
    mesh, st, p = case
    _same(chnss.host_operator3(N, "M1", p), t3.mass_p1(mesh))
    _same(chnss.host_operator3(N, "K1", p), t3.stiffness_p1(mesh))
    _same(chnss.host_operator3(N, "C1", p, st), t3.convection_p1(mesh, st["v"]))
    _same(chnss.host_operator3(N, "CP", p, st), t3.convection_p1(mesh, st["v"], t3.ns_shift(mesh, st, p)))


def test_p2_and_velocity_operators(case):
    mesh, st, p = case
    _same(chnss.host_operator3(N, "M2", p), t3.mass_p2(mesh))
    _same(chnss.host_operator3(N, "J2", p, st), t3.convection_p2(mesh, st["v"], t3.ns_shift(mesh, st, p)))
    _same(chnss.host_operator3(N, "KSYM", p), t3.ksym(mesh, p["eta"]))
    _same(chnss.host_operator3(N, "B", p), t3.divergence(mesh))


def test_transfers(case):
    mesh, _, p = case
    coarse = t3.Mesh3D(N // 2)
    _same(chnss.host_operator3(N, "P1PROL", p), t3.prolongation_p1(coarse), rel=1e-15)
    _same(chnss.host_operator3(N, "VPROL", p), t3.prolongation_velocity(coarse, mesh), rel=1e-15)


def test_open_top_transfer(case):
    """Velocity prolongation between meshes with an open top face: the top
    face's interior nodes are unknowns on both meshes."""
    mesh, _, p = case
    coarse, fine = t3.Mesh3D(N // 2, top_free=True), t3.Mesh3D(N, top_free=True)
    P = chnss.host_operator3(N, "VPROL_OPEN", p)
    _same(P, t3.prolongation_velocity(coarse, fine), rel=1e-15)
    assert P.nnz > chnss.host_operator3(N, "VPROL", p).nnz


def test_loads(case):
    mesh, st, p = case
    got = chnss.host_operator3(N, "LOADS", p, st).reshape(5, mesh.N1)
    ref = t3.potential_loads(mesh, st["phi"], st["Phi_v"])
    for k in range(5):
        assert np.allclose(got[k], ref[k], rtol=1e-12, atol=1e-14 * np.abs(ref[k]).max()), k
    got = chnss.host_operator3(N, "KORTEWEG", p, st)
    ref = t3.korteweg(mesh, t3.korteweg_tensor(mesh, st, p))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    assert np.allclose(chnss.host_operator3(N, "TOP", p), t3.top_load_p1(mesh), rtol=1e-14, atol=1e-16)


def test_weighted_stiffness(case):
    """K_kappa of the concentration-dependent mobility gamma_i (phi_i (1 - phi_i)
    + m0), exact on each tetrahedron, against the oracle's degree-2 rule."""
    mesh, st, p = case
    pv = dict(p, mobility_kind=1, mobility_m0=1e-3, gamma=[1.0, 0.7, 1.3])
    for sp in range(3):
        ref = t3.weighted_stiffness_p1(mesh, t3.mobility_at(mesh, st["phi"][sp], pv, sp))
        _same(chnss.host_operator3(N, f"KK{sp}", pv, st), ref)
    # phi = 0 everywhere: gamma m0 K
    zero = dict(st, phi=np.zeros_like(st["phi"]))
    _same(chnss.host_operator3(N, "KK1", pv, zero), 0.7e-3 * t3.stiffness_p1(mesh))


def test_argument_errors():
    p = _params()
    with pytest.raises(chnss.ChnssError):
        chnss.host_operator3(3, "P1PROL", p)          # odd n has no coarse mesh
    with pytest.raises(chnss.ChnssError):
        chnss.host_operator3(N, "C1", p)              # needs the velocity
    with pytest.raises(chnss.ChnssError):
        chnss.host_operator3(0, "M1", p)
