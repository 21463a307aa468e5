"""The 3D step at the 3D bench size: 32^3 Kuhn cubes (35,937 P1 nodes,
823,875 velocity dofs), FP32 multigrid inside FP64 FGMRES with double-FP32
Gram-Schmidt, tau = 1e-4.  The oracle is too slow for whole steps here, so
the properties that hold at any size are checked instead: every solve of two
steps from the seeded start (the second with convection) meets its stopping
rule ||b - A x|| <= 1e-8 ||b|| when the residual is recomputed in FP64 by
scipy from the oracle's own operators (oracle/three_d.py, built from the
step's input state; nothing shared with the library), the air potential
solves its mass system to the PCG tolerance, and the enclosed-flow pressure
has zero mean."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import three_d as t3
from paper_2501_11767_gb300 import chnss, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _rel_res(A, x, b):
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


def test_full_size_3d_solves_meet_the_stopping_rule(torch):
    n = 32
    p = dict(inputs.default_params(), tau=1e-4, precision=1, ortho=1)
    ctx = chnss.Context3(n, p)
    mesh = t3.Mesh3D(n)
    F = t3.Forms3D(mesh, p)
    tau, rtol, beta = p["tau"], p["rtol"], p["beta"]
    st = chnss.state_to_device(inputs.initial_state_3d(n, seed=0))
    for k in range(2):
        out, info, status = ctx.step(st)
        torch.cuda.synchronize()
        assert status == 0
        s, got = chnss.state_to_numpy(st), chnss.state_to_numpy(out)
        conv = t3.convection_p1(mesh, s["v"])
        loads = t3.potential_loads(mesh, s["phi"], s["Phi_v"])
        j = p["evap_rate"] * (s["phi"][2][mesh.top_reference_node()] - p["phi_s_inf"])
        f = [loads[0], loads[1], loads[2] - beta[2] * j * F.top, loads[3] + beta[3] * j * F.top]
        for i, name in enumerate(("ch_p", "ch_N", "ch_s")):
            g = p["gamma"][i]
            c = tau * g / beta[i]
            A = sp.bmat([[F.M + tau * conv, tau * g * F.K], [tau * g * F.K, -c * F.M]], format="csr")
            rhs = np.concatenate([F.M @ s["phi"][i], -c * f[i]])
            r = _rel_res(A, np.concatenate([got["phi"][i], got["mu"][i]]), rhs)
            assert info[name]["converged"] and r <= rtol * (1 + 1e-6), (k, name, r, info[name])
        Aac = (F.M + tau * p["delta_v"] * F.K + tau * conv).tocsr()
        rac = F.M @ s["Phi_v"] - tau * p["gamma_v"] * loads[4]
        if p["ac_top_flux"]:
            rac = rac + tau * p["delta_v"] * j * F.top
        r = _rel_res(Aac, got["Phi_v"], rac)
        assert info["ac"]["converged"] and r <= rtol * (1 + 1e-6), (k, r, info["ac"])
        rmu = f[3] + beta[3] * (F.K @ (1.0 - got["phi"].sum(axis=0)))
        assert _rel_res(F.M, got["mu"][3], rmu) <= 1e-10, k
        A, B, rhs_v, _, _ = t3.ns_system(F, s, p)
        v, pr = got["v"], got["p"]
        res = np.concatenate([rhs_v - A @ v - B.T @ pr, -(B @ v)])
        r = float(np.linalg.norm(res) / np.linalg.norm(rhs_v))
        assert info["ns"]["converged"] and r <= rtol * (1 + 1e-6), (k, r, info["ns"])
        mp = F.M @ pr
        assert abs(mp).sum() > 0 and abs(mp.sum()) <= 1e-9 * abs(mp).sum(), k
        del A, B, Aac
        st = out
