"""Seeded synthetic inputs and named parameter sets.

This module holds no arithmetic of the method: it only draws the initial
fields (counter-based SplitMix64 noise) and spells out the parameter sets of
the thin-film workloads. Both the CUDA path's tests/bench and the CPU oracle
take their inputs from here.

Initial data (paper Sec. 5, Fig. "Initial condition in 2D"): polymer and NFA
volume fractions a +- 0.01 uniform noise, solvent b, vapour order parameter 0,
velocity 0.  The configurations used here fill the whole unit square with
liquid (a = 0.3, b = 0.4), the chemical potentials start at 0 and the
pressure at 0.

Noise generator: SplitMix64 (Steele, Lea, Flood 2014) started from state 0,
output number key = seed * 2^40 + field * 2^32 + node, mapped to [0, 1) by
its top 53 bits, then to [-amp, amp).
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(keys: np.ndarray) -> np.ndarray:
    """Output number ``key`` (0-based) of SplitMix64 started from state 0:
    mix((key + 1) * 0x9E3779B97F4A7C15 mod 2^64)."""
    with np.errstate(over="ignore"):
        z = (keys.astype(np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_noise(seed: int, field: int, count: int, amp: float = 0.01) -> np.ndarray:
    """``count`` values in [-amp, amp) keyed by (seed, field, node index)."""
    node = np.arange(count, dtype=np.uint64)
    key = (np.uint64(seed) << np.uint64(40)) + (np.uint64(field) << np.uint64(32)) + node
    u = (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (2.0 * u - 1.0) * amp


FIELD_POLYMER = 0
FIELD_NFA = 1


def p1_count(n: int) -> int:
    return (n + 1) * (n + 1)


def p2_count(n: int) -> int:
    return (2 * n + 1) * (2 * n + 1)


def initial_state(n: int, seed: int = 0, a: float = 0.3, b: float = 0.4, amp: float = 0.01) -> dict:
    """Initial state on an n x n structured mesh, as float64 numpy arrays.

    Keys: phi (3, N1) for polymer, NFA, solvent; mu (4, N1) for polymer, NFA,
    solvent, air; Phi_v (N1,); v (2*N2,) interleaved (x, y) per P2 node;
    p (N1,).
    """
    n1, n2 = p1_count(n), p2_count(n)
    phi = np.empty((3, n1))
    phi[0] = a + uniform_noise(seed, FIELD_POLYMER, n1, amp)
    phi[1] = a + uniform_noise(seed, FIELD_NFA, n1, amp)
    phi[2] = b
    return {
        "phi": phi,
        "mu": np.zeros((4, n1)),
        "Phi_v": np.zeros(n1),
        "v": np.zeros(2 * n2),
        "p": np.zeros(n1),
    }


def initial_state_3d(n: int, seed: int = 0, a: float = 0.3, b: float = 0.4, amp: float = 0.01) -> dict:
    """The same start on an n x n x n box mesh: P1 nodes (n+1)^3 (node
    (i, j, k) has id (k (n+1) + j)(n+1) + i), velocity (3 (2n+1)^3,)
    interleaved (x, y, z) per P2 node of the doubled lattice; the noise keyed
    like the 2D fields."""
    n1, n2 = (n + 1) ** 3, (2 * n + 1) ** 3
    phi = np.empty((3, n1))
    phi[0] = a + uniform_noise(seed, FIELD_POLYMER, n1, amp)
    phi[1] = a + uniform_noise(seed, FIELD_NFA, n1, amp)
    phi[2] = b
    return {"phi": phi, "mu": np.zeros((4, n1)), "Phi_v": np.zeros(n1), "v": np.zeros(3 * n2), "p": np.zeros(n1)}


def film_betas(eps: float) -> list:
    """Gradient-energy coefficients (beta_p, beta_NFA, beta_s, beta_a).

    The workloads' interface parameter eps is the gradient-energy coefficient
    of the phase-separating polymer / NFA pair; solvent and air keep the
    values of the paper's 2D all-species runs (beta_s = 0.1, beta_a = 1).
    Reading beta = eps^2 for every species makes the semi-implicit scheme
    (explicit potential, implicit beta Laplacian) unstable at these time
    steps: a Fourier mode grows when tau gamma lambda^2 > 8 beta, with lambda
    the potential's Hessian eigenvalue along the explicit coupling (about 10.6
    for the solvent, 1.9 for the polymer / NFA pair at 0.3 / 0.3).
    """
    return [eps, eps, 0.1, 1.0]


def default_params() -> dict:
    """Parameter set of the 32 x 32 FP64 parity workload.

    eps = 0.02 (see film_betas); dt = 1e-3; constant mobility 1; viscosity 1;
    evaporation rate 0.1; alpha_i = 1e-8 and beta_v = gamma_v = delta_v = 1
    as in the caption of the paper's 2D all-species runs; Krylov tolerance
    1e-8 relative.
    """
    eps = 0.02
    return {
        "tau": 1e-3,
        "beta": film_betas(eps),
        "gamma": [1.0, 1.0, 1.0],
        "mobility_kind": 0,
        "mobility_m0": 1e-3,
        "eta": 1.0,
        "alpha": [1e-8] * 4,
        "beta_v": 1.0,
        "gamma_v": 1.0,
        "delta_v": 1.0,
        "evap_rate": 0.1,
        "phi_s_inf": 0.0,
        "ac_top_flux": 1,
        "precision": 0,
        "rtol": 1e-8,
        "atol": 0.0,
        "restart": 30,
        "maxit": 600,
        # velocity on the top edge: 0 no-slip (eqn:bc), 1 open (a mesh property on
        # the GPU: chnss_mesh_create_ex; read by the oracle from here)
        "top_bc": 0,
        # solvent-air sub-model (model = 1) only: Flory-Huggins constants
        "model": 0,
        "chi_sa": 0.0,
        "n_s": 1.0,
        "n_a": 1.0,
        "phi_sat_s": 1e-6,
        "phi_sat_a": 1.0,
        # multigrid blocks: one V-cycle (0), or V-cycles to this relative
        # tolerance, at most inner_maxit (Sec. 5 uses 1e-4 for its AMG)
        "inner_rtol": 0.0,
        "inner_maxit": 20,
        # Oseen stopping rule of its own when ns_rtol > 0 (0: rtol, atol)
        "ns_rtol": 0.0,
        "ns_atol": 0.0,
        # Gram-Schmidt arithmetic of FGMRES: 0 FP64, 1 double-FP32 (pairs of FP32)
        "ortho": 0,
        # multigrid of the AC block: 0 geometric, 1 smoothed aggregation (Sec. 5's AMG)
        "amg": 0,
    }


FIELD_SOLVENT = 2


def initial_state_solvent_air(n: int, seed: int = 0, amp: float = 0.01, width: float = 0.05) -> dict:
    """Solvent-air start of Sec. 5.1 (initial condition figure with a = 0,
    b = 1): liquid solvent (phi_s = 1 + U[-amp, amp), Phi_v = 0) below a
    wavy interface y = 1/2 + 0.05 sin(2 pi x), air (phi_s = 0, Phi_v = 1)
    above, joined by a tanh profile of the given width so that the initial
    gradients do not grow with the resolution; no polymer or NFA."""
    n1, n2 = p1_count(n), p2_count(n)
    i = np.arange(n1) % (n + 1)
    j = np.arange(n1) // (n + 1)
    x, y = i / n, j / n
    liquid = 0.5 * (1.0 - np.tanh((y - 0.5 - 0.05 * np.sin(2.0 * np.pi * x)) / width))
    phi = np.zeros((3, n1))
    phi[2] = liquid * (1.0 + uniform_noise(seed, FIELD_SOLVENT, n1, amp))
    return {
        "phi": phi,
        "mu": np.zeros((4, n1)),
        "Phi_v": 1.0 - liquid,
        "v": np.zeros(2 * n2),
        "p": np.zeros(n1),
    }


def solvent_air_params() -> dict:
    """Parameters of the paper's solvent-air runs (Sec. 5.1 figure captions):
    beta_s = beta_a = 0.1, beta_v = 1, gamma = 1, delta_v = 1, alpha = 1e-8,
    N_s = N_a = 1, chi_sa = 0, tau = 1e-4; evaporation rate and Krylov
    tolerance as in the default set."""
    p = default_params()
    p.update(model=1, tau=1e-4, beta=[0.1, 0.1, 0.1, 0.1], chi_sa=0.0, n_s=1.0, n_a=1.0)
    return p


def workload(name: str) -> dict:
    """Named workloads: mesh size n, parameters, number of steps."""
    p = default_params()
    if name == "film32_fp64":
        return {"n": 32, "params": p, "steps": 1}
    if name == "film256_mobility":
        p.update(beta=film_betas(0.01), mobility_kind=1)
        return {"n": 256, "params": p, "steps": 20}
    if name == "film1024_mixed":
        p.update(beta=film_betas(0.005), tau=5e-4, precision=1, ortho=1)
        return {"n": 1024, "params": p, "steps": 10}
    if name == "film512_mixed":      # the same parameters on 512 x 512 (profiling captures)
        p.update(beta=film_betas(0.005), tau=5e-4, precision=1, ortho=1)
        return {"n": 512, "params": p, "steps": 10}
    if name == "film1024_amg_mixed":     # the bench set with the AC block on smoothed aggregation (Sec. 5)
        p.update(beta=film_betas(0.005), tau=5e-4, precision=1, ortho=1, amg=1)
        return {"n": 1024, "params": p, "steps": 10}
    if name == "film1024_mixed_inner":   # the bench set with every MG block solved to 1e-4 (Sec. 5)
        p.update(beta=film_betas(0.005), tau=5e-4, precision=1, inner_rtol=1e-4, inner_maxit=20, ortho=1)
        return {"n": 1024, "params": p, "steps": 10}
    if name == "film1024_paper_solver":   # the bench film with the solver settings of Sec. 5
        p.update(beta=film_betas(0.005), tau=5e-4, precision=1, rtol=1e-6, atol=1e-8, ns_rtol=1e-4, ns_atol=1e-8,
                 inner_rtol=1e-4, inner_maxit=20, ortho=1)
        return {"n": 1024, "params": p, "steps": 10}
    if name == "film1024_open_mixed":     # open top on the bench mesh with the paper's time step 1e-4
        p.update(beta=film_betas(0.005), tau=1e-4, precision=1, top_bc=1, ortho=1)
        return {"n": 1024, "params": p, "steps": 10}
    if name == "film512_open_mixed":      # the bench set with an open (do-nothing) top, 512 x 512
        p.update(beta=film_betas(0.005), tau=5e-4, precision=1, top_bc=1, ortho=1)
        return {"n": 512, "params": p, "steps": 10}
    if name == "solvent_air1024_mixed":   # Sec. 5.1 sub-model on the bench mesh
        p = solvent_air_params()
        p.update(precision=1, ortho=1)
        return {"n": 1024, "params": p, "steps": 10, "init": "solvent_air"}
    raise KeyError(name)


SWEEP_MESHES = (128, 192, 256, 384, 512)
FIELD_SWEEP = 7          # key space of the sweep draws (fields 0, 1 are the noise)


def sweep_instances(count: int = 64, seed: int = 0) -> list:
    """A parameter sweep of independent thin-film runs (Sec. 5 varies the
    evaporation rate and the resolution): instance i gets a mesh drawn
    uniformly from SWEEP_MESHES, an evaporation rate uniform in [0.05, 0.5],
    noise seed 1000 + i, and otherwise the default parameters with FP32
    preconditioners.  Returns [{"n", "params", "seed"}]."""
    u = uniform_noise(seed, FIELD_SWEEP, 2 * count, amp=1.0) * 0.5 + 0.5     # U[0, 1)
    out = []
    for i in range(count):
        n = SWEEP_MESHES[min(int(u[2 * i] * len(SWEEP_MESHES)), len(SWEEP_MESHES) - 1)]
        p = default_params()
        p.update(evap_rate=0.05 + 0.45 * float(u[2 * i + 1]), precision=1, ortho=1)
        out.append({"n": n, "params": p, "seed": 1000 + i})
    return out


FIELD_MESH = 9           # key space of the unstructured-mesh draws


def unstructured_square(n: int, seed: int = 0, jitter: float = 0.2):
    """A seeded unstructured triangulation of the unit square: the (n+1)^2
    lattice with every interior node moved by up to jitter * h in each
    coordinate, and every square split along a diagonal drawn at random
    (vertex degrees 3 to 8 instead of the structured mesh's 6).  Returns
    (x (N, 2) float64, tri (E, 3) int64, counter-clockwise), the node (i, j)
    at index j * (n + 1) + i."""
    h = 1.0 / n
    m = n + 1
    N = m * m
    u = uniform_noise(seed, FIELD_MESH, 2 * N + n * n, amp=1.0)       # U[-1, 1)
    ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    ii, jj = ii.ravel(), jj.ravel()
    x = np.stack([ii * h, jj * h], axis=1).astype(np.float64)
    inner = (ii > 0) & (ii < n) & (jj > 0) & (jj < n)
    x[inner, 0] += jitter * h * u[0:N][inner]
    x[inner, 1] += jitter * h * u[N:2 * N][inner]
    si, sj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    si, sj = si.ravel(), sj.ravel()
    v = lambda a, b: b * m + a          # noqa: E731
    flip = u[2 * N:] >= 0.0                                        # split along the other diagonal
    tri = np.empty((2 * n * n, 3), dtype=np.int64)
    lo = np.stack([v(si, sj), v(si + 1, sj), v(si + 1, sj + 1)], axis=1)
    up = np.stack([v(si, sj), v(si + 1, sj + 1), v(si, sj + 1)], axis=1)
    lo_f = np.stack([v(si, sj), v(si + 1, sj), v(si, sj + 1)], axis=1)
    up_f = np.stack([v(si + 1, sj), v(si + 1, sj + 1), v(si, sj + 1)], axis=1)
    tri[0::2] = np.where(flip[:, None], lo_f, lo)
    tri[1::2] = np.where(flip[:, None], up_f, up)
    return x, tri
