"""Python binding of the chnss C ABI (include/chnss.h): argument marshalling
only.  Every step of the method runs in the CUDA library; there is no CPU
fallback: if libchnss.so is missing or fails to load, this module raises.

Device arrays are torch CUDA tensors (float64, contiguous); a state is a dict
  phi (3, N1), mu (4, N1), Phi_v (N1,), v (2*N2,), p (N1,)
with the node numbering described in include/chnss.h.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SYS_CH_P, SYS_CH_N, SYS_CH_S, SYS_AC, SYS_MU_A, SYS_NS = range(6)
SYSTEM_NAMES = ("ch_p", "ch_N", "ch_s", "ac", "mu_a", "ns")
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOCONV", 5: "ERR_BREAKDOWN",
          6: "ERR_NAN", 7: "ERR_TIMEOUT", 8: "ERR_STATE"}
MAT_L, MAT_AC, MAT_A, MAT_B, MAT_AP, MAT_M, MAT_K = range(7)


class Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("beta", ctypes.c_double * 4), ("gamma", ctypes.c_double * 3),
                ("mobility_kind", ctypes.c_int), ("mobility_m0", ctypes.c_double), ("eta", ctypes.c_double),
                ("alpha", ctypes.c_double * 4), ("beta_v", ctypes.c_double), ("gamma_v", ctypes.c_double),
                ("delta_v", ctypes.c_double), ("evap_rate", ctypes.c_double), ("phi_s_inf", ctypes.c_double),
                ("ac_top_flux", ctypes.c_int), ("precision", ctypes.c_int), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("model", ctypes.c_int), ("chi_sa", ctypes.c_double), ("n_s", ctypes.c_double),
                ("n_a", ctypes.c_double), ("phi_sat_s", ctypes.c_double), ("phi_sat_a", ctypes.c_double),
                ("inner_rtol", ctypes.c_double), ("inner_maxit", ctypes.c_int),
                ("ns_rtol", ctypes.c_double), ("ns_atol", ctypes.c_double), ("ortho", ctypes.c_int),
                ("amg", ctypes.c_int)]


class State(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_void_p * 3), ("mu", ctypes.c_void_p * 4), ("Phi_v", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("p", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "converged": bool(self.converged), "rel_residual": self.rel_residual,
                "seconds": self.seconds}


INNER_BLOCKS = ("L", "AC", "A", "Kp", "X1_p", "X1_N", "X1_s", "X2_p", "X2_N", "X2_s")


class InnerStats(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_longlong * 10), ("cycles", ctypes.c_longlong * 10),
                ("last_rel_residual", ctypes.c_double * 10)]

    def as_dict(self):
        return {name: {"solves": self.solves[i], "cycles": self.cycles[i],
                       "last_rel_residual": self.last_rel_residual[i]} for i, name in enumerate(INNER_BLOCKS)}


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("nkinds", ctypes.c_int), ("name", (ctypes.c_char * 32) * 8),
                ("kind_launches", ctypes.c_longlong * 8), ("kind_ms", ctypes.c_double * 8),
                ("kind_bytes", ctypes.c_double * 8), ("kind_flops", ctypes.c_double * 8)]

    def as_dict(self):
        kinds = {}
        for k in range(self.nkinds):
            kinds[self.name[k].value.decode()] = {"launches": self.kind_launches[k], "ms": self.kind_ms[k],
                                                  "bytes": self.kind_bytes[k], "flops": self.kind_flops[k]}
        return {"launches": self.launches, "kinds": kinds}


class Tuning(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int * 3), ("ms_p1", ctypes.c_double * 3), ("ms_p2", ctypes.c_double * 3),
                ("block_p1", ctypes.c_int), ("block_p2", ctypes.c_int)]

    def as_dict(self):
        return {"candidates": list(self.candidates), "ms_p1": list(self.ms_p1), "ms_p2": list(self.ms_p2),
                "block_p1": self.block_p1, "block_p2": self.block_p2}


class Diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 4), ("div_norm", ctypes.c_double), ("p_mean", ctypes.c_double),
                ("energy", ctypes.c_double), ("energy_local", ctypes.c_double),
                ("energy_gradient", ctypes.c_double), ("energy_kinetic", ctypes.c_double)]

    def as_dict(self):
        return {"mass": list(self.mass[:3]), "mass_a": self.mass[3], "div": self.div_norm, "p_mean": self.p_mean,
                "energy": self.energy,
                "energy_parts": {"local": self.energy_local, "gradient": self.energy_gradient,
                                 "kinetic": self.energy_kinetic}}


class ChnssError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"chnss {STATUS.get(status, status)}: {msg}")
        self.status = status


_LIB = None

EXPORTS = {
    "chnss_mesh_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "chnss_mesh_create_ex": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "chnss_mesh_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "chnss_mesh_sizes": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 4),
    "chnss_ctx_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "chnss_ctx_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "chnss_assemble": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State)]),
    "chnss_system_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "chnss_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(SolveInfo)]),
    "chnss_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.POINTER(State),
                                  ctypes.POINTER(SolveInfo)]),
    "chnss_step_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.POINTER(State),
                                       ctypes.POINTER(SolveInfo)]),
    "chnss_export_csr": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "chnss_export_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "chnss_mass_solve_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.POINTER(SolveInfo)]),
    "chnss_adjoint_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.POINTER(State),
                                          ctypes.POINTER(State), ctypes.POINTER(State),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo)]),
    "chnss_objective": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_void_p]),
    "chnss_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.POINTER(Diag)]),
    "chnss_debug_cgs2": (ctypes.c_int, [ctypes.c_int, ctypes.c_long, ctypes.c_int, ctypes.c_void_p, ctypes.c_long,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "chnss_debug_spmv": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "chnss_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "chnss_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Profile)]),
    "chnss_inner_stats_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(InnerStats)]),
    "chnss3_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Params), ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "chnss3_ctx_create_ex": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params), ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "chnss3_ctx_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "chnss3_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "chnss3_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.POINTER(State),
                                   ctypes.POINTER(SolveInfo)]),
    "chnss3_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "chnss3_set_step_concurrency": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "chnss3_adjoint_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.POINTER(State),
                                           ctypes.POINTER(State), ctypes.POINTER(State),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo)]),
    "chnss3_objective": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.c_void_p]),
    "chnss3_host_operator": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params), ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "chnss_step_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(State),
                                          ctypes.POINTER(State), ctypes.POINTER(SolveInfo), ctypes.c_int]),
    "chnss_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Tuning)]),
    "chnss_set_spmv_block": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "chnss_set_step_concurrency": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "chnss_set_step_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "chnss_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "chnss_set_batch_mode": (ctypes.c_int, [ctypes.c_int]),
    "chnss_batch_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "chnss_amg_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "chnss_amg_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "chnss_amg_levels": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "chnss_amg_export_level": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 8),
    "chnss_amg_vcycle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "chnss_amg_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
    "chnss_amg_destroy": (None, [ctypes.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libchnss.so (building it in-tree if it is missing or stale)."""
    global _LIB
    if _LIB is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ChnssError(2, f"CUDA library not found at {path}")
        lib = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _check(status, ctx=None):
    if status != 0:
        msg = load().chnss_last_error(ctx)
        raise ChnssError(status, msg.decode() if msg else "")


# fields of the solvent-air sub-model, defaulted when a parameter set omits them
_OPTIONAL = {"model": 0, "chi_sa": 0.0, "n_s": 1.0, "n_a": 1.0, "phi_sat_s": 1e-6, "phi_sat_a": 1.0,
             "inner_rtol": 0.0, "inner_maxit": 20, "ns_rtol": 0.0, "ns_atol": 0.0,
             "ortho": 0, "amg": 0}


def make_params(d: dict) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        val = d[name] if name in d or name not in _OPTIONAL else _OPTIONAL[name]
        if isinstance(val, (list, tuple)):
            arr = getattr(p, name)
            for i, x in enumerate(val):
                arr[i] = x
        else:
            setattr(p, name, val)
    return p


def _ptr(t, n=None, where=None):
    """Address of a contiguous float64 array.  n: the number of elements the
    call reads or writes (a shorter array is refused); where: "device" (a
    CUDA tensor), "host" (a numpy array or CPU tensor) or None (unchecked).
    The C ABI takes bare pointers, so these checks are the only guard against
    out-of-bounds accesses from a wrongly sized or placed array."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous() or str(t.dtype) != "torch.float64":
            raise ValueError("chnss needs contiguous float64 tensors")
        if where == "device" and not t.is_cuda:
            raise ValueError("chnss needs CUDA tensors here (device pointers)")
        if where == "host" and t.is_cuda:
            raise ValueError("chnss needs host arrays here")
        size = t.numel()
        ptr = t.data_ptr()
    elif isinstance(t, np.ndarray):
        if t.dtype != np.float64 or not t.flags["C_CONTIGUOUS"]:
            raise ValueError("chnss needs C-contiguous float64 arrays")
        if where == "device":
            raise ValueError("chnss needs CUDA tensors here (device pointers), not numpy arrays")
        size = t.size
        ptr = t.ctypes.data
    else:
        raise TypeError(type(t))
    if n is not None and size < n:
        raise ValueError(f"chnss: an array of {size} elements where {n} are needed")
    return ptr


def make_state(d: dict, N1: int = None, N2: int = None, dim: int = 2, where: str = None) -> State:
    """chnss_state of the arrays of d; with N1, N2 (and the space dimension)
    every field's length is checked, with where its placement (see _ptr)."""
    nv = dim * N2 if N2 is not None else None
    s = State()
    for i in range(3):
        s.phi[i] = _ptr(d["phi"][i], N1, where)
    for i in range(4):
        s.mu[i] = _ptr(d["mu"][i], N1, where)
    s.Phi_v = _ptr(d["Phi_v"], N1, where)
    s.v = _ptr(d["v"], nv, where)
    s.p = _ptr(d["p"], N1, where)
    return s


class Mesh:
    """Structured n x n triangulation of [0, lx] x [0, ly] with its multigrid
    hierarchy (chnss_mesh_create)."""

    def __init__(self, n: int, lx: float = 1.0, ly: float = 1.0, top_bc: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.chnss_mesh_create_ex(n, n, lx, ly, top_bc, ctypes.byref(h)))
        self._h = h
        self.n, self.lx, self.ly, self.top_bc = n, lx, ly, top_bc
        v = [ctypes.c_int() for _ in range(4)]
        _check(lib.chnss_mesh_sizes(h, *[ctypes.byref(x) for x in v]))
        self.N1, self.N2, self.E, self.levels = (x.value for x in v)

    def close(self):
        if self._h:
            load().chnss_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Parameters, operators and workspace on one CUDA stream
    (chnss_ctx_create)."""

    def __init__(self, mesh: Mesh, params: dict, stream=None):
        import torch
        lib = load()
        self.mesh = mesh
        self.params = dict(params)
        self._p = make_params(self.params)
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        h = ctypes.c_void_p()
        _check(lib.chnss_ctx_create(mesh._h, ctypes.byref(self._p), ctypes.c_void_p(st.cuda_stream),
                                    ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h:
            load().chnss_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def system_size(self, sys: int) -> int:
        return load().chnss_system_size(self._h, sys)

    def new_state(self, device="cuda"):
        import torch
        N1, N2 = self.mesh.N1, self.mesh.N2
        z = lambda *s: torch.zeros(*s, dtype=torch.float64, device=device)  # noqa: E731
        return {"phi": z(3, N1), "mu": z(4, N1), "Phi_v": z(N1), "v": z(2 * N2), "p": z(N1)}

    def _state(self, d: dict, where: str = "device") -> State:
        return make_state(d, self.mesh.N1, self.mesh.N2, 2, where)

    def assemble(self, state: dict):
        s = self._state(state)
        _check(load().chnss_assemble(self._h, ctypes.byref(s)), self._h)

    def solve(self, sys: int, rhs=None, x=None, check: bool = True):
        import torch
        n = self.system_size(sys)
        if x is None:
            x = torch.empty(n, dtype=torch.float64, device="cuda")
        info = SolveInfo()
        st = load().chnss_solve(self._h, sys, _ptr(rhs, n, "device"), _ptr(x, n, "device"), ctypes.byref(info))
        if check:
            _check(st, self._h)
        return x, info.as_dict(), st

    def step(self, state_in: dict, state_out: dict = None, check: bool = True):
        if state_out is None:
            state_out = self.new_state()
        a, b = self._state(state_in), self._state(state_out)
        infos = (SolveInfo * 6)()
        st = load().chnss_step(self._h, ctypes.byref(a), ctypes.byref(b), infos)
        if check:
            _check(st, self._h)
        return state_out, {SYSTEM_NAMES[i]: infos[i].as_dict() for i in range(6)}, st

    def step_host(self, host_in: dict, host_out: dict, check: bool = True):
        a, b = self._state(host_in, "host"), self._state(host_out, "host")
        infos = (SolveInfo * 6)()
        st = load().chnss_step_host(self._h, ctypes.byref(a), ctypes.byref(b), infos)
        if check:
            _check(st, self._h)
        return host_out, {SYSTEM_NAMES[i]: infos[i].as_dict() for i in range(6)}, st

    def export_csr(self, which: int):
        lib = load()
        nr, nz = ctypes.c_int(), ctypes.c_int()
        _check(lib.chnss_export_csr(self._h, which, ctypes.byref(nr), ctypes.byref(nz), None, None, None), self._h)
        rowptr = np.zeros(nr.value + 1, dtype=np.int32)
        col = np.zeros(nz.value, dtype=np.int32)
        val = np.zeros(nz.value, dtype=np.float64)
        _check(lib.chnss_export_csr(self._h, which, ctypes.byref(nr), ctypes.byref(nz), rowptr.ctypes.data,
                                    col.ctypes.data, val.ctypes.data), self._h)
        return rowptr, col, val

    def adjoint_step(self, state_k: dict, state_k1: dict, adj_k1: dict, adj_k: dict = None, check: bool = True):
        """Returns (adj_k, [d/d evap_rate, d/d gamma], infos, status)."""
        if adj_k is None:
            adj_k = self.new_state()
        a, b, c, d = (self._state(x) for x in (state_k, state_k1, adj_k1, adj_k))
        grad = (ctypes.c_double * 2)(0.0, 0.0)
        infos = (SolveInfo * 6)()
        st = load().chnss_adjoint_step(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                       grad, infos)
        if check:
            _check(st, self._h)
        return adj_k, [grad[0], grad[1]], {SYSTEM_NAMES[i]: infos[i].as_dict() for i in range(6)}, st

    def objective(self, phi_p, grad=None):
        """J = int |grad phi_p|^2 and, if grad is a device array, 2 K phi_p."""
        J = ctypes.c_double()
        N1 = self.mesh.N1
        _check(load().chnss_objective(self._h, _ptr(phi_p, N1, "device"), ctypes.byref(J), _ptr(grad, N1, "device")),
               self._h)
        return J.value

    def diagnostics(self, state: dict) -> dict:
        """chnss_diagnostics: FP64 mass sums of the four species, ||B v||,
        int p and the energy parts of a device state (keys as the oracle's
        Oracle.diagnostics)."""
        d = Diag()
        _check(load().chnss_diagnostics(self._h, ctypes.byref(self._state(state)), ctypes.byref(d)), self._h)
        return d.as_dict()

    def mass_solve_noalloc(self, rhs, x=None, check: bool = True):
        """M x = rhs through chnss_mass_solve_noalloc (no device allocation
        inside the library call; x must be given to avoid one here)."""
        import torch
        if x is None:
            x = torch.empty(self.mesh.N1, dtype=torch.float64, device="cuda")
        info = SolveInfo()
        N1 = self.mesh.N1
        st = load().chnss_mass_solve_noalloc(self._h, _ptr(rhs, N1, "device"), _ptr(x, N1, "device"), ctypes.byref(info))
        if check:
            _check(st, self._h)
        return x, info.as_dict(), st

    def autotune(self) -> dict:
        """Pick the SpMV threads-per-block of the mesh's scalar and velocity
        operators by timing (chnss_autotune); re-captures this context's
        preconditioner graphs."""
        t = Tuning()
        _check(load().chnss_autotune(self._h, ctypes.byref(t)), self._h)
        return t.as_dict()

    def set_step_mode(self, mode: int):
        """chnss_set_step_mode: 0 host-driven Krylov loops (default), 1 the
        whole step as one recorded CUDA graph launch."""
        _check(load().chnss_set_step_mode(self._h, int(mode)), self._h)

    def set_step_concurrency(self, on: bool):
        """chnss_set_step_concurrency: solve CH, AC and NS of a step on three
        streams at once (default) or one after the other."""
        _check(load().chnss_set_step_concurrency(self._h, 1 if on else 0), self._h)

    def set_spmv_block(self, block_p1: int, block_p2: int):
        """Pin the SpMV threads-per-block of the mesh's scalar and velocity
        operators (chnss_set_spmv_block)."""
        _check(load().chnss_set_spmv_block(self._h, block_p1, block_p2), self._h)

    def profile_enable(self, on: bool = True):
        _check(load().chnss_profile_enable(self._h, 1 if on else 0), self._h)

    def profile_read(self) -> dict:
        p = Profile()
        _check(load().chnss_profile_read(self._h, ctypes.byref(p)), self._h)
        return p.as_dict()

    def inner_stats(self, reset: bool = False) -> dict:
        """Per multigrid block of the preconditioners: inner solves, V-cycles
        and the last relative residual (inner_rtol > 0)."""
        st = InnerStats()
        _check(load().chnss_inner_stats_read(self._h, 1 if reset else 0, ctypes.byref(st)), self._h)
        return st.as_dict()

    def export_rhs(self, sys: int):
        out = np.zeros(self.system_size(sys), dtype=np.float64)
        _check(load().chnss_export_rhs(self._h, sys, out.ctypes.data), self._h)
        return out


class Context3:
    """The 3D step on the Kuhn mesh of n^3 cubes of the unit box
    (chnss3_ctx_create_ex / chnss3_step): device states with phi (3, N1),
    mu (4, N1), Phi_v, p (N1) and v (3 N2).  params["top_bc"] = 1 opens
    the top face (do-nothing condition); default 0, no-slip everywhere."""

    def __init__(self, n: int, params: dict, stream=None):
        lib = load()
        self._p = make_params(params)
        h = ctypes.c_void_p()
        sptr = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(lib.chnss3_ctx_create_ex(n, int(params.get("top_bc", 0)), ctypes.byref(self._p), sptr,
                                        ctypes.byref(h)))
        self._h = h
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib.chnss3_sizes(h, ctypes.byref(a), ctypes.byref(b)))
        self.n, self.N1, self.N2 = n, a.value, b.value

    def __del__(self):
        if getattr(self, "_h", None):
            load().chnss3_ctx_destroy(self._h)
            self._h = None

    def set_step_concurrency(self, on: bool):
        _check(load().chnss3_set_step_concurrency(self._h, 1 if on else 0))

    def new_state(self):
        import torch
        z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")   # noqa: E731
        return {"phi": z((3, self.N1)), "mu": z((4, self.N1)), "Phi_v": z(self.N1), "v": z(3 * self.N2),
                "p": z(self.N1)}

    def step(self, state_in: dict, state_out: dict = None, check: bool = True):
        if state_out is None:
            state_out = self.new_state()
        a, b = (make_state(x, self.N1, self.N2, 3, "device") for x in (state_in, state_out))
        infos = (SolveInfo * 6)()
        st = load().chnss3_step(self._h, ctypes.byref(a), ctypes.byref(b), infos)
        if check and st != 0:
            msg = load().chnss3_last_error(self._h)
            raise ChnssError(st, msg.decode() if msg else "")
        return state_out, {SYSTEM_NAMES[i]: infos[i].as_dict() for i in range(6)}, st

    def _check3(self, st):
        if st != 0:
            msg = load().chnss3_last_error(self._h)
            raise ChnssError(st, msg.decode() if msg else "")

    def adjoint_step(self, state_k: dict, state_k1: dict, adj_k1: dict, adj_k: dict = None, check: bool = True):
        """chnss3_adjoint_step: returns (adj_k, [d/d evap_rate, d/d gamma], infos, status)."""
        if adj_k is None:
            adj_k = self.new_state()
        a, b, c, d = (make_state(x, self.N1, self.N2, 3, "device") for x in (state_k, state_k1, adj_k1, adj_k))
        grad = (ctypes.c_double * 2)(0.0, 0.0)
        infos = (SolveInfo * 6)()
        st = load().chnss3_adjoint_step(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                        grad, infos)
        if check:
            self._check3(st)
        return adj_k, [grad[0], grad[1]], {SYSTEM_NAMES[i]: infos[i].as_dict() for i in range(6)}, st

    def objective(self, phi_p, grad=None):
        """J = int |grad phi_p|^2 on the 3D mesh and, if grad is a device array, 2 K phi_p."""
        J = ctypes.c_double()
        self._check3(load().chnss3_objective(self._h, _ptr(phi_p, self.N1, "device"), ctypes.byref(J),
                                             _ptr(grad, self.N1, "device")))
        return J.value


OPS3 = ("M1", "K1", "C1", "CP", "M2", "J2", "KSYM", "B", "P1PROL", "VPROL", "LOADS", "KORTEWEG", "TOP",
        "KK0", "KK1", "KK2", "VPROL_OPEN")


def host_operator3(n: int, which: str, params: dict, state: dict = None):
    """One operator of the 3D (Kuhn tetrahedra) discretisation built on the
    host by the library (chnss3_host_operator): a scipy CSR matrix, or a
    numpy vector for LOADS, KORTEWEG and TOP.  state: host float64 arrays
    of the 3D sizes (phi (3, N1), mu (4, N1), Phi_v, v (3 N2), p)."""
    import scipy.sparse as sp
    lib = load()
    op = OPS3.index(which)
    prm = make_params(params)
    st = make_state(state, (n + 1) ** 3, (2 * n + 1) ** 3, 3, "host") if state is not None else None
    sptr = ctypes.byref(st) if st is not None else None
    nr, nc, nnz = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _check(lib.chnss3_host_operator(n, op, ctypes.byref(prm), sptr, ctypes.byref(nr), ctypes.byref(nc),
                                    ctypes.byref(nnz), None, None, None))
    val = np.zeros(nnz.value)
    if which in ("LOADS", "KORTEWEG", "TOP"):
        _check(lib.chnss3_host_operator(n, op, ctypes.byref(prm), sptr, ctypes.byref(nr), ctypes.byref(nc),
                                        ctypes.byref(nnz), None, None, val.ctypes.data))
        return val
    rowptr = np.zeros(nr.value + 1, dtype=np.int32)
    col = np.zeros(nnz.value, dtype=np.int32)
    _check(lib.chnss3_host_operator(n, op, ctypes.byref(prm), sptr, ctypes.byref(nr), ctypes.byref(nc),
                                    ctypes.byref(nnz), rowptr.ctypes.data, col.ctypes.data, val.ctypes.data))
    return sp.csr_matrix((val, col, rowptr), shape=(nr.value, nc.value))


def debug_spmv(layout: int, precision: int, mode: int, rowptr, col, val, x, b=None, w=None, dinv=None,
               coef=None, y=None, ncols: int = None):
    """chnss_debug_spmv: one SpMV through the library's SELL kernels on HOST
    numpy data (layout 0 scalar, 1 2x2 blocks, 2 3x3 blocks; val (nnz, bs^2)).
    Returns (y, warps per slice)."""
    bs = (1, 2, 3)[layout] if 0 <= layout <= 2 else 1   # other layouts: refused by the library
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    nrows = len(rowptr) - 1
    ncols = nrows if ncols is None else ncols
    val = np.ascontiguousarray(val, dtype=np.float64).reshape(-1)
    if val.size != len(col) * bs * bs:
        raise ValueError("val must hold bs^2 values per entry")
    arr = lambda a, n: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(n)   # noqa: E731
    x = arr(x, bs * ncols)
    b, w, dinv = arr(b, bs * nrows), arr(w, bs * nrows), arr(dinv, bs * nrows)
    coef = arr(coef, 3)
    y = np.zeros(bs * nrows) if y is None else np.array(y, dtype=np.float64).reshape(bs * nrows)
    ptr = lambda a: None if a is None else a.ctypes.data   # noqa: E731
    k = ctypes.c_int()
    _check(load().chnss_debug_spmv(layout, precision, mode, nrows, ncols, rowptr.ctypes.data, col.ctypes.data,
                                   val.ctypes.data, x.ctypes.data, ptr(b), ptr(w), ptr(dinv), ptr(coef),
                                   y.ctypes.data, ctypes.byref(k)))
    return y, k.value


def debug_cgs2(V, w, arith: int):
    """chnss_debug_cgs2: one CGS2 step of the CUDA device vector w against the
    rows of the (k, ld) CUDA array V (FP64 or double-FP32 kernels).
    Returns (h1, h2, ||w'||^2, vout)."""
    import torch
    k, ld = V.shape
    n = w.numel()
    if not (V.is_cuda and w.is_cuda) or V.dtype != torch.float64 or w.dtype != torch.float64:
        raise ValueError("V and w must be CUDA float64 tensors")
    if not V.is_contiguous() or not w.is_contiguous() or ld < n:
        raise ValueError("V must be contiguous (k, ld) with ld >= n")
    h = np.zeros(2 * k + 1)
    vout = torch.empty(n, dtype=torch.float64, device=w.device)
    _check(load().chnss_debug_cgs2(arith, n, k, V.data_ptr(), ld, w.data_ptr(), h.ctypes.data, vout.data_ptr()))
    return h[:k], h[k:2 * k], h[2 * k], vout


def step_batched(ctxs, states_in, states_out=None, max_threads: int = 0, check: bool = True):
    """One chnss_step of every context, concurrently (chnss_step_batched).
    Give each context its own stream (Context(..., stream=torch.cuda.Stream()))
    or the instances serialise on the shared one.  Returns (states_out,
    per-instance solve records, status)."""
    n = len(ctxs)
    if len(states_in) != n or (states_out is not None and len(states_out) != n):
        raise ValueError("one input (and output) state per context")
    if states_out is None:
        states_out = [c.new_state() for c in ctxs]
    hs = (ctypes.c_void_p * n)(*[c._h.value for c in ctxs])
    a = (State * n)(*[c._state(x) for c, x in zip(ctxs, states_in)])
    b = (State * n)(*[c._state(x) for c, x in zip(ctxs, states_out)])
    infos = (SolveInfo * (6 * n))()
    st = load().chnss_step_batched(n, hs, a, b, infos, max_threads)
    if check:
        _check(st, None)
    recs = [{SYSTEM_NAMES[k]: infos[6 * i + k].as_dict() for k in range(6)} for i in range(n)]
    return states_out, recs, st


def set_batch_mode(mode: int):
    """chnss_set_batch_mode: 0 one graph launch per instance, 1 one graph per batch."""
    _check(load().chnss_set_batch_mode(int(mode)))


def batch_stats() -> dict:
    """chnss_step_batched calls run as one batch graph / one graph per instance."""
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().chnss_batch_stats(ctypes.byref(a), ctypes.byref(b)))
    return {"one_graph": a.value, "per_instance": b.value}


def state_to_device(state: dict, device="cuda") -> dict:
    import torch
    return {k: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=device).contiguous()
            for k, v in state.items()}


def state_to_numpy(state: dict) -> dict:
    return {k: v.detach().cpu().numpy() for k, v in state.items()}


def _int32_device(t, n):
    """Address of a contiguous int32 CUDA tensor of at least n entries."""
    if not hasattr(t, "data_ptr") or not t.is_cuda or str(t.dtype) != "torch.int32" or not t.is_contiguous():
        raise ValueError("chnss needs contiguous int32 CUDA tensors here")
    if t.numel() < n:
        raise ValueError(f"chnss: an array of {t.numel()} elements where {n} are needed")
    return t.data_ptr()


class Amg:
    """Smoothed-aggregation AMG hierarchy of a square CSR matrix on the device
    (chnss_amg_*): rowptr / col int32 and val float64 CUDA tensors."""

    def __init__(self, rowptr, col, val, precision: int = 0):
        n = rowptr.numel() - 1
        nnz = col.numel()
        self.n, self.nnz = n, nnz
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.chnss_amg_create(n, nnz, _int32_device(rowptr, n + 1), _int32_device(col, nnz),
                                    _ptr(val, nnz, "device"), int(precision), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().chnss_amg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, val):
        _check(load().chnss_amg_update(self._h, _ptr(val, self.nnz, "device")))

    def levels(self):
        """[(rows, nnz of A_l, nnz of P_l)] per level."""
        nl = ctypes.c_int()
        rows, nnz, pnnz = (np.zeros(12, np.int32) for _ in range(3))
        _check(load().chnss_amg_levels(self._h, ctypes.byref(nl), rows.ctypes.data, nnz.ctypes.data,
                                       pnnz.ctypes.data))
        return [(int(rows[l]), int(nnz[l]), int(pnnz[l])) for l in range(nl.value)]

    def export_level(self, level: int) -> dict:
        """Level l on the host: A (rowptr, col, val), hi, and unless it is the
        coarsest, agg and P (rowptr, col, val)."""
        lv = self.levels()
        rows, nnz, pnnz = lv[level]
        last = level == len(lv) - 1
        out = {"hi": np.zeros(1), "a_rowptr": np.zeros(rows + 1, np.int32), "a_col": np.zeros(nnz, np.int32),
               "a_val": np.zeros(nnz)}
        if not last:
            out.update(agg=np.zeros(rows, np.int32), p_rowptr=np.zeros(rows + 1, np.int32),
                       p_col=np.zeros(pnnz, np.int32), p_val=np.zeros(pnnz))
        g = lambda k: out[k].ctypes.data if k in out else None   # noqa: E731
        _check(load().chnss_amg_export_level(self._h, level, g("agg"), g("hi"), g("a_rowptr"), g("a_col"),
                                             g("a_val"), g("p_rowptr"), g("p_col"), g("p_val")))
        out["hi"] = float(out["hi"][0])
        return out

    def vcycle(self, b, x=None):
        import torch
        x = torch.empty_like(b) if x is None else x
        _check(load().chnss_amg_vcycle(self._h, _ptr(b, self.n, "device"), _ptr(x, self.n, "device")))
        return x

    def solve(self, b, x=None, rtol=1e-8, atol=0.0, maxit=500, check=True):
        import torch
        x = torch.empty_like(b) if x is None else x
        info = SolveInfo()
        st = load().chnss_amg_solve(self._h, _ptr(b, self.n, "device"), _ptr(x, self.n, "device"), rtol, atol,
                                    maxit, ctypes.byref(info))
        if check and st != 0:
            _check(st)
        return x, {"iters": info.iters, "converged": bool(info.converged), "rel_residual": info.rel_residual,
                   "seconds": info.seconds}, st
