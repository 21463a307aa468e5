"""The C-ABI library builds, loads and exports every symbol include/chnss.h
declares; argument validation happens before any device call (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_2501_11767_gb300 import build as B
from paper_2501_11767_gb300 import chnss

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "chnss.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chnss3?_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return chnss.load()


def test_header_declares_the_step_api():
    names = declared_functions()
    for required in ("chnss_mesh_create", "chnss_ctx_create", "chnss_assemble", "chnss_solve", "chnss_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the Python binding covers exactly the declared calls
    assert sorted(chnss.EXPORTS) == declared_functions()


def test_library_is_built_for_sm_103a():
    assert os.path.exists(B.LIB)
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_argument_errors_need_no_device(lib):
    h = ctypes.c_void_p()
    assert lib.chnss_mesh_create(7, 7, 1.0, 1.0, ctypes.byref(h)) == 1      # odd n
    assert lib.chnss_mesh_create(2050, 2050, 1.0, 1.0, ctypes.byref(h)) == 1  # int32 element offsets
    assert b"even" in lib.chnss_last_error(None)
    assert lib.chnss_mesh_create(258, 258, 1.0, 1.0, ctypes.byref(h)) == 1  # coarsens to 129 x 129
    assert b"coarsens to 129 x 129" in lib.chnss_last_error(None)
    assert lib.chnss_mesh_create(54, 54, 1.0, 1.0, ctypes.byref(h)) == 1    # coarsens to 27 x 27
    assert lib.chnss_mesh_create(8, 16, 1.0, 1.0, ctypes.byref(h)) == 1     # nx != ny
    assert lib.chnss_mesh_create(8, 8, -1.0, 1.0, ctypes.byref(h)) == 1     # bad length
    assert lib.chnss_mesh_create(8, 8, 1.0, 1.0, None) == 1
    assert lib.chnss_mesh_create_ex(8, 8, 1.0, 1.0, 2, ctypes.byref(h)) == 1   # unknown top condition
    assert lib.chnss_ctx_create(None, None, None, ctypes.byref(h)) == 1
    assert lib.chnss_step(None, None, None, None) == 1
    assert lib.chnss_system_size(None, 0) == -1
    assert lib.chnss_mesh_destroy(None) == 0
    assert lib.chnss_ctx_destroy(None) == 0
    assert lib.chnss_step_batched(-1, None, None, None, None, 0) == 1
    assert lib.chnss_step_batched(0, None, None, None, None, 0) == 0     # empty batch: nothing to do
    hs = (ctypes.c_void_p * 2)(None, None)
    two = (chnss.State * 2)()
    assert lib.chnss_step_batched(2, hs, two, two, None, 0) == 1         # null context
    assert lib.chnss_autotune(None, None) == 1
    assert lib.chnss_set_spmv_block(None, 256, 256) == 1
    assert lib.chnss_set_step_concurrency(None, 1) == 1
    assert lib.chnss_diagnostics(None, None, None) == 1


def test_params_struct_matches_header():
    text = open(HEADER).read()
    body = text[text.index("typedef struct {\n  double tau;"):text.index("} chnss_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith("typedef"):
            decl = decl.replace("typedef struct {", "").strip()
            if not decl:
                continue
        typ, rest = decl.split(None, 1)
        for nm in rest.split(","):
            fields.append(re.sub(r"\[.*\]", "", nm).strip())
    assert fields == [f for f, _ in chnss.Params._fields_]


def test_three_d_argument_errors_need_no_device(lib):
    """chnss3_ctx_create / _create_ex reject bad meshes and parameter sets on
    the host, before any device call."""
    from paper_2501_11767_gb300 import inputs
    h = ctypes.c_void_p()

    def create(n, top_bc=0, **kw):
        p = chnss.make_params(dict(inputs.default_params(), **kw))
        return lib.chnss3_ctx_create_ex(n, top_bc, ctypes.byref(p), None, ctypes.byref(h))

    assert create(3) == 1                                    # odd n
    assert create(66) == 1                                   # above the 3D size limit (int32 host counts)
    assert create(4, top_bc=2) == 1                          # unknown top condition
    assert b"top_bc" in lib.chnss_last_error(None)
    assert create(4, mobility_kind=2) == 1
    assert create(4, inner_rtol=1.5) == 1
    assert create(4, inner_rtol=1e-4, inner_maxit=0) == 1
    assert create(4, model=1) == 1                           # solvent-air sub-model is 2D only
    assert create(4, precision=3) == 1
    assert create(4, tau=0.0) == 1
    assert lib.chnss3_ctx_create(4, None, None, ctypes.byref(h)) == 1
    assert lib.chnss3_step(None, None, None, None) == 1
    assert lib.chnss3_sizes(None, None, None) == 1
    assert lib.chnss3_set_step_concurrency(None, 1) == 1
    assert lib.chnss3_ctx_destroy(None) == 0


def test_binding_checks_array_sizes_and_placement():
    """The C ABI takes bare pointers; the binding refuses arrays that are too
    short or on the wrong side (host vs device) before any call."""
    import numpy as np
    import torch
    from paper_2501_11767_gb300 import inputs
    N1, N2 = 25, 81
    host = {"phi": np.zeros((3, N1)), "mu": np.zeros((4, N1)), "Phi_v": np.zeros(N1), "v": np.zeros(2 * N2),
            "p": np.zeros(N1)}
    chnss.make_state(host, N1, N2, 2, "host")
    with pytest.raises(ValueError):
        chnss.make_state(host, N1, N2, 2, "device")              # numpy is never a device array
    with pytest.raises(ValueError):
        chnss.make_state(dict(host, v=np.zeros(2 * N2 - 1)), N1, N2, 2, "host")
    with pytest.raises(ValueError):
        chnss.make_state(host, N1, N2, 3, "host")                 # 3D velocity is longer
    cpu = {k: torch.as_tensor(v) for k, v in host.items()}
    chnss.make_state(cpu, N1, N2, 2, "host")
    with pytest.raises(ValueError):
        chnss.make_state(cpu, N1, N2, 2, "device")                # CPU tensor where a device pointer goes
    with pytest.raises(ValueError):
        chnss._ptr(torch.zeros(4, dtype=torch.float32))
    n = 2
    st3 = inputs.initial_state_3d(n, seed=0)
    with pytest.raises(ValueError):
        chnss.host_operator3(n, "C1", inputs.default_params(), dict(st3, v=st3["v"][:-3].copy()))


def test_amg_argument_errors_need_no_device(lib):
    h = ctypes.c_void_p()
    assert lib.chnss_amg_create(0, 0, None, None, None, 0, ctypes.byref(h)) == 1
    assert lib.chnss_amg_create(4, 4, None, None, None, 0, ctypes.byref(h)) == 1
    assert lib.chnss_amg_create(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 2,
                                ctypes.byref(h)) == 1          # unknown precision
    assert b"precision" in lib.chnss_last_error(None)
    assert lib.chnss_amg_create(4, 4, None, None, None, 0, None) == 1
    assert lib.chnss_amg_update(None, None) == 1
    assert lib.chnss_amg_vcycle(None, None, None) == 1
    assert lib.chnss_amg_solve(None, None, None, 1e-8, 0.0, 10, None) == 1
    lib.chnss_amg_destroy(None)


def test_batch_mode_argument_errors_need_no_device(lib):
    assert lib.chnss_set_batch_mode(2) == 1
    assert b"batch mode" in lib.chnss_last_error(None)
    a, b = ctypes.c_longlong(-1), ctypes.c_longlong(-1)
    assert lib.chnss_batch_stats(ctypes.byref(a), ctypes.byref(b)) == 0 and a.value >= 0 and b.value >= 0


def test_amg_binding_refuses_host_or_wrong_typed_arrays():
    """The binding passes bare device pointers: host arrays or wrong dtypes are
    refused before the C ABI is called (no device needed)."""
    torch = pytest.importorskip("torch")
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    col = torch.tensor([0, 1], dtype=torch.int32)
    val = torch.ones(2, dtype=torch.float64)
    with pytest.raises(ValueError):
        chnss.Amg(rp, col, val)                       # host tensors
    with pytest.raises(ValueError):
        chnss._int32_device(rp.to(torch.int64), 3)   # wrong index type
