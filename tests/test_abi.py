"""C-ABI checks that need no GPU: the library builds, loads, exports every
function ``include/vlbm.h`` declares, the ctypes struct matches the C
layout, and argument validation answers before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vlbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(vlbm_\w+)\s*\([^;{]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def V():
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vlbm_create", "vlbm_init_fields", "vlbm_step", "vlbm_moments", "vlbm_destroy",
                     "vlbm_conservation", "vlbm_create_batch", "vlbm_save", "vlbm_load"):
        assert required in names
    assert len(names) >= 25


def test_library_exports_every_declared_symbol(V):
    lib = ctypes.CDLL(V.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", V.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(vlbm_\w+)\b", out))
    assert set(declared_functions()) <= exported


def test_binding_declares_a_signature_for_every_entry_point(V):
    # the thin binding marshals every call of the header (argument types set)
    lib = V.load()
    missing = [n for n in declared_functions() if getattr(lib, n).argtypes is None]
    assert not missing, missing


def test_params_struct_layout_matches_c(V):
    p = V.vlbm_default_params()
    assert (p.model, p.dim, p.nx, p.ny, p.nz, p.storage) == (0, 3, 64, 64, 64, V.VLBM_F32)
    assert abs(p.gamma - 5 / 3) < 1e-15
    assert list(p.tau) == [0.51] * 8
    assert list(p.q_scale) == [1.0] * 8
    assert list(p.source) == [0.0] * 8 and list(p.q_ref) == [0.0] * 8
    assert (p.walls_y, p.check_every) == (0, 0)
    assert p.stream is None and p.alloc_user is None
    assert (p.tau_d, p.tau_m, p.tau_g) == (0.51, 1.0, 0.51)
    assert (p.nu, p.eta0, p.j_c, p.powell, p.p_theta) == (0.0, 0.0, 0.0, 0, 0.01)


def test_status_strings(V):
    assert V.status_string(V.VLBM_OK) == "VLBM_OK"
    assert V.status_string(V.VLBM_ERR_NONPHYSICAL) == "VLBM_ERR_NONPHYSICAL"
    assert V.status_string(99) == "unknown status"


def _create_status(V, p):
    ctx = ctypes.c_void_p()
    st = V.load().vlbm_create(ctypes.byref(p), ctypes.byref(ctx))
    if st == V.VLBM_OK:
        V.vlbm_destroy(ctx.value)
    return st


def test_validation_before_any_device_work(V):
    L = V.load()
    p = V.make_params(shape=(8, 8, 8), tau=0.5)
    assert _create_status(V, p) == V.VLBM_ERR_UNSTABLE
    p = V.make_params(shape=(8, 8, 8))
    p.dim = 4
    assert _create_status(V, p) == V.VLBM_ERR_ARG
    p = V.make_params(shape=(8, 8), gamma=1.0)
    assert _create_status(V, p) == V.VLBM_ERR_ARG
    p = V.make_params(model=V.VLBM_RESISTIVE, shape=(8, 8, 8), storage="f16dev")
    assert _create_status(V, p) == V.VLBM_ERR_UNSUPPORTED
    p = V.make_params(model=V.VLBM_RESISTIVE, shape=(8, 2, 8), walls_y=True)
    assert _create_status(V, p) == V.VLBM_ERR_ARG
    p = V.make_params(shape=(8, 8, 8))
    p.nz = 0
    assert _create_status(V, p) == V.VLBM_ERR_ARG
    # the dissipative model: 2-D or 3-D, F32 / F64, tau_g > 1/2, nu and eta0 >= 0
    p = V.make_params(model=V.VLBM_DISSIPATIVE, shape=(8, 8, 8), storage="bf16dev")
    assert _create_status(V, p) == V.VLBM_ERR_UNSUPPORTED
    p = V.make_params(model=V.VLBM_DISSIPATIVE, shape=(8, 8), storage="bf16dev")
    assert _create_status(V, p) == V.VLBM_ERR_UNSUPPORTED
    p = V.make_params(model=V.VLBM_DISSIPATIVE, shape=(8, 8), tau_g=0.5)
    assert _create_status(V, p) == V.VLBM_ERR_UNSTABLE
    p = V.make_params(model=V.VLBM_DISSIPATIVE, shape=(8, 8), eta0=-1e-3)
    assert _create_status(V, p) == V.VLBM_ERR_ARG
    p = V.make_params(shape=(8, 8))
    p.model = 4
    assert _create_status(V, p) == V.VLBM_ERR_ARG
    # deviation storage: the FP64 pressure-recovery threshold must be finite and >= 0
    p = V.make_params(shape=(8, 8, 8), storage="f16dev", p_theta=-0.1)
    assert _create_status(V, p) == V.VLBM_ERR_ARG
    # NULL contexts and pointers are argument errors, never crashes
    assert L.vlbm_step(None, 1) == V.VLBM_ERR_ARG
    assert L.vlbm_sync(None) == V.VLBM_ERR_ARG
    assert L.vlbm_moments(None, 0, None) == V.VLBM_ERR_ARG
    assert L.vlbm_init_fields(None, 0, None) == V.VLBM_ERR_ARG
    assert L.vlbm_conservation(None, 0, None) == V.VLBM_ERR_ARG
    assert L.vlbm_init_fields_f32(None, 0, None) == V.VLBM_ERR_ARG
    assert L.vlbm_moments_f32(None, 0, None) == V.VLBM_ERR_ARG
    assert L.vlbm_check_bounded_wait(None, 64) == V.VLBM_ERR_ARG
    assert L.vlbm_set_slab(None, 1) == V.VLBM_ERR_ARG
    assert L.vlbm_halo_pack(None, None, None) == V.VLBM_ERR_ARG
    assert L.vlbm_halo_unpack(None, None, None) == V.VLBM_ERR_ARG
    assert L.vlbm_halo_bytes(None) == 0
    assert L.vlbm_slabs_step(None, 2, 1) == V.VLBM_ERR_ARG
    assert L.vlbm_measure_fp64_rate(4096, None, None) == V.VLBM_ERR_ARG
    assert L.vlbm_closure_grad_step_ctx(None, None, None, None, None) == V.VLBM_ERR_ARG
    assert L.vlbm_closure_apply_grads(None, None) == V.VLBM_ERR_ARG
    assert L.vlbm_closure_train_step_ctx(None, None, None, None) == V.VLBM_ERR_ARG
    assert L.vlbm_nvar(None) == 0
    L.vlbm_destroy(None)


def test_create_without_a_device_reports_cuda_error(V):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    st = _create_status(V, V.make_params(shape=(8, 8, 8)))
    assert st == V.VLBM_ERR_CUDA
    assert V.last_error()  # one-line reason recorded
