"""Thin ctypes binding of the C ABI in ``include/vlbm.h`` (``libvlbm.so``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The functions keep the C names (``vlbm_create``,
``vlbm_init_fields``, ``vlbm_step``, ``vlbm_moments``, ``vlbm_destroy`` ...);
``Context`` wraps one ``vlbm_ctx*`` for convenience.

PyTorch is used only as plumbing: ``torch_hooks()`` routes the library's
device allocations through torch's caching allocator, and a torch stream can
be passed as the context's stream.  There is no CPU fallback: importing this
module fails loudly when the compiled library is missing or cannot load.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

VLBM_OK = 0
VLBM_ERR_ARG = 1
VLBM_ERR_UNSTABLE = 2
VLBM_ERR_OOM = 3
VLBM_ERR_CUDA = 4
VLBM_ERR_NONPHYSICAL = 5
VLBM_ERR_TIMEOUT = 6
VLBM_ERR_STATE = 7
VLBM_ERR_UNSUPPORTED = 8

VLBM_IDEAL = 0
VLBM_RESISTIVE = 1
VLBM_IDEAL_POWELL = 2
VLBM_DISSIPATIVE = 3
VLBM_BC_PERIODIC = 0
VLBM_BC_EQUILIBRIUM = 1
FACES = {"x-": 0, "x+": 1, "y-": 2, "y+": 3, "z-": 4, "z+": 5}

VLBM_F64 = 0
VLBM_F32 = 1
VLBM_F16_DEV = 2
VLBM_BF16_DEV = 3

STORAGE_NAMES = {"f64": VLBM_F64, "f32": VLBM_F32, "f16dev": VLBM_F16_DEV, "bf16dev": VLBM_BF16_DEV}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class vlbm_params(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int),
        ("dim", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("tau", ctypes.c_double * 8),
        ("source", ctypes.c_double * 8),
        ("force", ctypes.c_double * 3),
        ("b_wall", ctypes.c_double * 3),
        ("walls_y", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("q_ref", ctypes.c_double * 8),
        ("q_scale", ctypes.c_double * 8),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("dealloc", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("tau_d", ctypes.c_double),
        ("tau_m", ctypes.c_double),
        ("tau_g", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("eta0", ctypes.c_double),
        ("j_c", ctypes.c_double),
        ("powell", ctypes.c_int),
        ("p_theta", ctypes.c_double),
    ]


class vlbm_closure_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("mu", ctypes.c_double * 8),
        ("sigma", ctypes.c_double * 8),
        ("out_scale", ctypes.c_double * 8),
        ("lr", ctypes.c_double),
        ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


class VlbmError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__("%s: %s%s" % (what, status_string(status), (" (" + detail + ")") if detail else ""))


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libvlbm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libvlbm.so is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, i, d, s = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    pp = ctypes.POINTER(vlbm_params)
    sig = {
        "vlbm_default_params": (None, [pp]),
        "vlbm_create": (i, [pp, ctypes.POINTER(P)]),
        "vlbm_create_batch": (i, [pp, i, ctypes.POINTER(P)]),
        "vlbm_init_fields": (i, [P, i, P]),
        "vlbm_init_fields_device": (i, [P, i, P]),
        "vlbm_init_fields_f32": (i, [P, i, P]),
        "vlbm_moments_f32": (i, [P, i, P]),
        "vlbm_step": (i, [P, i]),
        "vlbm_sync": (i, [P]),
        "vlbm_moments": (i, [P, i, P]),
        "vlbm_moments_device": (i, [P, i, P]),
        "vlbm_gather_populations": (i, [P, i, P, i, P]),
        "vlbm_conservation": (i, [P, i, P]),
        "vlbm_save": (i, [P, P, ctypes.POINTER(s)]),
        "vlbm_load": (i, [P, P, s]),
        "vlbm_autotune": (i, [P, i, ctypes.POINTER(i)]),
        "vlbm_tile_shapes": (i, [P]),
        "vlbm_set_tile_shape": (i, [P, i]),
        "vlbm_nvar": (i, [P]),
        "vlbm_slots_per_cell": (i, [P]),
        "vlbm_num_domains": (i, [P]),
        "vlbm_num_cells": (ctypes.c_int64, [P, i]),
        "vlbm_step_count": (ctypes.c_int64, [P]),
        "vlbm_launch_count": (ctypes.c_int64, [P]),
        "vlbm_population_bytes": (s, [P]),
        "vlbm_stream": (P, [P]),
        "vlbm_last_error": (ctypes.c_char_p, [P]),
        "vlbm_status_string": (ctypes.c_char_p, [i]),
        "vlbm_destroy": (None, [P]),
        "vlbm_closure_create": (i, [ctypes.POINTER(vlbm_closure_params), ctypes.POINTER(P)]),
        "vlbm_closure_num_params": (s, [P]),
        "vlbm_closure_set_weights": (i, [P, P, s]),
        "vlbm_closure_get_weights": (i, [P, P, s]),
        "vlbm_closure_forward": (i, [P, P, P]),
        "vlbm_closure_backward": (i, [P, P, P, P]),
        "vlbm_closure_train_step": (i, [P, P, P, ctypes.POINTER(d)]),
        "vlbm_closure_train_step_ctx": (i, [P, P, P, ctypes.POINTER(d)]),
        "vlbm_closure_grad_step_ctx": (i, [P, P, P, ctypes.POINTER(d), P]),
        "vlbm_closure_apply_grads": (i, [P, P]),
        "vlbm_set_closure": (i, [P, P]),
        "vlbm_set_solid": (i, [P, P]),
        "vlbm_set_boundary": (i, [P, i, i, ctypes.c_uint, P]),
        "vlbm_porosity_from_distance": (i, [P, ctypes.c_int64, d, P, P]),
        "vlbm_closure_destroy": (None, [P]),
        "vlbm_restrict": (i, [P, i, i, i, i, P, P]),
        "vlbm_check_bounded_wait": (i, [P, i]),
        "vlbm_conservation_noalloc": (i, [P, i, i, i, i, i, ctypes.c_int64, i, P, P, P, P]),
        "vlbm_set_slab": (i, [P, i]),
        "vlbm_halo_bytes": (s, [P]),
        "vlbm_halo_pack": (i, [P, P, P]),
        "vlbm_halo_unpack": (i, [P, P, P]),
        "vlbm_slabs_step": (i, [ctypes.POINTER(P), i, i]),
        "vlbm_measure_fp64_rate": (i, [i, P, ctypes.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_string(status: int) -> str:
    return load().vlbm_status_string(int(status)).decode()


def last_error(ctx=None) -> str:
    msg = load().vlbm_last_error(ctx)
    return msg.decode() if msg else ""


def _check(status: int, what: str, ctx=None):
    if status != VLBM_OK:
        raise VlbmError(status, what, last_error(ctx))


def vlbm_default_params() -> vlbm_params:
    p = vlbm_params()
    load().vlbm_default_params(ctypes.byref(p))
    return p


def make_params(model: int = VLBM_IDEAL, shape=(64, 64, 64), storage="f32", gamma=5.0 / 3.0,
                tau=0.51, source=None, force=(0.0, 0.0, 0.0), b_wall=(0.0, 0.0, 0.0),
                walls_y: bool = False, check_every: int = 0, q_ref=None, q_scale=None,
                stream: Optional[int] = None, hooks=None, tau_d: float = 0.51,
                tau_m: float = 1.0, tau_g: float = 0.51, nu: float = 0.0, eta0: float = 0.0,
                j_c: float = 0.0, powell: bool = False, p_theta: float = 0.01) -> vlbm_params:
    """Parameters for one domain; ``shape`` is (ny, nx) in 2-D, (nz, ny, nx) in 3-D.

    ``tau_d`` / ``tau_m`` apply to the Powell model (VLBM_IDEAL_POWELL): the BGK
    time of the divergence lattice and the relaxation time of D (div B = D / tau_m).
    The dissipative model (VLBM_DISSIPATIVE) takes ``tau_m`` as the relaxation time
    of its gradient tensors G and W, ``tau_g`` as their lattices' BGK time, the
    viscosity ``nu``, the resistivity eta0 (1 + |j|^2 / j_c^2) and the Powell switch.
    ``p_theta``: deviation storage recomputes the gas pressure in FP64 in cells where
    the FP32 value is below p_theta * e_tot (0 disables).
    """
    p = vlbm_default_params()
    p.model = int(model)
    shape = tuple(int(n) for n in shape)
    if len(shape) == 2:
        p.dim, p.nz, p.ny, p.nx = 2, 1, shape[0], shape[1]
    else:
        p.dim, p.nz, p.ny, p.nx = 3, shape[0], shape[1], shape[2]
    p.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
    p.gamma = float(gamma)
    tau = np.broadcast_to(np.asarray(tau, dtype=float), (8,)) if np.ndim(tau) == 0 else \
        np.concatenate([np.asarray(tau, dtype=float), np.ones(8 - len(tau))])
    for k in range(8):
        p.tau[k] = float(tau[k])
        p.source[k] = float(source[k]) if source is not None else 0.0
        p.q_ref[k] = float(q_ref[k]) if q_ref is not None else 0.0
        p.q_scale[k] = float(q_scale[k]) if q_scale is not None else 1.0
    for a in range(3):
        p.force[a] = float(force[a])
        p.b_wall[a] = float(b_wall[a])
    p.walls_y = int(bool(walls_y))
    p.check_every = int(check_every)
    p.tau_d = float(tau_d)
    p.tau_m = float(tau_m)
    p.tau_g = float(tau_g)
    p.nu = float(nu)
    p.eta0 = float(eta0)
    p.j_c = float(j_c)
    p.powell = int(bool(powell))
    p.p_theta = float(p_theta)
    p.stream = stream if stream else None
    if hooks is not None:
        p.alloc, p.dealloc, p.alloc_user = hooks.alloc, hooks.dealloc, None
    return p


class TorchHooks:
    """Device allocator hooks backed by torch's caching allocator."""

    def __init__(self, device: int = 0):
        import torch
        self._torch = torch
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.dealloc = FREE_FN(_free)


def torch_hooks(device: int = 0) -> TorchHooks:
    return TorchHooks(device)


def vlbm_create(params: vlbm_params) -> int:
    ctx = ctypes.c_void_p()
    _check(load().vlbm_create(ctypes.byref(params), ctypes.byref(ctx)), "vlbm_create")
    return ctx.value


def vlbm_create_batch(params: Sequence[vlbm_params]) -> int:
    arr = (vlbm_params * len(params))(*params)
    ctx = ctypes.c_void_p()
    _check(load().vlbm_create_batch(arr, len(params), ctypes.byref(ctx)), "vlbm_create_batch")
    return ctx.value


def _device_inputs_ready():
    """Order torch's work before a library call that reads device memory.

    Library calls run on the context's stream, which does not synchronise
    with torch's current stream; device inputs produced by torch kernels must
    be complete before the call enqueues its work."""
    import sys as _sys
    torch = _sys.modules.get("torch")
    if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
        torch.cuda.current_stream().synchronize()


def _host_f64(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def vlbm_init_fields(ctx: int, domain: int, Q: np.ndarray) -> int:
    """Host fields Q [nvar, (nz,) ny, nx] float64; returns the status (raises on CUDA errors)."""
    Q = _host_f64(Q)
    st = load().vlbm_init_fields(ctx, domain, Q.ctypes.data_as(ctypes.c_void_p))
    if st not in (VLBM_OK, VLBM_ERR_UNSTABLE, VLBM_ERR_NONPHYSICAL):
        _check(st, "vlbm_init_fields", ctx)
    return st


def vlbm_init_fields_ptr(ctx: int, domain: int, host_ptr: int) -> int:
    """Host fields from a raw host address (for pinned buffers)."""
    return load().vlbm_init_fields(ctx, domain, ctypes.c_void_p(host_ptr))


def vlbm_init_fields_f32(ctx: int, domain: int, Q: np.ndarray) -> int:
    """Single-precision host fields Q [nvar, (nz,) ny, nx] (half the host-link bytes)."""
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    st = load().vlbm_init_fields_f32(ctx, domain, Q.ctypes.data_as(ctypes.c_void_p))
    if st not in (VLBM_OK, VLBM_ERR_UNSTABLE, VLBM_ERR_NONPHYSICAL):
        _check(st, "vlbm_init_fields_f32", ctx)
    return st


def vlbm_init_fields_f32_ptr(ctx: int, domain: int, host_ptr: int) -> int:
    return load().vlbm_init_fields_f32(ctx, domain, ctypes.c_void_p(host_ptr))


def vlbm_init_fields_device(ctx: int, domain: int, dev_ptr: int) -> int:
    _device_inputs_ready()
    st = load().vlbm_init_fields_device(ctx, domain, ctypes.c_void_p(dev_ptr))
    if st not in (VLBM_OK, VLBM_ERR_UNSTABLE, VLBM_ERR_NONPHYSICAL):
        _check(st, "vlbm_init_fields_device", ctx)
    return st


def vlbm_step(ctx: int, n: int) -> int:
    st = load().vlbm_step(ctx, int(n))
    if st not in (VLBM_OK, VLBM_ERR_NONPHYSICAL, VLBM_ERR_TIMEOUT):
        _check(st, "vlbm_step", ctx)
    return st


def vlbm_sync(ctx: int) -> int:
    st = load().vlbm_sync(ctx)
    if st not in (VLBM_OK, VLBM_ERR_NONPHYSICAL, VLBM_ERR_TIMEOUT):
        _check(st, "vlbm_sync", ctx)
    return st


def vlbm_nvar(ctx: int) -> int:
    return load().vlbm_nvar(ctx)


def vlbm_num_cells(ctx: int, domain: int = 0) -> int:
    return int(load().vlbm_num_cells(ctx, domain))


def vlbm_moments(ctx: int, domain: int, shape) -> np.ndarray:
    out = np.empty((vlbm_nvar(ctx),) + tuple(shape), dtype=np.float64)
    _check(load().vlbm_moments(ctx, domain, out.ctypes.data_as(ctypes.c_void_p)), "vlbm_moments", ctx)
    return out


def vlbm_moments_ptr(ctx: int, domain: int, host_ptr: int):
    _check(load().vlbm_moments(ctx, domain, ctypes.c_void_p(host_ptr)), "vlbm_moments", ctx)


def vlbm_moments_f32(ctx: int, domain: int, shape) -> np.ndarray:
    out = np.empty((vlbm_nvar(ctx),) + tuple(shape), dtype=np.float32)
    _check(load().vlbm_moments_f32(ctx, domain, out.ctypes.data_as(ctypes.c_void_p)), "vlbm_moments_f32", ctx)
    return out


def vlbm_moments_f32_ptr(ctx: int, domain: int, host_ptr: int):
    _check(load().vlbm_moments_f32(ctx, domain, ctypes.c_void_p(host_ptr)), "vlbm_moments_f32", ctx)


def vlbm_moments_device(ctx: int, domain: int, dev_ptr: int):
    _check(load().vlbm_moments_device(ctx, domain, ctypes.c_void_p(dev_ptr)), "vlbm_moments_device", ctx)


def vlbm_slots_per_cell(ctx: int) -> int:
    return load().vlbm_slots_per_cell(ctx)


def vlbm_gather_populations(ctx: int, domain: int, cells) -> np.ndarray:
    """Pre-collision populations [ncell, slots] at the listed linear cell indices."""
    cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty((len(cells), vlbm_slots_per_cell(ctx)), dtype=np.float64)
    _check(load().vlbm_gather_populations(ctx, domain, cells.ctypes.data_as(ctypes.c_void_p), len(cells),
                                          out.ctypes.data_as(ctypes.c_void_p)), "vlbm_gather_populations", ctx)
    return out


def vlbm_conservation(ctx: int, domain: int = 0) -> np.ndarray:
    """Domain sums of the conserved fields (the eight MHD fields for the Powell model)."""
    out = np.zeros(min(vlbm_nvar(ctx), 8), dtype=np.float64)
    _check(load().vlbm_conservation(ctx, domain, out.ctypes.data_as(ctypes.c_void_p)), "vlbm_conservation", ctx)
    return out


def vlbm_save(ctx: int) -> bytes:
    L = load()
    n = ctypes.c_size_t(0)
    _check(L.vlbm_save(ctx, None, ctypes.byref(n)), "vlbm_save", ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(L.vlbm_save(ctx, buf, ctypes.byref(n)), "vlbm_save", ctx)
    return buf.raw[:n.value]


def vlbm_load(ctx: int, data: bytes):
    _check(load().vlbm_load(ctx, data, len(data)), "vlbm_load", ctx)


def vlbm_autotune(ctx: int, steps: int = 10) -> int:
    ch = ctypes.c_int(0)
    _check(load().vlbm_autotune(ctx, int(steps), ctypes.byref(ch)), "vlbm_autotune", ctx)
    return ch.value


def vlbm_tile_shapes(ctx: int) -> int:
    return load().vlbm_tile_shapes(ctx)


def vlbm_set_tile_shape(ctx: int, shape: int):
    _check(load().vlbm_set_tile_shape(ctx, int(shape)), "vlbm_set_tile_shape", ctx)


def vlbm_step_count(ctx: int) -> int:
    return int(load().vlbm_step_count(ctx))


def vlbm_launch_count(ctx: int) -> int:
    return int(load().vlbm_launch_count(ctx))


def vlbm_population_bytes(ctx: int) -> int:
    return int(load().vlbm_population_bytes(ctx))


def vlbm_stream(ctx: int) -> int:
    return load().vlbm_stream(ctx) or 0


def vlbm_destroy(ctx: int):
    if ctx:
        load().vlbm_destroy(ctx)


def vlbm_conservation_noalloc(pop_ptr: int, storage, dim: int, nx: int, ny: int, nz: int, stride: int,
                              parity: int, sums_ptr: int, q_ref=None, q_scale=None, stream: int = 0) -> None:
    """Domain sums of the eight ideal-MHD fields from a caller-owned population buffer into 8
    caller-owned device doubles, allocating nothing (see vlbm.h); enqueued on `stream`."""
    st_code = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
    ref = scale = None
    if q_ref is not None:
        ref = np.ascontiguousarray(np.asarray(q_ref, dtype=np.float64).reshape(8))
    if q_scale is not None:
        scale = np.ascontiguousarray(np.asarray(q_scale, dtype=np.float64).reshape(8))
    _device_inputs_ready()
    _check(load().vlbm_conservation_noalloc(
        ctypes.c_void_p(pop_ptr), st_code, int(dim), int(nx), int(ny), int(nz), int(stride), int(parity),
        ref.ctypes.data_as(ctypes.c_void_p) if ref is not None else None,
        scale.ctypes.data_as(ctypes.c_void_p) if scale is not None else None,
        ctypes.c_void_p(sums_ptr), ctypes.c_void_p(stream) if stream else None), "vlbm_conservation_noalloc")


def vlbm_set_slab(ctx: int, on: bool = True) -> None:
    """Mark (or unmark) a context as one slab of a domain decomposed along its last axis."""
    _check(load().vlbm_set_slab(ctx, int(bool(on))), "vlbm_set_slab", ctx)


def vlbm_halo_bytes(ctx: int) -> int:
    """Bytes of one face message (lo or hi) of a slab."""
    return int(load().vlbm_halo_bytes(ctx))


def vlbm_halo_pack(ctx: int, lo_ptr: int, hi_ptr: int) -> None:
    """Enqueue the copy of the slab's face planes into two device buffers."""
    _check(load().vlbm_halo_pack(ctx, ctypes.c_void_p(lo_ptr), ctypes.c_void_p(hi_ptr)), "vlbm_halo_pack", ctx)


def vlbm_halo_unpack(ctx: int, lo_ptr: int, hi_ptr: int) -> None:
    """Enqueue the write of two received face messages into the slab's face planes."""
    _check(load().vlbm_halo_unpack(ctx, ctypes.c_void_p(lo_ptr), ctypes.c_void_p(hi_ptr)), "vlbm_halo_unpack", ctx)


def vlbm_slabs_step(ctx_ptrs, n: int) -> int:
    """n steps of the slabs of one domain in this process (one device, one stream),
    each step followed by their halo exchange; returns slab 0's health status."""
    arr = (ctypes.c_void_p * len(ctx_ptrs))(*ctx_ptrs)
    st = load().vlbm_slabs_step(arr, len(ctx_ptrs), int(n))
    if st not in (VLBM_OK, VLBM_ERR_NONPHYSICAL, VLBM_ERR_TIMEOUT):
        _check(st, "vlbm_slabs_step", ctx_ptrs[0] if st == VLBM_ERR_STATE else None)
    return st


def vlbm_measure_fp64_rate(iters: int = 4096, stream: int = 0) -> float:
    """FP64 FMA throughput of the current device's CUDA cores, TFLOP/s."""
    out = ctypes.c_double(0.0)
    _check(load().vlbm_measure_fp64_rate(int(iters), ctypes.c_void_p(stream) if stream else None,
                                         ctypes.byref(out)), "vlbm_measure_fp64_rate")
    return out.value


def vlbm_check_bounded_wait(ctx: int, tries: int = 64) -> None:
    """Enqueue the failure-detection self-check: a bounded wait that gives up and
    raises the context's timeout flag (the next sync returns VLBM_ERR_TIMEOUT)."""
    _check(load().vlbm_check_bounded_wait(ctx, int(tries)), "vlbm_check_bounded_wait", ctx)


def vlbm_restrict(Qf_ptr: int, shape, factor: int, Qc_ptr: int, stream: int = 0):
    """Conservative block average of 8 device fields (fine shape (nz, ny, nx))."""
    nz, ny, nx = shape
    _device_inputs_ready()
    _check(load().vlbm_restrict(ctypes.c_void_p(Qf_ptr), nx, ny, nz, factor, ctypes.c_void_p(Qc_ptr),
                                ctypes.c_void_p(stream) if stream else None), "vlbm_restrict")


def vlbm_set_boundary(ctx: int, face, kind: int, dirichlet_mask: int = 0, values=None) -> None:
    """Open (VLBM_BC_EQUILIBRIUM) or close (VLBM_BC_PERIODIC) one face (sec. 2.4,
    "Static boundaries"); face 0..5 or "x-", "x+", ...; bit k of the mask makes Q_k
    Dirichlet at values[k], the others are copied from the next cell inwards."""
    f = FACES[face] if isinstance(face, str) else int(face)
    buf = None
    if values is not None:
        buf = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(8))
    _check(load().vlbm_set_boundary(ctx, f, int(kind), int(dirichlet_mask),
                                    buf.ctypes.data_as(ctypes.c_void_p) if buf is not None else None),
           "vlbm_set_boundary", ctx)


def vlbm_set_solid(ctx: int, solid_ptr) -> None:
    """Attach homogenised solid fields ([7][N] float32 on the device: d, uB, BB) or detach (None)."""
    if solid_ptr:
        _device_inputs_ready()
    _check(load().vlbm_set_solid(ctx, solid_ptr if solid_ptr else None), "vlbm_set_solid", ctx)


def vlbm_porosity_from_distance(phi_ptr: int, n: int, eps_h: float, d_ptr: int, stream: int = 0) -> None:
    """d = porosity(phi) on the device (sec. 2.4); float32 arrays of n values."""
    _device_inputs_ready()
    _check(load().vlbm_porosity_from_distance(ctypes.c_void_p(phi_ptr), int(n), float(eps_h),
                                              ctypes.c_void_p(d_ptr), ctypes.c_void_p(stream) if stream else None),
           "vlbm_porosity_from_distance")


def vlbm_set_closure(ctx: int, closure) -> None:
    _check(load().vlbm_set_closure(ctx, closure.ptr if closure is not None else None), "vlbm_set_closure", ctx)


class Closure:
    """Learned flux closure (3-layer 3x3x3 conv net on the tensor cores)."""

    def __init__(self, shape, gamma: float, tau: float, mu, sigma, out_scale, lr: float = 1e-3,
                 beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream: int = 0):
        p = vlbm_closure_params()
        p.nz, p.ny, p.nx = (int(n) for n in shape)
        p.gamma, p.tau = float(gamma), float(tau)
        for k in range(8):
            p.mu[k], p.sigma[k], p.out_scale[k] = float(mu[k]), float(sigma[k]), float(out_scale[k])
        p.lr, p.beta1, p.beta2, p.eps = float(lr), float(beta1), float(beta2), float(eps)
        p.stream = stream if stream else None
        ptr = ctypes.c_void_p()
        _check(load().vlbm_closure_create(ctypes.byref(p), ctypes.byref(ptr)), "vlbm_closure_create")
        self.ptr = ptr.value
        self.shape = tuple(int(n) for n in shape)
        self.nparam = int(load().vlbm_closure_num_params(self.ptr))

    def set_weights(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.nparam
        _check(load().vlbm_closure_set_weights(self.ptr, flat.ctypes.data_as(ctypes.c_void_p), flat.size),
               "vlbm_closure_set_weights")

    def get_weights(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        _check(load().vlbm_closure_get_weights(self.ptr, out.ctypes.data_as(ctypes.c_void_p), out.size),
               "vlbm_closure_get_weights")
        return out

    def forward(self, Q_ptr: int, dphi_ptr: int):
        _device_inputs_ready()
        _check(load().vlbm_closure_forward(self.ptr, ctypes.c_void_p(Q_ptr), ctypes.c_void_p(dphi_ptr)),
               "vlbm_closure_forward")

    def backward(self, Q_ptr: int, gy_ptr: int) -> np.ndarray:
        _device_inputs_ready()
        out = np.empty(self.nparam, dtype=np.float32)
        _check(load().vlbm_closure_backward(self.ptr, ctypes.c_void_p(Q_ptr), ctypes.c_void_p(gy_ptr),
                                            out.ctypes.data_as(ctypes.c_void_p)), "vlbm_closure_backward")
        return out

    def train_step(self, Q0_ptr: int, Qt_ptr: int) -> float:
        _device_inputs_ready()
        loss = ctypes.c_double(0.0)
        _check(load().vlbm_closure_train_step(self.ptr, ctypes.c_void_p(Q0_ptr), ctypes.c_void_p(Qt_ptr),
                                              ctypes.byref(loss)), "vlbm_closure_train_step")
        return loss.value

    def train_step_ctx(self, ctx_ptr: int, Qt_ptr: int) -> float:
        """One Adam step along a coarse run: ctx advances one corrected step."""
        _device_inputs_ready()
        loss = ctypes.c_double(0.0)
        _check(load().vlbm_closure_train_step_ctx(self.ptr, ctx_ptr, ctypes.c_void_p(Qt_ptr),
                                                  ctypes.byref(loss)), "vlbm_closure_train_step_ctx", ctx_ptr)
        return loss.value

    def grad_step_ctx(self, ctx_ptr: int, Qt_ptr: int, grads_ptr: int) -> float:
        """Loss and gradient of one corrected step of ctx into grads (device floats); no update."""
        _device_inputs_ready()
        loss = ctypes.c_double(0.0)
        _check(load().vlbm_closure_grad_step_ctx(self.ptr, ctx_ptr, ctypes.c_void_p(Qt_ptr), ctypes.byref(loss),
                                                 ctypes.c_void_p(grads_ptr)), "vlbm_closure_grad_step_ctx", ctx_ptr)
        return loss.value

    def apply_grads(self, grads_ptr: int):
        """One Adam step with the gradient at grads_ptr (device floats)."""
        _device_inputs_ready()
        _check(load().vlbm_closure_apply_grads(self.ptr, ctypes.c_void_p(grads_ptr)), "vlbm_closure_apply_grads")

    def close(self):
        if self.ptr:
            load().vlbm_closure_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One library context (a single domain, or a batch of 2-D domains)."""

    def __init__(self, params, batch: bool = False, hooks: Optional[TorchHooks] = None):
        self._hooks = hooks  # keep the callbacks alive as long as the context
        if batch:
            self.params = list(params)
            self.ptr = vlbm_create_batch(self.params)
            first = self.params[0]
        else:
            self.params = [params]
            self.ptr = vlbm_create(params)
            first = params
        self.nvar = vlbm_nvar(self.ptr)
        self.nslot = vlbm_slots_per_cell(self.ptr)

    def shape(self, domain: int = 0):
        p = self.params[domain]
        return (p.ny, p.nx) if p.dim == 2 else (p.nz, p.ny, p.nx)

    def init_fields(self, Q, domain: int = 0) -> int:
        return vlbm_init_fields(self.ptr, domain, Q)

    def step(self, n: int) -> int:
        return vlbm_step(self.ptr, n)

    def sync(self) -> int:
        return vlbm_sync(self.ptr)

    def moments(self, domain: int = 0) -> np.ndarray:
        return vlbm_moments(self.ptr, domain, self.shape(domain))

    def init_fields_f32(self, Q, domain: int = 0) -> int:
        return vlbm_init_fields_f32(self.ptr, domain, Q)

    def moments_f32(self, domain: int = 0) -> np.ndarray:
        return vlbm_moments_f32(self.ptr, domain, self.shape(domain))

    def populations(self, cells, domain: int = 0) -> np.ndarray:
        return vlbm_gather_populations(self.ptr, domain, cells)

    def conservation(self, domain: int = 0) -> np.ndarray:
        return vlbm_conservation(self.ptr, domain)

    def set_boundary(self, face, kind: int = VLBM_BC_EQUILIBRIUM, dirichlet_mask: int = 0, values=None) -> None:
        """Open or close one face; see ``vlbm_set_boundary``."""
        vlbm_set_boundary(self.ptr, face, kind, dirichlet_mask, values)

    def set_solid(self, solid_ptr) -> None:
        """Attach ([7][N] float32 device fields d, uB, BB) or detach (None) homogenised solids.

        A moving object waits for the steps already enqueued (``sync()``: they read
        the array when they run), rewrites the array, and calls this again so that
        torch's writes are complete before the next step reads them."""
        vlbm_set_solid(self.ptr, solid_ptr)

    def set_slab(self, on: bool = True) -> None:
        """Mark this context as one slab of a decomposed domain (``vlbm_set_slab``)."""
        vlbm_set_slab(self.ptr, on)

    @property
    def halo_bytes(self) -> int:
        return vlbm_halo_bytes(self.ptr)

    def halo_pack(self, lo_ptr: int, hi_ptr: int) -> None:
        vlbm_halo_pack(self.ptr, lo_ptr, hi_ptr)

    def halo_unpack(self, lo_ptr: int, hi_ptr: int) -> None:
        vlbm_halo_unpack(self.ptr, lo_ptr, hi_ptr)

    def save(self) -> bytes:
        return vlbm_save(self.ptr)

    def load(self, data: bytes):
        vlbm_load(self.ptr, data)

    def autotune(self, steps: int = 10) -> int:
        return vlbm_autotune(self.ptr, steps)

    def tile_shapes(self) -> int:
        return vlbm_tile_shapes(self.ptr)

    def set_tile_shape(self, shape: int):
        vlbm_set_tile_shape(self.ptr, shape)

    @property
    def step_count(self) -> int:
        return vlbm_step_count(self.ptr)

    @property
    def launches(self) -> int:
        return vlbm_launch_count(self.ptr)

    @property
    def stream(self) -> int:
        return vlbm_stream(self.ptr)

    def close(self):
        if self.ptr:
            vlbm_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
