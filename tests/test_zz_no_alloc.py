"""The allocation-free domain sums (vlbm_conservation_noalloc) agree with the
context entry point (vlbm_conservation) on the same population buffer.

Callers that cannot allocate device memory (an embedding host that owns every
allocation, a loop that must not pay for cudaMalloc) pass their own buffers;
the partial sums live in a fixed array inside the library.  The buffer used
here is the context's own, found through the public allocator hooks.  Two
calls in a row must give the context's sums to the FP64 test tolerance and
identical values to each other.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu


def _noalloc_fn(vlbm):
    L = vlbm.load()
    fn = L.vlbm_conservation_noalloc
    P, i = ctypes.c_void_p, ctypes.c_int
    fn.argtypes = [P, i, i, i, i, i, ctypes.c_int64, i, P, P, P, P]
    fn.restype = i
    return fn


# (storage, shape, steps): several 65,536-cell reduction blocks with a partial
# last one (163,840 cells: 3 blocks; 210,000 cells: 4 blocks) at both AA
# parities, 2-D (D2Q5) and 3-D (D3Q7), plain and deviation storage, and one
# domain smaller than a block.
CASES = [
    ("f64", (40, 64, 64), 4),
    ("f64", (40, 64, 64), 5),
    ("f32", (40, 64, 64), 5),
    ("f16dev", (40, 64, 64), 3),
    ("bf16dev", (12, 20, 70), 5),
    ("f32", (12, 20, 70), 0),
    ("f64", (300, 700), 2),
    ("f64", (300, 700), 3),
    ("f16dev", (300, 700), 1),
]


@pytest.mark.parametrize("storage,shape,steps", CASES)
def test_noalloc_sums_match_context_sums(storage, shape, steps):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    fn = _noalloc_fn(vlbm)

    allocs = []

    class Recording(vlbm.TorchHooks):
        def __init__(self):
            super().__init__(0)
            inner = self.alloc

            def rec(nbytes, stream, user):
                p = inner(nbytes, stream, user)
                allocs.append((p, nbytes))
                return p
            self.alloc = vlbm.ALLOC_FN(rec)

    hooks = Recording()
    dim = len(shape)
    f0 = fields.ideal_fields(shape, 909, mach=1.0, beta=1.0, cfl=0.2 if dim == 3 else 0.1)
    flat = f0.Q.reshape(8, -1)
    qref = flat.mean(1)
    qscale = np.abs(flat - qref[:, None]).max(1)
    p = vlbm.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=0.6, q_ref=qref,
                         q_scale=qscale, hooks=hooks)
    ctx = vlbm.Context(p, hooks=hooks)
    try:
        nbytes = vlbm.vlbm_population_bytes(ctx.ptr)
        pop = [a for a, n in allocs if n == nbytes]
        assert len(pop) == 1
        assert ctx.init_fields(f0.Q) == vlbm.VLBM_OK
        ctx.step(steps)
        ref = ctx.conservation()
        nz, ny, nx = (1,) + tuple(shape) if dim == 2 else shape
        ncell = nx * ny * nz
        stride = (ncell + 63) // 64 * 64  # the context's layout: cell count rounded up to 64 elements
        slots = 40 if dim == 2 else 56
        assert nbytes == slots * stride * {"f64": 8, "f32": 4}.get(storage, 2)
        qr = np.ascontiguousarray(qref, dtype=np.float64)
        qs = np.ascontiguousarray(qscale, dtype=np.float64)
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        scale = np.abs(flat).sum(1)
        results = []
        n_alloc = len(allocs)
        for _ in range(2):
            out.fill_(-1.0)
            torch.cuda.synchronize()
            st = fn(pop[0], vlbm.STORAGE_NAMES[storage], dim, nx, ny, nz, stride, steps & 1,
                    qr.ctypes.data, qs.ctypes.data, out.data_ptr(), ctx.stream)
            assert st == vlbm.VLBM_OK, vlbm.last_error()
            vlbm.vlbm_sync(ctx.ptr)
            got = out.cpu().numpy()
            assert (np.abs(got - ref) / scale).max() < 1e-12, (got, ref)
            results.append(got)
        assert len(allocs) == n_alloc, "the allocation-free sums allocated through the context's hooks"
        assert np.array_equal(results[0], results[1])
        # sizes beyond the fixed scratch are refused before any device work
        st = fn(pop[0], vlbm.STORAGE_NAMES[storage], 3, 1024, 1024, 512, 1024 * 1024 * 512, 0,
                qr.ctypes.data, qs.ctypes.data, out.data_ptr(), ctx.stream)
        assert st == vlbm.VLBM_ERR_ARG and "2^28" in vlbm.last_error()
    finally:
        ctx.close()
