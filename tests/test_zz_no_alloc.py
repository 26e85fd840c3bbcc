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


@pytest.mark.parametrize("storage,steps", [("f64", 3), ("f32", 4), ("bf16dev", 5), ("f32", 0)])
def test_noalloc_sums_match_context_sums(storage, steps):
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
    shape = (12, 20, 70)
    f0 = fields.ideal_fields(shape, 909, mach=1.0, beta=1.0, cfl=0.2)
    qref = f0.Q.reshape(8, -1).mean(1)
    qscale = np.abs(f0.Q - qref.reshape(8, 1, 1, 1)).reshape(8, -1).max(1)
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
        nz, ny, nx = shape
        ncell = nx * ny * nz
        stride = (ncell + 63) // 64 * 64
        qr = np.ascontiguousarray(qref, dtype=np.float64)
        qs = np.ascontiguousarray(qscale, dtype=np.float64)
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        scale = np.abs(f0.Q).reshape(8, -1).sum(1)
        results = []
        for _ in range(2):
            out.fill_(-1.0)
            torch.cuda.synchronize()
            st = fn(pop[0], vlbm.STORAGE_NAMES[storage], 3, nx, ny, nz, stride, steps & 1,
                    qr.ctypes.data, qs.ctypes.data, out.data_ptr(), ctx.stream)
            assert st == vlbm.VLBM_OK, vlbm.last_error()
            vlbm.vlbm_sync(ctx.ptr)
            got = out.cpu().numpy()
            assert (np.abs(got - ref) / scale).max() < 1e-12, (got, ref)
            results.append(got)
        assert np.array_equal(results[0], results[1])
        # sizes beyond the fixed scratch are refused before any device work
        st = fn(pop[0], vlbm.STORAGE_NAMES[storage], 3, 1024, 1024, 512, 1024 * 1024 * 512, 0,
                qr.ctypes.data, qs.ctypes.data, out.data_ptr(), ctx.stream)
        assert st == vlbm.VLBM_ERR_ARG and "2^28" in vlbm.last_error()
    finally:
        ctx.close()
