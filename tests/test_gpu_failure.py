"""Failure detection without a GPU fault: the error paths are forced on the
host (an allocator that refuses, non-physical fields) or by a bounded device
wait that is made to give up, and each must come back as a status while the
context stays usable.  Nothing here faults, traps or hangs a GPU."""
import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def rel_err(got, ref):
    scale = np.maximum(np.abs(ref).reshape(ref.shape[0], -1).max(1), 1e-300)
    return (np.abs(got - ref).reshape(ref.shape[0], -1).max(1) / scale).max()


def test_bounded_wait_gives_up_and_the_context_recovers(V):
    shape = (16, 24)
    f0 = fields.ideal_fields(shape, 81)
    p = V.make_params(shape=shape, storage="f64", gamma=f0.gamma, tau=0.6)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        assert ctx.step(3) == V.VLBM_OK
        V.vlbm_check_bounded_wait(ctx.ptr, 64)  # a wait no arrival completes: gives up in ~1 ms
        assert ctx.sync() == V.VLBM_ERR_TIMEOUT
        assert ctx.step(1) == V.VLBM_ERR_TIMEOUT  # sticky
        with pytest.raises(V.VlbmError):
            V.vlbm_check_bounded_wait(ctx.ptr, 0)  # tries outside 1 .. 65536
        # a fresh init clears the failure, and the context computes as before
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        assert ctx.step(5) == V.VLBM_OK
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    assert rel_err(got, oracle.ideal_run(f0.Q, f0.gamma, 0.6, 5)) < 1e-12


class _Hooks:
    """Device allocator hooks over torch's caching allocator that refuse every
    allocation after the first `allow` (host-side fault injection)."""

    def __init__(self, V, allow):
        import torch
        self.count = 0
        self.live = {}

        def _alloc(nbytes, stream, user):
            self.count += 1
            if self.count > allow:
                return None
            ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream))
            self.live[ptr] = nbytes
            return ptr

        def _free(ptr, nbytes, stream, user):
            self.live.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = V.ALLOC_FN(_alloc)
        self.dealloc = V.FREE_FN(_free)


def test_refused_allocations_come_back_as_oom(V):
    shape = (8, 12, 16)
    f0 = fields.ideal_fields(shape, 82, cfl=0.2)
    # nothing allowed: the context cannot be created, and nothing is left behind
    h = _Hooks(V, 0)
    with pytest.raises(V.VlbmError) as e:
        V.Context(V.make_params(shape=shape, storage="f32", gamma=f0.gamma, hooks=h), hooks=h)
    assert e.value.status == V.VLBM_ERR_OOM
    assert not h.live
    # populations and status memory allowed, the host-field staging refused: the
    # host init reports OOM, the device init (no staging) still works
    import torch
    h = _Hooks(V, 2)
    with V.Context(V.make_params(shape=shape, storage="f32", gamma=f0.gamma, hooks=h), hooks=h) as ctx:
        with pytest.raises(V.VlbmError) as e:
            ctx.init_fields(f0.Q)
        assert e.value.status == V.VLBM_ERR_OOM
        Qd = torch.from_numpy(f0.Q).cuda()
        assert V.vlbm_init_fields_device(ctx.ptr, 0, Qd.data_ptr()) == V.VLBM_OK
        assert ctx.step(4) == V.VLBM_OK and ctx.sync() == V.VLBM_OK
        s = ctx.conservation()
        assert np.isfinite(s).all()
    assert not h.live  # every block the context took went back through the hook
