"""Single-precision host fields (vlbm_init_fields_f32, vlbm_moments_f32): half
the bytes over the host link, the same arithmetic.  The init widens each staged
chunk to double before the usual init kernel, so it must equal
vlbm_init_fields on the float-rounded fields bit for bit; the moments of FP32
storage are FP32 sums, so the float read-back must equal the double one
exactly, and that of 16-bit storage its round-to-nearest float."""
import numpy as np
import pytest

from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def both_ways(V, p, Q, steps, probe=None):
    q32 = np.asarray(Q, dtype=np.float32)
    out = []
    for f32 in (True, False):
        with V.Context(p) as ctx:
            st = ctx.init_fields_f32(q32) if f32 else ctx.init_fields(q32.astype(np.float64))
            assert st == V.VLBM_OK, V.status_string(st)
            ctx.step(steps)
            m64 = ctx.moments()
            m32 = ctx.moments_f32()
            cells = np.arange(0, m64[0].size, max(1, m64[0].size // 97), dtype=np.int64)
            pops = ctx.populations(cells)
            assert ctx.sync() == V.VLBM_OK
        np.testing.assert_array_equal(m32, m64.astype(np.float32))  # FP32 read-back: RN of the double one
        out.append((m64, pops))
    return out


@pytest.mark.parametrize("shape", [(24, 40), (6, 10, 36), (2100, 2048)])  # the last: two staging chunks
def test_ideal_f32_fields_match_rounded_double_fields(V, shape):
    f0 = fields.ideal_fields(shape, 61, mach=1.0, cfl=0.1 if len(shape) == 2 else 0.2)
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.6)
    (a, pa), (b, pb) = both_ways(V, p, f0.Q, 5)
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(a, b)


def test_dissipative_and_powell_f32_fields(V):
    shape = (12, 40)
    f0 = fields.ideal_fields(shape, 62, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(62)
    Qd = np.concatenate([f0.Q, 0.001 * rng.normal(size=(12,) + shape)])
    p = V.make_params(model=V.VLBM_DISSIPATIVE, shape=shape, storage="f32", gamma=f0.gamma, tau=0.6, tau_g=0.7,
                      tau_m=2.0, nu=0.02, eta0=0.03, j_c=0.05, powell=True)
    (a, pa), (b, pb) = both_ways(V, p, Qd, 4)
    np.testing.assert_array_equal(pa, pb)
    Qp = np.concatenate([f0.Q, np.zeros((1,) + shape)])
    p = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, storage="f32", gamma=f0.gamma, tau=0.6)
    (a, pa), (b, pb) = both_ways(V, p, Qp, 4)
    np.testing.assert_array_equal(pa, pb)


def test_resistive_f32_fields(V):
    shape = (8, 12, 32)
    setup = fields.hartmann_setup(shape, 63, Ha=10.0)
    p = V.make_params(model=V.VLBM_RESISTIVE, shape=shape, storage="f32",
                      tau=[setup.tau_f, setup.tau_m, setup.tau_m, setup.tau_m], force=setup.force,
                      b_wall=setup.b_wall, walls_y=True)
    (a, pa), (b, pb) = both_ways(V, p, setup.Q, 3)
    np.testing.assert_array_equal(pa, pb)


@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
def test_deviation_storage_f32_fields(V, storage):
    shape = (6, 8, 32)
    f0 = fields.ideal_fields(shape, 64, mach=1.0, cfl=0.2)
    flat = f0.Q.reshape(8, -1)
    qref = flat.mean(1)
    qscale = np.maximum(np.abs(flat - qref[:, None]).max(1), 1e-30)
    p = V.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=0.6, q_ref=qref, q_scale=qscale)
    (a, pa), (b, pb) = both_ways(V, p, f0.Q, 3)
    np.testing.assert_array_equal(pa, pb)


def test_f64_storage_refuses_f32_fields(V):
    shape = (8, 16)
    f0 = fields.ideal_fields(shape, 65)
    with V.Context(V.make_params(shape=shape, storage="f64", gamma=f0.gamma)) as ctx:
        with pytest.raises(V.VlbmError) as e:
            ctx.init_fields_f32(f0.Q)
        assert e.value.status == V.VLBM_ERR_UNSUPPORTED
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        with pytest.raises(V.VlbmError) as e:
            ctx.moments_f32()
        assert e.value.status == V.VLBM_ERR_UNSUPPORTED
