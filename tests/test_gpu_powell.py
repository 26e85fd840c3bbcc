"""Ideal MHD with the Powell correction (model VLBM_IDEAL_POWELL) on the GPU
against the FP64 oracle (sec. 2.3, "Powell correction"; sec. 2.2.1, local
moments evolution: the ninth lattice carries D with div B = D / tau_M).

Tolerances as for the ideal model: FP64 storage 1e-12, FP32 storage 1e-5,
relative to max(the field's maximum, its reference scale).  D's reference
scale is tau_M max|B| (D ~ tau_M grad B on the unit lattice): D is built from
differences of B, so its FP32 round-off scales with B, not with D.
"""
import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu

TAU = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]
TAU_D, TAU_M = 0.7, 2.0


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def powell_fields(shape, seed):
    # the ideal recipe with a non-solenoidal part added to B_x, and D from rest
    f0 = fields.ideal_fields(shape, seed, mach=1.0, beta=1.0, cfl=0.2)
    Q = f0.Q.copy()
    nx = shape[-1]
    x = np.arange(nx)
    bump = 0.05 * np.abs(Q[5:8]).max() * np.sin(2 * np.pi * x / nx)
    Q[5] += bump  # div B != 0 along x
    Q[4] += 0.5 * ((Q[5] ** 2) - (f0.Q[5] ** 2))  # keep the gas pressure
    rng = np.random.default_rng(seed)
    D = 0.01 * np.abs(Q[5:8]).max() * rng.normal(size=shape)
    return np.concatenate([Q, D[None]]), f0.gamma


def field_errors(got, ref):
    scale = np.maximum(np.abs(ref).reshape(ref.shape[0], -1).max(1), 1e-300)
    scale[8] = max(scale[8], TAU_M * np.abs(ref[5:8]).max())
    return np.abs(got - ref).reshape(ref.shape[0], -1).max(1) / scale


@pytest.mark.parametrize("shape", [(12, 130), (5, 9, 33), (4, 6, 64)])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("steps", [4, 5])
def test_powell_matches_oracle(V, shape, storage, tol, steps):
    Q0, gamma = powell_fields(shape, 31)
    p = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, storage=storage, gamma=gamma, tau=TAU,
                      tau_d=TAU_D, tau_m=TAU_M)
    with V.Context(p) as ctx:
        assert ctx.nvar == 9
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(steps)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    ref = oracle.powell_run(Q0, gamma, TAU + [TAU_D], TAU_M, steps)
    err = field_errors(got, ref)
    assert err.max() < tol, err


def test_powell_populations_at_odd_parity(V):
    shape = (4, 6, 64)
    Q0, gamma = powell_fields(shape, 32)
    p = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, storage="f64", gamma=gamma, tau=TAU,
                      tau_d=TAU_D, tau_m=TAU_M)
    f = oracle.powell_init(Q0, gamma)
    for _ in range(3):
        f = oracle.powell_step(f, gamma, TAU + [TAU_D], TAU_M)
    cells = np.array([0, 1, 63, 64, 200, 383, 1000, 1535], dtype=np.int64)
    with V.Context(p) as ctx:
        assert ctx.nslot == 63
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(3)
        got = ctx.populations(cells)
    ref = f.reshape(9 * 7, -1)[:, cells].T
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_powell_uniform_state_D_decays_geometrically(V):
    # a uniform state stays uniform and D loses the fraction 1/tau_M per step
    # (the state satisfies the init check |u| + c_f < cs: c_f ~ 0.40 < 0.5)
    shape = (4, 4, 16)
    Q0 = np.array([1.1, 0.0, 0.0, 0.0, 0.15, 0.1, -0.05, 0.05, 0.04])
    Q = np.broadcast_to(Q0.reshape(9, 1, 1, 1), (9,) + shape).copy()
    tau_m = 3.0
    p = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, storage="f64", tau=0.6, tau_d=0.6, tau_m=tau_m)
    with V.Context(p) as ctx:
        assert ctx.init_fields(Q) == V.VLBM_OK
        ctx.step(7)
        got = ctx.moments()
    np.testing.assert_allclose(got[8], Q0[8] * (1 - 1 / tau_m) ** 7, rtol=1e-13)
    assert np.ptp(got.reshape(9, -1), axis=1).max() < 1e-14


def test_powell_api_contract(V):
    shape = (4, 6, 16)
    Q0, gamma = powell_fields(shape, 33)
    p = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, storage="f32", gamma=gamma, tau_d=TAU_D,
                      tau_m=TAU_M)
    with V.Context(p) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        m0 = ctx.conservation()
        assert m0.shape == (8,)  # the eight MHD fields; D is not conserved
        ctx.step(6)
        m1 = ctx.conservation()
        assert abs(m1[0] - m0[0]) <= 1e-6 * abs(m0[0])  # mass: Powell has no mass source
    for storage in ("f16dev", "bf16dev"):
        bad = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, storage=storage)
        with pytest.raises(Exception):
            V.Context(bad)
    for tau_d, tau_m in ((0.5, 1.0), (0.6, 0.4)):
        bad = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, tau_d=tau_d, tau_m=tau_m)
        with pytest.raises(Exception):
            V.Context(bad)


def test_powell_512cubed_light_cones(V):
    """The benchmark's Powell leg at its size: 512^3, FP32, tau 0.51, tau_M 1, D from
    rest, the headline fields; after 4 + 4 steps (the leg's first calls) the moments
    of sampled cells (corners, faces, interior) equal the oracle run on the periodic
    (2n+1)^3 box centred on each (a cell after n D3Q7 steps depends only on cells
    within L1 distance n)."""
    import torch
    n, steps = 512, 8
    shape = (n, n, n)
    f0 = fields.ideal_fields(shape, 3003, gamma=5.0 / 3.0, mach=2.0, beta=1.0, cfl=0.2,
                             device=torch.device("cuda"))
    Q = torch.cat([f0.Q, torch.zeros((1,) + shape, dtype=f0.Q.dtype, device=f0.Q.device)])
    gamma = f0.gamma
    del f0
    p = V.make_params(model=V.VLBM_IDEAL_POWELL, shape=shape, storage="f32", gamma=gamma, tau=0.51,
                      tau_d=0.51, tau_m=1.0, stream=torch.cuda.Stream().cuda_stream)
    cells = [(0, 0, 0), (511, 511, 511), (0, 256, 511), (300, 0, 17), (128, 400, 255), (511, 1, 128),
             (63, 511, 0), (200, 99, 129)]
    w = steps
    boxes = []
    for z, y, x in cells:
        iz, iy, ix = (torch.arange(c - w, c + w + 1, device=Q.device) % n for c in (z, y, x))
        boxes.append(Q[:, iz][:, :, iy][:, :, :, ix].cpu().numpy())
    scale = Q.abs().reshape(9, -1).amax(1).cpu().numpy()
    scale[1:4] = scale[1:4].max()
    scale[5:8] = scale[5:8].max()
    scale[8] = 1.0 * scale[5:8].max()  # D ~ tau_M grad B: its round-off scales with B
    with V.Context(p) as ctx:
        assert V.vlbm_init_fields_device(ctx.ptr, 0, Q.data_ptr()) == V.VLBM_OK
        del Q
        torch.cuda.empty_cache()
        V.vlbm_step(ctx.ptr, 4)
        V.vlbm_step(ctx.ptr, 4)
        idx = np.array([x + n * (y + n * z) for z, y, x in cells], dtype=np.int64)
        pops = ctx.populations(idx)  # the pre-collision populations: their sums are the moments
        assert ctx.sync() == V.VLBM_OK
    got = pops.reshape(len(cells), 9, 7).sum(2)
    for r, box in enumerate(boxes):
        ref = oracle.powell_run(box, gamma, [0.51] * 9, 1.0, steps)[:, w, w, w]
        err = np.abs(got[r] - ref) / scale
        assert err.max() < 1e-5, (cells[r], err)
