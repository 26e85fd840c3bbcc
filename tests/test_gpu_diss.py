"""Dissipative MHD with locally evolved gradients (model VLBM_DISSIPATIVE) on the
GPU against the FP64 oracle (sec. 2.2.1 local moments evolution; sec. 2.3, the
full dissipative system: viscous stress, eta(j) resistivity, optional Powell
source; D2Q5, 20 lattices, 100 populations per cell; and the 3-D form on D3Q7,
26 lattices, 182 populations per cell).

Tolerances as for the ideal model: FP64 storage 1e-12, FP32 storage 1e-5,
relative L-infinity per field against max(the field's maximum, its reference
scale).  The reference scale of G (~ tau_M grad B) is tau_M max|B| and that of
W (~ tau_M grad u) is tau_M max|u|: G and W are sums of populations that carry
-B and -u, so their round-off scales with B and u, not with G and W.
"""
import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu

TAU8 = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]
TAU_G, TAU_M = 0.7, 2.0


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def diss_fields(shape, seed, tau_m=TAU_M):
    # the ideal recipe, G and W at tau_M times the centred gradients plus noise
    f0 = fields.ideal_fields(shape, seed, mach=1.0, beta=1.0, cfl=0.2)
    Q = f0.Q
    u = Q[1:4] / Q[0]
    rng = np.random.default_rng(seed)
    G = np.zeros((12,) + tuple(shape))
    for a in range(2):
        for b in range(3):
            ax = 1 - a  # array axis of x (a = 0) and y (a = 1)
            G[3 * a + b] = tau_m * 0.5 * (np.roll(Q[5 + b], -1, ax) - np.roll(Q[5 + b], 1, ax))
            G[6 + 3 * a + b] = tau_m * 0.5 * (np.roll(u[b], -1, ax) - np.roll(u[b], 1, ax))
    G += 0.1 * np.abs(G).max() * rng.normal(size=G.shape)
    return np.concatenate([Q, G]), f0.gamma


def field_scales(ref, tau_m=TAU_M):
    """Per-field reference scale: the field's maximum, and for vector and tensor
    components the maximum over the components (a component may vanish)."""
    n = ref.shape[0]
    m = np.abs(ref).reshape(n, -1).max(1)
    scale = m.copy()
    scale[1:4] = m[1:4].max()
    scale[5:8] = m[5:8].max()
    if n == 20:
        umax = np.abs(ref[1:4] / ref[0]).max()
        scale[8:14] = max(m[8:14].max(), tau_m * m[5:8].max())
        scale[14:20] = max(m[14:20].max(), tau_m * umax)
    return np.maximum(scale, 1e-300)


def field_errors(got, ref, tau_m=TAU_M):
    n = ref.shape[0]
    return np.abs(got - ref).reshape(n, -1).max(1) / field_scales(ref, tau_m)


def dissipation(powell, jc=0.05):
    return oracle.Dissipation(nu=0.02, eta0=0.03, j_c=jc, tau_m=TAU_M, powell=powell)


def make(V, shape, storage, dp, tau=TAU8, tau_g=TAU_G, gamma=5.0 / 3.0, **kw):
    return V.make_params(model=V.VLBM_DISSIPATIVE, shape=shape, storage=storage, gamma=gamma, tau=tau,
                         tau_g=tau_g, tau_m=dp.tau_m, nu=dp.nu, eta0=dp.eta0, j_c=dp.j_c, powell=dp.powell, **kw)


@pytest.mark.parametrize("shape", [(12, 130), (9, 33), (64, 64), (1, 40)])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("steps", [4, 5])
@pytest.mark.parametrize("powell", [False, True])
def test_dissipative_matches_oracle(V, shape, storage, tol, steps, powell):
    Q0, gamma = diss_fields(shape, 41)
    dp = dissipation(powell)
    with V.Context(make(V, shape, storage, dp, gamma=gamma)) as ctx:
        assert ctx.nvar == 20 and ctx.nslot == 100
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(steps)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    ref = oracle.diss_run(Q0, gamma, TAU8, dp, steps, tau_g=TAU_G)
    err = field_errors(got, ref)
    assert err.max() < tol, dict(zip(fields.DISSIPATIVE_FIELDS, err))


def test_dissipation_changes_the_result(V):
    # the comparison above is not one of two ideal runs: with nu = eta0 = 0 the GPU
    # result moves by far more than the tolerance
    shape = (16, 32)
    Q0, gamma = diss_fields(shape, 42)
    out = []
    for dp in (dissipation(False), oracle.Dissipation(tau_m=TAU_M)):
        with V.Context(make(V, shape, "f64", dp, gamma=gamma)) as ctx:
            assert ctx.init_fields(Q0) == V.VLBM_OK
            ctx.step(6)
            out.append(ctx.moments())
    assert field_errors(out[0][:8], out[1][:8]).max() > 1e-4


def test_dissipative_populations_at_odd_parity(V):
    shape = (6, 40)
    Q0, gamma = diss_fields(shape, 43)
    dp = dissipation(True)
    f = oracle.diss_init(Q0, gamma, dp)
    for _ in range(3):
        f = oracle.diss_step(f, gamma, TAU8, dp, tau_g=TAU_G)
    cells = np.array([0, 1, 39, 40, 41, 79, 120, 200, 239], dtype=np.int64)
    with V.Context(make(V, shape, "f64", dp, gamma=gamma)) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(3)
        got = ctx.populations(cells)
    ref = f.reshape(100, -1)[:, cells].T
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_dissipative_uniform_step_closed_form(V):
    # a uniform state does not stream: G and W lose 1/tau_M per step and, with the
    # Powell source, the MHD fields move by -(div B)(0, B, u.B, u) once per step
    Q0 = np.zeros(20)
    Q0[0], Q0[1:4], Q0[4], Q0[5:8] = 1.1, [0.05, -0.02, 0.01], 0.1, [0.1, -0.05, 0.04]
    Q0[8:] = 0.01 * np.arange(1, 13)
    shape = (3, 8)
    Q = np.broadcast_to(Q0[:, None, None], (20,) + shape).copy()
    tau_m = 2.5
    dp = oracle.Dissipation(nu=0.01, eta0=0.02, j_c=0.1, tau_m=tau_m, powell=True)
    with V.Context(make(V, shape, "f64", dp, tau=0.6, tau_g=0.7)) as ctx:
        assert ctx.init_fields(Q) == V.VLBM_OK
        ctx.step(1)
        one = ctx.moments()[:, 0, 0]
    divB = (Q0[8] + Q0[12]) / tau_m
    u = Q0[1:4] / Q0[0]
    expect = Q0.copy()
    expect[1:4] -= divB * Q0[5:8]
    expect[4] -= divB * (u @ Q0[5:8])
    expect[5:8] -= divB * u
    expect[8:] *= 1 - 1 / tau_m
    np.testing.assert_allclose(one, expect, rtol=1e-12, atol=1e-16)


# FP32 bound: half an FP32 ulp of the sums per step (37 steps x 2^-24 = 2.2e-6).
# The step's weights sum to one exactly in FP32 (w0 = 1 - 4 w1, omega w0 =
# omega - 4 omega w1); with rounded products instead (omega * w0) every cell
# moves by the same fraction each step, about two ulps per step here (measured
# 4.3e-6 after 37 steps), which this bound rejects.
@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 37 * 2.0 ** -24)])
def test_dissipative_conserves_the_mhd_sums(V, storage, tol):
    shape = (24, 50)
    Q0, gamma = diss_fields(shape, 44)
    dp = dissipation(False)
    with V.Context(make(V, shape, storage, dp, gamma=gamma)) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        s0 = ctx.conservation()
        assert s0.shape == (8,)
        ctx.step(37)  # odd: the sums read the AA layout of odd parity
        s1 = ctx.conservation()
        assert ctx.sync() == V.VLBM_OK
    scale = np.abs(Q0[:8]).reshape(8, -1).sum(1)
    assert (np.abs(s1 - s0) / scale).max() < tol


def test_dissipative_checkpoint_and_graphs(V):
    # 70 steps on a non-default stream (captured graphs of 32 steps) equal 70 single
    # steps, and a checkpoint restores the state bit for bit
    import torch
    shape = (20, 36)
    Q0, gamma = diss_fields(shape, 45)
    dp = dissipation(True)
    stream = torch.cuda.Stream()
    with V.Context(make(V, shape, "f32", dp, gamma=gamma, stream=stream.cuda_stream)) as a, \
            V.Context(make(V, shape, "f32", dp, gamma=gamma)) as b:
        assert a.init_fields(Q0) == V.VLBM_OK and b.init_fields(Q0) == V.VLBM_OK
        a.step(70)
        for _ in range(70):
            b.step(1)
        qa, qb = a.moments(), b.moments()
        np.testing.assert_array_equal(qa, qb)
        blob = a.save()
        a.step(3)
        a.load(blob)
        np.testing.assert_array_equal(a.moments(), qa)


def test_dissipative_api_contract(V):
    dp = dissipation(False)
    for shape, storage in (((4, 6, 16), "f16dev"), ((8, 16), "f16dev"), ((8, 16), "bf16dev")):
        with pytest.raises(V.VlbmError) as e:
            V.Context(make(V, shape, storage, dp))
        assert e.value.status == V.VLBM_ERR_UNSUPPORTED
    for kw, status in (({"tau_g": 0.5}, V.VLBM_ERR_UNSTABLE), ({"tau": 0.5}, V.VLBM_ERR_UNSTABLE)):
        with pytest.raises(V.VlbmError) as e:
            V.Context(make(V, (8, 16), "f32", dp, **kw))
        assert e.value.status == status
    bad = make(V, (8, 16), "f32", dp)
    bad.nu = -0.1
    with pytest.raises(V.VlbmError) as e:
        V.Context(bad)
    assert e.value.status == V.VLBM_ERR_ARG
    bad = make(V, (8, 16), "f32", dp)
    bad.tau_m = 0.4
    with pytest.raises(V.VlbmError):
        V.Context(bad)
    with V.Context(make(V, (8, 16), "f32", dp)) as ctx:
        with pytest.raises(V.VlbmError):
            ctx.set_boundary("x-", V.VLBM_BC_EQUILIBRIUM)
        with pytest.raises(V.VlbmError):
            ctx.set_solid(1 << 20)  # rejected before any use of the pointer
        # non-physical initial state
        Q, gamma = diss_fields((8, 16), 46)
        Q[0, 2, 3] = -1.0
        assert ctx.init_fields(Q) == V.VLBM_ERR_NONPHYSICAL
        Q, gamma = diss_fields((8, 16), 46)
        assert ctx.init_fields(Q) == V.VLBM_OK
        m_old = Q[1].copy()
        Q[1] *= 40.0  # |u| far beyond the lattice sound speed, gas pressure kept
        Q[4] += 0.5 * (Q[1] ** 2 - m_old ** 2) / Q[0]
        assert ctx.init_fields(Q) == V.VLBM_ERR_UNSTABLE


def test_low_mach_orszag_tang_full_size_sampled(V):
    """The benchmark run itself: 2048^2 low-Mach resistive Orszag-Tang set-up,
    FP32, the benchmark's stream and call sequence (4 + 20 steps), sampled at
    cells checked against the oracle on the periodic (2n+1)^2 box centred on each:
    on D2Q5 a cell after n steps depends only on cells within L1 distance n, and
    on that box no path of n steps wraps around."""
    import torch
    n = 2048
    setup = fields.low_mach_orszag_tang(n)
    dp = oracle.Dissipation(nu=setup.nu, eta0=setup.eta0, j_c=setup.j_c, tau_m=setup.tau_m, powell=True)
    stream = torch.cuda.Stream()
    p = V.make_params(model=V.VLBM_DISSIPATIVE, shape=(n, n), storage="f32", gamma=setup.gamma, tau=setup.tau,
                      tau_g=setup.tau_g, tau_m=setup.tau_m, nu=setup.nu, eta0=setup.eta0, j_c=setup.j_c,
                      powell=True, stream=stream.cuda_stream)
    Qd = torch.from_numpy(setup.Q).cuda()
    with V.Context(p) as ctx:
        assert V.vlbm_init_fields_device(ctx.ptr, 0, Qd.data_ptr()) == V.VLBM_OK
        del Qd
        V.vlbm_step(ctx.ptr, 4)
        V.vlbm_step(ctx.ptr, 20)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    steps = 24
    w = steps
    scale = field_scales(setup.Q, setup.tau_m)
    ys = [0, 1, 517, 1024, 1500, 2047, 2047, 300]
    xs = [0, 2047, 1023, 1024, 7, 2047, 0, 1999]
    for y, x in zip(ys, xs):
        iy = (np.arange(y - w, y + w + 1)) % n
        ix = (np.arange(x - w, x + w + 1)) % n
        box = np.ascontiguousarray(setup.Q[:, iy][:, :, ix])
        ref = oracle.diss_run(box, setup.gamma, setup.tau, dp, steps, tau_g=setup.tau_g)[:, w, w]
        err = np.abs(got[:, y, x] - ref) / scale
        assert err.max() < 1e-5, (y, x, dict(zip(fields.DISSIPATIVE_FIELDS, err)))



# ---------------------------------------------------------------------------
# 3-D: 26 lattices of D3Q7 (G_ab at 8 + 3a + b, W_ab at 17 + 3a + b)
# ---------------------------------------------------------------------------

def diss3_fields(shape, seed, tau_m=TAU_M):
    # the 3-D ideal recipe, G and W at tau_M times the centred gradients plus noise
    f0 = fields.ideal_fields(shape, seed, mach=1.0, beta=1.0, cfl=0.2)
    Q = f0.Q
    u = Q[1:4] / Q[0]
    rng = np.random.default_rng(seed)
    G = np.zeros((18,) + tuple(shape))
    for a in range(3):
        ax = 2 - a  # array axis of x, y, z
        for b in range(3):
            G[3 * a + b] = tau_m * 0.5 * (np.roll(Q[5 + b], -1, ax) - np.roll(Q[5 + b], 1, ax))
            G[9 + 3 * a + b] = tau_m * 0.5 * (np.roll(u[b], -1, ax) - np.roll(u[b], 1, ax))
    G += 0.1 * np.abs(G).max() * rng.normal(size=G.shape)
    return np.concatenate([Q, G]), f0.gamma


def field_scales3(ref, tau_m=TAU_M):
    n = ref.shape[0]
    m = np.abs(ref).reshape(n, -1).max(1)
    scale = m.copy()
    scale[1:4] = m[1:4].max()
    scale[5:8] = m[5:8].max()
    umax = np.abs(ref[1:4] / ref[0]).max()
    scale[8:17] = max(m[8:17].max(), tau_m * m[5:8].max())
    scale[17:26] = max(m[17:26].max(), tau_m * umax)
    return np.maximum(scale, 1e-300)


TAU26 = TAU8 + [TAU_G] * 18


@pytest.mark.parametrize("shape", [(5, 6, 16), (4, 7, 9), (1, 6, 130), (6, 1, 8)])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("steps", [4, 5])
@pytest.mark.parametrize("powell", [False, True])
def test_dissipative_3d_matches_oracle(V, shape, storage, tol, steps, powell):
    Q0, gamma = diss3_fields(shape, 47)
    dp = dissipation(powell)
    with V.Context(make(V, shape, storage, dp, gamma=gamma)) as ctx:
        assert ctx.nvar == 26 and ctx.nslot == 182
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(steps)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    ref = oracle.diss_run(Q0, gamma, TAU8, dp, steps, tau_g=TAU_G)
    err = np.abs(got - ref).reshape(26, -1).max(1) / field_scales3(ref)
    assert err.max() < tol, err


@pytest.mark.parametrize("steps", [3, 4])
def test_dissipative_3d_populations_match_oracle(V, steps):
    shape = (4, 5, 12)
    Q0, gamma = diss3_fields(shape, 48)
    dp = dissipation(True)
    cells = np.arange(np.prod(shape))
    with V.Context(make(V, shape, "f64", dp, gamma=gamma)) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(steps)
        got = ctx.populations(cells)
    f = oracle.diss_init(Q0, gamma, dp)
    for _ in range(steps):
        f = oracle.diss_step(f, gamma, TAU8, dp, tau_g=TAU_G)
    ref = f.reshape(26 * 7, -1).T
    scale = np.abs(ref).max(0) + np.abs(ref).max() * 1e-3
    assert (np.abs(got - ref) / scale).max() < 1e-12


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 21 * 2.0 ** -24)])
def test_dissipative_3d_conserves_the_mhd_sums(V, storage, tol):
    shape = (10, 12, 16)
    Q0, gamma = diss3_fields(shape, 49)
    dp = dissipation(False)
    with V.Context(make(V, shape, storage, dp, gamma=gamma)) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        s0 = ctx.conservation()
        ctx.step(21)
        s1 = ctx.conservation()
        assert ctx.sync() == V.VLBM_OK
    scale = np.abs(Q0[:8]).reshape(8, -1).sum(1)
    assert (np.abs(s1 - s0) / scale).max() < tol


def test_vortex_3d_full_size_sampled(V):
    """The 3-D benchmark workload at its size: 256^3 low-Mach resistive vortex,
    FP32, the benchmark's stream and first calls (4 + 4 steps), sampled at cells
    on the domain's corners, faces and interior, each checked against the oracle
    on the periodic (2n+1)^3 box centred on it (a cell after n D3Q7 steps depends
    only on cells within L1 distance n; no path of n steps wraps on that box)."""
    import torch
    n = 256
    setup = fields.low_mach_vortex_3d(n)
    dp = oracle.Dissipation(nu=setup.nu, eta0=setup.eta0, j_c=setup.j_c, tau_m=setup.tau_m, powell=True)
    stream = torch.cuda.Stream()
    p = V.make_params(model=V.VLBM_DISSIPATIVE, shape=(n, n, n), storage="f32", gamma=setup.gamma, tau=setup.tau,
                      tau_g=setup.tau_g, tau_m=setup.tau_m, nu=setup.nu, eta0=setup.eta0, j_c=setup.j_c,
                      powell=True, stream=stream.cuda_stream)
    with V.Context(p) as ctx:
        assert V.vlbm_init_fields(ctx.ptr, 0, setup.Q) == V.VLBM_OK
        V.vlbm_step(ctx.ptr, 4)
        V.vlbm_step(ctx.ptr, 4)
        cells = [(0, 0, 0), (255, 255, 255), (0, 128, 255), (131, 0, 7), (64, 200, 127), (255, 1, 128),
                 (17, 255, 0), (200, 99, 129)]
        Qall = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    steps = 8
    w = steps
    scale = field_scales3(setup.Q, setup.tau_m)
    for z, y, x in cells:
        iz, iy, ix = ((np.arange(c - w, c + w + 1)) % n for c in (z, y, x))
        box = np.ascontiguousarray(setup.Q[:, iz][:, :, iy][:, :, :, ix])
        ref = oracle.diss_run(box, setup.gamma, setup.tau, dp, steps, tau_g=setup.tau_g)[:, w, w, w]
        err = np.abs(Qall[:, z, y, x] - ref) / scale
        assert err.max() < 1e-5, ((z, y, x), dict(zip(fields.DISSIPATIVE3_FIELDS, err)))
