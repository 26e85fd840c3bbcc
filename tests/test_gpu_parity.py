"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative L-infinity per field, after a fixed step count):
  FP64 storage/arithmetic   1e-12
  FP32 storage/arithmetic   1e-5
normalised per field by max(max|Q_oracle|, s_k), s_k the field's reference
scale (velocity-like fields: rho_max * the largest lattice speed present, so
that fields that are small differences of O(1) populations are compared on
the scale their populations carry).
"""
import math

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


def ideal_scales(Q0):
    """Reference scale per ideal field: magnitudes of the initial state."""
    rho = np.abs(Q0[0]).max()
    mom = np.abs(Q0[1:4]).max()
    B = np.abs(Q0[5:8]).max()
    return np.array([rho, mom, mom, mom, np.abs(Q0[4]).max(), B, B, B])


def rel_err(got, ref, scales):
    nv = got.shape[0]
    g = got.reshape(nv, -1)
    r = ref.reshape(nv, -1)
    den = np.maximum(np.abs(r).max(1), scales) + 1e-300
    return np.abs(g - r).max(1) / den


def run_gpu(V, Q0, gamma, tau, steps, storage="f64", **kw):
    shape = Q0.shape[1:]
    p = V.make_params(shape=shape, storage=storage, gamma=gamma, tau=tau, **kw)
    with V.Context(p) as ctx:
        st = ctx.init_fields(Q0)
        assert st == V.VLBM_OK, V.status_string(st)
        ctx.step(steps)
        out = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    return out


# ---------------------------------------------------------------------------
# ideal MHD: D2Q5 / D3Q7, FP64 and FP32
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(24, 40), (33, 130), (9, 10, 12), (5, 7, 131)])
@pytest.mark.parametrize("steps", [0, 1, 2, 5, 40])
def test_ideal_fp64_matches_oracle(V, shape, steps):
    f0 = fields.ideal_fields(shape, 101, mach=1.2, beta=1.0, cfl=0.1 if len(shape) == 2 else 0.2)
    tau = np.array([0.51, 0.6, 0.7, 0.8, 0.55, 0.9, 1.0, 0.65])
    got = run_gpu(V, f0.Q, f0.gamma, tau, steps, "f64")
    ref = oracle.ideal_run(f0.Q, f0.gamma, tau, steps)
    assert rel_err(got, ref, ideal_scales(f0.Q)).max() < 1e-12


def test_config_128sq_fp64_200_steps(V):
    # 2-D ideal MHD, 128 x 128 periodic, 8 fields on D2Q5, FP64, gamma 5/3,
    # peak Mach 1, beta 10/3, CFL 0.1, tau 0.51, 200 steps, seed 1001
    f0 = fields.ideal_fields((128, 128), 1001)
    got = run_gpu(V, f0.Q, f0.gamma, 0.51, 200, "f64")
    ref = oracle.ideal_run(f0.Q, f0.gamma, 0.51, 200, nthreads=8)
    err = rel_err(got, ref, ideal_scales(f0.Q))
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("shape,steps,mach", [((64, 72), 50, 1.5), ((16, 20, 140), 50, 1.5),
                                              ((3, 130, 5), 31, 0.5)])
def test_ideal_fp32_matches_oracle(V, shape, steps, mach):
    f0 = fields.ideal_fields(shape, 202, mach=mach, beta=1.0, cfl=0.1 if len(shape) == 2 else 0.2)
    got = run_gpu(V, f0.Q, f0.gamma, 0.51, steps, "f32")
    ref = oracle.ideal_run(f0.Q, f0.gamma, 0.51, steps)
    err = rel_err(got, ref, ideal_scales(f0.Q))
    assert err.max() < 1e-5, err


@pytest.mark.parametrize("steps", [3, 4])
def test_populations_match_oracle_at_both_parities(V, steps):
    shape = (6, 9, 70)
    f0 = fields.ideal_fields(shape, 303, mach=1.0, cfl=0.2)
    tau = 0.7
    p = V.make_params(shape=shape, storage="f64", gamma=f0.gamma, tau=tau)
    rng = np.random.default_rng(5)
    cells = rng.choice(np.prod(shape), size=200, replace=False)
    with V.Context(p) as ctx:
        ctx.init_fields(f0.Q)
        ctx.step(steps)
        got = ctx.populations(cells)
    f = oracle.ideal_init(f0.Q, f0.gamma)
    for _ in range(steps):
        f = oracle.ideal_step(f, f0.gamma, tau)
    ref = f.reshape(8 * 7, -1)[:, cells].T
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_conservation_sums_fp64(V):
    f0 = fields.ideal_fields((48, 56), 404, mach=1.0)
    p = V.make_params(shape=(48, 56), storage="f64", gamma=f0.gamma, tau=0.51)
    with V.Context(p) as ctx:
        ctx.init_fields(f0.Q)
        s0 = ctx.conservation()
        again = ctx.conservation()
        ctx.step(200)
        s1 = ctx.conservation()
    exact0 = np.array([math.fsum(f0.Q[k].ravel()) for k in range(8)])
    scale = np.abs(f0.Q).reshape(8, -1).sum(1)
    assert (np.abs(s0 - exact0) / scale).max() < 1e-14
    assert np.array_equal(s0, again)  # fixed reduction order
    assert (np.abs(s1 - s0) / scale).max() < 1e-12


@pytest.mark.parametrize("shape", [(48, 56), (10, 12, 16)])
@pytest.mark.parametrize("batched", [False, True])
def test_conservation_sums_fp32_drift_below_half_an_ulp_per_step(V, shape, batched):
    # FP32 collisions use weights that sum to one exactly (D2Q5: w0 = 1 - 4 w1 and
    # omega w0 = omega - 4 omega w1; D3Q7's 1/4 and 1/8 are exact), so the domain
    # sums only take unbiased rounding.  With rounded products (omega * w0) every
    # cell moves by the same fraction each step: about 1-2 FP32 ulps per step on
    # D2Q5, which this bound rejects.
    if batched and len(shape) == 3:
        pytest.skip("batched domains are 2-D")
    steps = 101
    f0 = fields.ideal_fields(shape, 405, mach=1.0)
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.6)
    with V.Context([p, p] if batched else p, batch=batched) as ctx:
        for d in range(2 if batched else 1):
            assert ctx.init_fields(f0.Q, d) == V.VLBM_OK
        s0 = ctx.conservation(0)
        ctx.step(steps)
        s1 = ctx.conservation(0)
        assert ctx.sync() == V.VLBM_OK
    scale = np.abs(f0.Q).reshape(8, -1).sum(1)
    assert (np.abs(s1 - s0) / scale).max() < steps * 2.0 ** -24


def test_direct_source_injection(V):
    f0 = fields.ideal_fields((32, 32), 5, cfl=0.1)
    S = np.array([1e-4, 2e-5, -3e-5, 0.0, 5e-6, 1e-6, -2e-6, 0.0])
    n = 20
    p = V.make_params(shape=(32, 32), storage="f64", gamma=f0.gamma, tau=0.6, source=S)
    with V.Context(p) as ctx:
        ctx.init_fields(f0.Q)
        s0 = ctx.conservation()
        ctx.step(n)
        s1 = ctx.conservation()
    np.testing.assert_allclose(s1 - s0, n * 32 * 32 * S, atol=1e-12)
    ref = oracle.ideal_run(f0.Q, f0.gamma, 0.6, n, src=S)
    got = run_gpu(V, f0.Q, f0.gamma, 0.6, n, "f64", source=S)
    assert rel_err(got, ref, ideal_scales(f0.Q)).max() < 1e-12


def test_divB_invariant_with_tau_B_one(V):
    shape = (12, 12, 12)
    f0 = fields.ideal_fields(shape, 42, mach=1.5, beta=0.5, cfl=0.2)
    tau = np.array([0.7] * 5 + [1.0] * 3)
    got = run_gpu(V, f0.Q, f0.gamma, tau, 40, "f64")
    div = fields.centred_divergence(got[5], got[6], got[7])
    assert np.abs(div).max() < 1e-13 * np.abs(f0.Q[5:8]).max()


def test_uniform_state_fixed_point_fp32(V):
    shape = (8, 16, 160)
    Q = fields.uniform_ideal_state(shape, rho=1.2, u=(0.03, -0.02, 0.01), p=0.02, B=(0.05, 0.04, -0.03))
    got = run_gpu(V, Q, 5 / 3, 0.51, 33, "f32")
    assert (np.abs(got - Q).reshape(8, -1).max(1) / ideal_scales(Q)).max() < 1e-6


# ---------------------------------------------------------------------------
# health flags, stability check, checkpoints
# ---------------------------------------------------------------------------

def test_health_and_stability_statuses(V):
    shape = (16, 16)
    f0 = fields.ideal_fields(shape, 9)
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma)
    with V.Context(p) as ctx:
        bad = f0.Q.copy()
        bad[0, 3, 4] = np.nan
        assert ctx.init_fields(bad) == V.VLBM_ERR_NONPHYSICAL
        bad = f0.Q.copy()
        bad[1, 5, 6] = 0.0  # rho u set, energy kept: a cell with p <= 0 somewhere is nonphysical
        bad[4, 5, 6] = -1.0
        assert ctx.init_fields(bad) == V.VLBM_ERR_NONPHYSICAL
        bad = f0.Q.copy()
        ke = 0.5 * (bad[1] ** 2) / bad[0]
        bad[1] *= 40.0  # |u| far above the lattice sound speed, gas pressure unchanged
        bad[4] += 0.5 * (bad[1] ** 2) / bad[0] - ke
        assert ctx.init_fields(bad) == V.VLBM_ERR_UNSTABLE
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        assert ctx.step(4) == V.VLBM_OK and ctx.sync() == V.VLBM_OK
    # an energy sink drives p below zero during the run: the step kernel flags it
    S = np.zeros(8)
    S[4] = -0.01
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, source=S, check_every=1)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        ctx.step(3)
        assert ctx.sync() == V.VLBM_ERR_NONPHYSICAL
        assert ctx.step(1) == V.VLBM_ERR_NONPHYSICAL  # sticky
        assert ctx.init_fields(f0.Q) == V.VLBM_OK      # init clears it


def test_nonphysical_flag_rises_at_the_oracle_step(V):
    # an under-resolved Mach 1.5 field on a 3 x 130 x 5 grid: the oracle's gas
    # pressure first turns negative during step 7; the step kernel's health
    # flag must rise at that step and not before
    shape = (3, 130, 5)
    f0 = fields.ideal_fields(shape, 202, mach=1.5, beta=1.0, cfl=0.2)
    f = oracle.ideal_init(f0.Q, f0.gamma)
    first_bad = None
    for s in range(12):
        f = oracle.ideal_step(f, f0.gamma, 0.51)
        Q = oracle.ideal_moments(f)
        pmin = min(oracle.ideal_pressure(f0.gamma, Q[:, z, y, x])
                   for z in range(3) for y in range(130) for x in range(5))
        if pmin <= 0:
            first_bad = s + 1
            break
    assert first_bad is not None
    p = V.make_params(shape=shape, storage="f64", gamma=f0.gamma, tau=0.51)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        ctx.step(first_bad)  # these kernels inspect only the physical states 0 .. first_bad-1
        assert ctx.sync() == V.VLBM_OK
        ctx.step(1)
        assert ctx.sync() == V.VLBM_ERR_NONPHYSICAL


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16dev"])
def test_checkpoint_restart_is_bit_exact(V, storage):
    shape = (10, 12, 66)
    f0 = fields.ideal_fields(shape, 77, cfl=0.2)
    p = V.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=0.55,
                      q_ref=f0.Q.reshape(8, -1).mean(1))
    with V.Context(p) as ctx:
        ctx.init_fields(f0.Q)
        ctx.step(5)
        blob = ctx.save()
        ctx.step(6)
        a = ctx.moments()
        ctx.load(blob)
        assert ctx.step_count == 5
        ctx.step(6)
        b = ctx.moments()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# reduced-precision storage (shifted deviations): stated error, no exact pin
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(12, 16, 40), (6, 8, 64), (3, 5, 128)])
@pytest.mark.parametrize("storage,bound", [("f16dev", 2e-3), ("bf16dev", 2e-2)])
def test_deviation_storage_error_bound(V, storage, bound, shape):
    f0 = fields.ideal_fields(shape, 606, mach=1.0, beta=1.0, cfl=0.2)
    qref = f0.Q.reshape(8, -1).mean(1)
    dev = np.abs(f0.Q - qref.reshape(8, 1, 1, 1)).reshape(8, -1).max(1)
    qscale = np.maximum(dev, 1e-12 * np.abs(qref).max())
    got = run_gpu(V, f0.Q, f0.gamma, 0.51, 20, storage, q_ref=qref, q_scale=qscale)
    ref = oracle.ideal_run(f0.Q, f0.gamma, 0.51, 20)
    err = rel_err(got, ref, ideal_scales(f0.Q))
    assert err.max() < bound, err


# 3-D rows with nx % 8 == 0 load through the bulk-copy engine: one tile (128),
# two tiles with a partial edge tile (136), degenerate extents whose y / z
# neighbours are the cell itself (1, 1, 64) and (2, 1, 16); nx = 44 takes the
# per-thread loads
@pytest.mark.parametrize("storage", ["f16dev", "bf16dev"])
@pytest.mark.parametrize("shape", [(4, 4, 64), (4, 6, 36), (6, 40)])
def test_fp64_pressure_recovery_in_a_cold_magnetised_plasma(V, storage, shape):
    # A static plasma at beta = 5e-9: e_tot = p/(gamma - 1) + B^2/2 with p = 1e-10,
    # B = 0.2.  In FP32, e_tot - B^2/2 = -1.24e-9 (p is below the ulp of e_tot), so
    # a step that took p in FP32 would flag the state non-physical; cells with
    # p < p_theta e_tot recompute it in FP64 from the FP64 reference state and the
    # state stays put.  (4, 4, 64): bulk-copy kernel; the others: one cell per thread.
    gamma, B0, p0 = 5.0 / 3.0, 0.2, 1e-10
    Q0 = np.zeros((8,) + shape)
    Q0[0] = 1.0
    Q0[4] = p0 / (gamma - 1) + 0.5 * B0 * B0
    Q0[7] = B0
    qref = Q0.reshape(8, -1)[:, 0].copy()
    qscale = [1.0, 0.01, 0.01, 0.01, 1.0, 1.0, 1.0, 1.0]  # momentum populations carry +-p_tot / 2
    with V.Context(V.make_params(shape=shape, storage=storage, gamma=gamma, tau=0.6, q_ref=qref,
                                 q_scale=qscale)) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(7)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    np.testing.assert_array_equal(got, Q0)  # moments decoded in FP64: the state exactly
    p = (gamma - 1) * (got[4] - 0.5 * (got[1:4] ** 2).sum(0) / got[0] - 0.5 * (got[5:8] ** 2).sum(0))
    assert np.abs(p / p0 - 1).max() < 1e-6
    # without the recovery the FP32 pressure is negative and the state is refused
    with V.Context(V.make_params(shape=shape, storage=storage, gamma=gamma, tau=0.6, q_ref=qref,
                                 q_scale=qscale, p_theta=0.0)) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_ERR_NONPHYSICAL


# (48, 64, 128) and (24, 40, 200): several row tiles per persistent CTA of the
# bulk-copy kernel (every staging buffer reused), the latter with ragged tiles
@pytest.mark.parametrize("shape", [(5, 6, 128), (4, 6, 136), (1, 1, 64), (2, 1, 16), (3, 5, 44), (9, 192),
                                   (48, 64, 128), (24, 40, 200)])
@pytest.mark.parametrize("storage,ulp", [("f16dev", 2.0 ** -11), ("bf16dev", 2.0 ** -8)])
@pytest.mark.parametrize("parity", [0, 1])
def test_deviation_storage_one_step_sampled(V, shape, storage, ulp, parity):
    # one step of the 16-bit deviation forms from gathered populations equals
    # the oracle collision up to the storage rounding, at warp and row edges
    dim = len(shape)
    q = 5 if dim == 2 else 7
    f0 = fields.ideal_fields(shape, 707, mach=1.0, beta=1.0, cfl=0.1 if dim == 2 else 0.2)
    qref = f0.Q.reshape(8, -1).mean(1)
    qscale = np.abs(f0.Q - qref.reshape((8,) + (1,) * dim)).reshape(8, -1).max(1)
    qscale = np.where(qscale > 0, qscale, 1.0)  # a uniform field (degenerate extents): unit scale
    p = V.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=0.6, q_ref=qref, q_scale=qscale)
    N = int(np.prod(shape))
    nx = shape[-1]
    dirs = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)][:q]
    full = (1,) * (3 - dim) + tuple(shape)

    def upstream(cell, c):
        nz, ny, nx_ = full
        x, y, z = cell % nx_, (cell // nx_) % ny, cell // (nx_ * ny)
        return (x - c[0]) % nx_ + nx_ * (((y - c[1]) % ny) + ny * ((z - c[2]) % nz))

    rng = np.random.default_rng(parity)
    # every warp-edge lane (x0 = 0, 62, 64, 126 ...) and row ends, plus random cells
    edge_x = sorted(e for e in {0, 1, 62, 63, 64, 65, 126, 127, nx - 2, nx - 1} if e < nx)
    base = rng.choice(N // nx, size=min(6, N // nx), replace=False) * nx
    cells = np.unique(np.concatenate([b + np.array(edge_x) for b in base] +
                                     [rng.choice(N, size=min(40, N), replace=False)])).astype(np.int64)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        ctx.step(2 + parity)
        src = {int(x): [upstream(int(x), c) for c in dirs] for x in cells}
        uniq = np.array(sorted({u for v in src.values() for u in v}), dtype=np.int64)
        pre = dict(zip(uniq.tolist(), ctx.populations(uniq)))
        ctx.step(1)
        post = ctx.populations(cells)
        assert ctx.sync() == V.VLBM_OK
    w = np.array([1 / 3 if dim == 2 else 1 / 4] + [1 / 6 if dim == 2 else 1 / 8] * (q - 1))
    coll = {u: oracle.ideal_collide_cell(dim, f0.gamma, 0.6, pre[u].reshape(8, q)) for u in uniq.tolist()}
    for r, x in enumerate(cells.tolist()):
        exp = np.array([[coll[src[x][i]][k, i] for i in range(q)] for k in range(8)])
        g_exp = (exp - w[None, :] * qref[:, None]) / qscale[:, None]
        g_got = (post[r].reshape(8, q) - w[None, :] * qref[:, None]) / qscale[:, None]
        tol = ulp * np.abs(g_exp) + 2e-3 * ulp * 64 * np.abs(g_exp).max()
        assert (np.abs(g_got - g_exp) <= tol).all(), (x, np.abs(g_got - g_exp).max())


# ---------------------------------------------------------------------------
# resistive channel: D3Q19 + 3 x D3Q7, walls, Guo force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("walls", [True, False])
def test_resistive_matches_oracle(V, walls):
    shape = (3, 10, 140)
    setup = fields.hartmann_setup(shape, 2002, Ha=10.0, U_c=0.05, Re=10.0)
    Q0 = setup.Q.copy()
    rng = np.random.default_rng(1)
    Q0[4:7] += 0.01 * rng.uniform(-1, 1, size=(3,) + shape)
    steps = 40
    p = V.make_params(model=V.VLBM_RESISTIVE, shape=shape, storage="f32",
                      tau=[setup.tau_f, setup.tau_m, setup.tau_m, setup.tau_m],
                      force=setup.force, b_wall=setup.b_wall, walls_y=walls)
    with V.Context(p) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(steps)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    ref = oracle.resistive_run(Q0, setup.tau_f, setup.tau_m, setup.force, setup.b_wall, walls, steps)
    cs = math.sqrt(1 / 3)
    scales = np.array([1.0, cs, cs, cs] + [np.abs(Q0[4:7]).max()] * 3)
    err = rel_err(got, ref, scales)
    assert err.max() < 1e-5, err


# ---------------------------------------------------------------------------
# batched 2-D domains in one launch
# ---------------------------------------------------------------------------

def test_batched_domains_match_oracle_for_every_tile_shape(V):
    specs = [((32, 32), 1.4, 0.8), ((48, 64), 5 / 3, 1.5), ((16, 80), 1.5, 2.5), ((64, 64), 1.6, 1.0)]
    params, inits = [], []
    for d, (shape, gamma, mach) in enumerate(specs):
        f0 = fields.ideal_fields(shape, 4004 + d, gamma=gamma, mach=mach, cfl=0.1)
        inits.append(f0)
        params.append(V.make_params(shape=shape, storage="f32", gamma=gamma, tau=0.51 + 0.02 * d))
    steps = 20
    refs = [oracle.ideal_run(f0.Q, f0.gamma, 0.51 + 0.02 * d, steps) for d, f0 in enumerate(inits)]
    results = []
    with V.Context(params, batch=True) as ctx:
        assert ctx.tile_shapes() >= 4
        for shape_id in range(ctx.tile_shapes()):
            ctx.set_tile_shape(shape_id)
            for d, f0 in enumerate(inits):
                assert ctx.init_fields(f0.Q, d) == V.VLBM_OK
            ctx.step(steps)
            outs = [ctx.moments(d) for d in range(len(specs))]
            assert ctx.sync() == V.VLBM_OK
            for d in range(len(specs)):
                err = rel_err(outs[d], refs[d], ideal_scales(inits[d].Q))
                assert err.max() < 1e-5, (shape_id, d, err)
            results.append(outs)
        # the tile shape changes only the schedule, not the arithmetic
        for outs in results[1:]:
            for d in range(len(specs)):
                assert np.abs(outs[d] - results[0][d]).max() <= 1e-6 * np.abs(results[0][d]).max()
        choice = ctx.autotune(4)
        assert 0 <= choice < ctx.tile_shapes()
