"""Pins of the oracle's homogenised solids (HLBM, sec. 2.4 "Homogenization").

The porosity d blends the cell's velocity and field with the solid's,
u_hat = d u + (1 - d) uB and B_hat = d B + (1 - d) BB, and the equilibrium is
taken at the blended state (rho and gas pressure kept).  Checked against: the
porosity's closed form, the pinned ideal scheme (d = 1), closed-form
relaxation of a uniform solid cell, exact mass conservation, and a
force-driven channel whose no-slip planes sit at the d = 1/2 level sets.
"""
import numpy as np
import pytest

import oracle
from oracle import numpy_ref as R
from paper_2606_00641_gb300 import fields

GAMMA = 5.0 / 3.0


def test_porosity_of_the_signed_distance():
    # 0 in the solid, 1 in the fluid, linear across eps_h, 1/2 on the surface
    eps = 1.5
    phi = np.array([-3.0, -0.75, -0.5, 0.0, 0.3, 0.75, 3.0])
    expect = [0.0, 0.0, 1.0 / 6.0, 0.5, 0.7, 1.0, 1.0]
    np.testing.assert_allclose(oracle.hlbm_porosity(phi, eps), expect, rtol=0, atol=1e-15)


def _solid(shape, d, uB=(0.0, 0.0, 0.0), BB=(0.0, 0.0, 0.0)):
    s = np.zeros((7,) + tuple(shape))
    s[0] = d
    for a in range(3):
        s[1 + a] = uB[a]
        s[4 + a] = BB[a]
    return s


@pytest.mark.parametrize("d", [0.0, 0.25, 0.6, 1.0])
def test_blended_state_of_one_cell(d):
    # sec. 2.4, "Homogenization": the blend moves u and B affinely from the solid's (d = 0) to
    # the cell's own (d = 1) and keeps the cell's density and gas pressure; d = 1 is the cell
    Q = np.array([1.3, 0.13, -0.26, 0.065, 2.0, 0.3, -0.1, 0.2])
    uB, BB = np.array([0.02, 0.05, -0.01]), np.array([-0.2, 0.1, 0.4])
    Qh = oracle.hlbm_target(GAMMA, Q, d, uB, BB)
    u = Q[1:4] / Q[0]
    assert Qh[0] == Q[0]
    np.testing.assert_allclose(Qh[1:4] / Qh[0], d * u + (1 - d) * uB, rtol=0, atol=1e-15)
    np.testing.assert_allclose(Qh[5:8], d * Q[5:8] + (1 - d) * BB, rtol=0, atol=1e-15)
    assert abs(oracle.ideal_pressure(GAMMA, Qh) / oracle.ideal_pressure(GAMMA, Q) - 1) < 1e-14
    if d == 1.0:
        np.testing.assert_allclose(Qh, Q, rtol=1e-15, atol=1e-16)
    if d == 0.0:
        np.testing.assert_array_equal(Qh[5:8], BB)


@pytest.mark.parametrize("shape", [(12, 10), (4, 6, 5)])
def test_fluid_everywhere_is_the_ideal_scheme(shape):
    # d = 1: the blend returns the cell's own u and B; the rebuilt energy equals e
    f0 = fields.ideal_fields(shape, 41, mach=1.0, beta=1.0, cfl=0.2)
    solid = _solid(shape, 1.0, (0.3, -0.1, 0.2), (0.5, 0.5, -0.5))
    got = oracle.hlbm_run(f0.Q, f0.gamma, 0.6, solid, 10)
    ref = oracle.ideal_run(f0.Q, f0.gamma, 0.6, 10)
    scale = np.abs(f0.Q).reshape(8, -1).max(1)
    assert (np.abs(got - ref).reshape(8, -1).max(1) / scale).max() < 1e-13


def test_uniform_solid_cell_relaxes_to_the_solid_state():
    # d = 0 on a uniform state: streaming is the identity, so each step is
    # Q <- Q + omega (Q_hat - Q) with Q_hat carrying uB and BB: the momentum and
    # field approach rho uB and BB as (1 - omega)^n, the density does not move
    shape = (3, 4, 5)
    Q0 = np.array([1.2, 0.12, -0.06, 0.03, 1.0, 0.2, -0.1, 0.05])
    Q = np.broadcast_to(Q0.reshape(8, 1, 1, 1), (8,) + shape).copy()
    uB, BB = np.array([0.05, 0.02, -0.04]), np.array([-0.1, 0.15, 0.0])
    tau = np.array([0.6, 0.8, 0.8, 0.8, 0.7, 0.9, 0.9, 0.9])
    n = 6
    out = oracle.hlbm_run(Q, GAMMA, tau, _solid(shape, 0.0, uB, BB), n)[:, 0, 0, 0]
    om_m, om_b = 1 / tau[1], 1 / tau[5]
    np.testing.assert_allclose(out[0], Q0[0], rtol=1e-15)
    np.testing.assert_allclose(out[1:4], Q0[0] * uB + (1 - om_m) ** n * (Q0[1:4] - Q0[0] * uB), rtol=1e-12)
    np.testing.assert_allclose(out[5:8], BB + (1 - om_b) ** n * (Q0[5:8] - BB), rtol=1e-12, atol=1e-16)


def _gas_pressure(Q):
    return (GAMMA - 1) * (Q[4] - 0.5 * (Q[1:4] ** 2).sum(0) / Q[0] - 0.5 * (Q[5:8] ** 2).sum(0))


@pytest.mark.parametrize("tau", [0.6, 1.5])
def test_uniform_cell_pressure_follows_the_relaxation_of_the_blend(tau):
    # The blended state keeps rho and p, so with one omega on every lattice a uniform
    # cell moves to Q + omega (Q_hat - Q).  For weights (1 - omega, omega) the convex
    # identity a|x|^2 + b|y|^2 - |a x + b y|^2 = a b |x - y|^2 gives the gas pressure
    # after one step as p + (gamma - 1) omega (1 - omega) (rho |u_hat - u|^2 + |B_hat - B|^2) / 2:
    # heating for omega < 1, a drain for omega > 1.  With d = 0 the target is fixed, the
    # contrast decays as (1 - omega)^n, and the n-step sum is geometric.
    shape = (2, 3, 4)
    Q0 = np.array([1.2, 0.12, -0.06, 0.03, 1.0, 0.2, -0.1, 0.05])
    Q = np.broadcast_to(Q0.reshape(8, 1, 1, 1), (8,) + shape).copy()
    uB, BB = np.array([0.05, 0.02, -0.04]), np.array([-0.1, 0.15, 0.0])
    om = 1.0 / tau
    rho, u, B = Q0[0], Q0[1:4] / Q0[0], Q0[5:8]
    p0 = _gas_pressure(Q0)
    d = 0.25
    contrast = rho * (((1 - d) * (uB - u)) ** 2).sum() + (((1 - d) * (BB - B)) ** 2).sum()
    one = oracle.hlbm_run(Q, GAMMA, tau, _solid(shape, d, uB, BB), 1)[:, 0, 0, 0]
    np.testing.assert_allclose(_gas_pressure(one), p0 + (GAMMA - 1) * om * (1 - om) * 0.5 * contrast,
                               rtol=1e-12)
    n = 9
    k0 = rho * ((uB - u) ** 2).sum() + ((BB - B) ** 2).sum()
    many = oracle.hlbm_run(Q, GAMMA, tau, _solid(shape, 0.0, uB, BB), n)[:, 0, 0, 0]
    expect = p0 - 0.5 * (GAMMA - 1) * (om - 1) / (2 - om) * (1 - (1 - om) ** (2 * n)) * k0
    np.testing.assert_allclose(_gas_pressure(many), expect, rtol=1e-12)


def test_mass_is_conserved_exactly():
    shape = (10, 12)
    f0 = fields.ideal_fields(shape, 43, mach=1.0, beta=1.0, cfl=0.2)
    y, x = np.mgrid[0:10, 0:12]
    phi = np.hypot(x - 6.0, y - 5.0) - 3.0
    solid = _solid(shape, oracle.hlbm_porosity(phi, 1.0), (0.01, -0.02, 0.0), (0.05, 0.0, 0.02))
    f = oracle.ideal_init(f0.Q, f0.gamma)
    m0 = f.sum(axis=1)[0].sum()
    for _ in range(12):
        f = oracle.hlbm_step(f, f0.gamma, 0.6, solid)
    assert abs(f.sum(axis=1)[0].sum() - m0) <= 1e-13 * m0


def test_channel_between_homogenised_walls_is_parabolic_with_walls_at_d_half():
    # a uniform force F along x drives gas at rest between two solid bands (uB = 0);
    # d comes from the signed distance to the planes y = y_lo, y_hi (eps_h = 1):
    # the steady x-velocity is the Poiseuille parabola F/(2 nu)(a^2 - (y - y_c)^2)
    # whose zeros sit on the d = 1/2 level sets (the paper's wall position).  The
    # momentum diffuses with nu = (tau - 1/2) c_s^2 at low Mach (D2Q5: c_s^2 = 1/3)
    ny, nx = 40, 4
    y_lo, y_hi = 6.3, 33.7  # walls between cells: an off-grid surface
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    phi = np.minimum(y - y_lo, y_hi - y)
    d = oracle.hlbm_porosity(phi, 1.0)
    solid = _solid((ny, nx), d)
    Q = np.zeros((8, ny, nx))
    Q[0] = 1.0
    Q[4] = 0.1 / (GAMMA - 1.0)  # p = 0.1 (sound speed 0.41 < c_s), at rest, no field
    F = 2e-6
    src = np.array([0.0, F, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    tau = 0.9
    out = oracle.hlbm_run(Q, GAMMA, tau, solid, 4000, src=src)
    ux = (out[1] / out[0])[:, 0]
    nu = (tau - 0.5) / 3.0
    a, yc = 0.5 * (y_hi - y_lo), 0.5 * (y_hi + y_lo)
    yy = np.arange(ny, dtype=float)
    inside = np.abs(yy - yc) < a - 2.0
    expect = F / (2 * nu) * (a * a - (yy - yc) ** 2)
    err = np.abs(ux[inside] - expect[inside]).max() / expect.max()
    assert err < 0.05, err
    # the fitted parabola's zeros are the d = 1/2 planes to within half a cell
    c2, c1, c0 = np.polyfit(yy[inside], ux[inside], 2)
    roots = np.sort(np.roots([c2, c1, c0]).real)
    assert abs(roots[0] - y_lo) < 0.5 and abs(roots[1] - y_hi) < 0.5, roots


@pytest.mark.parametrize("shape", [(12, 10), (4, 6, 5)])
def test_oracle_matches_numpy_restatement(shape):
    f0 = fields.ideal_fields(shape, 45, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(3)
    solid = np.concatenate([rng.random((1,) + shape), 0.05 * rng.normal(size=(6,) + shape)])
    tau = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]
    a = oracle.hlbm_run(f0.Q, f0.gamma, tau, solid, 15)
    b = R.hlbm_run(f0.Q, f0.gamma, tau, solid, 15)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_update_is_covariant_under_the_rotations_of_the_lattice(dim):
    # as for the ideal scheme, with the solid turned too: the porosity d moves with the
    # cells, the solid velocity u^B and field B^B turn as vectors
    from test_oracle_pins import _rotate_ideal

    def rotate_solid(S):
        # d and the u^B, B^B vectors in the ideal state's slots 0, 1-3 and 5-7
        eight = np.concatenate([S[:4], np.zeros((1,) + S.shape[1:]), S[4:7]])
        return np.delete(_rotate_ideal(eight), 4, axis=0)

    shape = (10, 10) if dim == 2 else (4, 5, 6)
    f0 = fields.ideal_fields(shape, 555, mach=0.5, beta=2.0, cfl=0.2)
    rng = np.random.default_rng(555)
    solid = np.concatenate([rng.uniform(0, 1, size=(1,) + shape),
                            0.02 * rng.normal(size=(3,) + shape), 0.05 * rng.normal(size=(3,) + shape)])
    tau = [0.6, 0.55, 0.55, 0.55, 0.7, 0.65, 0.65, 0.65]
    a = _rotate_ideal(oracle.hlbm_run(f0.Q, GAMMA, tau, solid, 7))
    b = oracle.hlbm_run(_rotate_ideal(f0.Q), GAMMA, tau, rotate_solid(solid), 7)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
