"""Pins of the resistive incompressible oracle (D3Q19 flow + 3 x D3Q7 B).

Closed forms: shear-wave decay exp(-nu k^2 t) with nu = (tau_f - 1/2)/3,
magnetic diffusion exp(-eta k^2 t) with eta = (tau_m - 1/2)/4 (Eq. 5 with
cs^2 = 1/3 and 1/4), the Guo force adding exactly F per cell per step, the
Poiseuille profile (Ha = 0) and the Hartmann profile, and an independent
NumPy restatement on a tiny channel.
"""
import math

import numpy as np
import pytest

from paper_2606_00641_gb300 import fields


def _uniform(shape, rho=1.0, m=(0, 0, 0), B=(0, 0, 0)):
    Q = np.zeros((7,) + tuple(shape))
    Q[0] = rho
    for a in range(3):
        Q[1 + a] = m[a]
        Q[4 + a] = B[a]
    return Q


def test_mass_exact_and_force_adds_F_per_cell(orc):
    shape = (6, 7, 8)
    rng = np.random.default_rng(3)
    Q = _uniform(shape, B=(0.01, 0.02, -0.01))
    Q[0] += 0.01 * rng.uniform(-1, 1, size=shape)
    Q[1:4] = 0.005 * rng.uniform(-1, 1, size=(3,) + shape)
    F = np.array([1e-5, -2e-6, 3e-6])
    n = 30
    out = orc.resistive_run(Q, 0.7, 0.8, F, (0, 0, 0), 0, n)
    N = np.prod(shape)
    assert abs(out[0].sum() - Q[0].sum()) < 1e-12 * Q[0].sum()
    dm = out[1:4].reshape(3, -1).sum(1) - Q[1:4].reshape(3, -1).sum(1)
    np.testing.assert_allclose(dm, n * N * F, rtol=1e-9, atol=1e-14)
    # total magnetic flux is conserved in periodic directions
    dB = out[4:7].reshape(3, -1).sum(1) - Q[4:7].reshape(3, -1).sum(1)
    assert np.abs(dB).max() < 1e-13


def test_shear_wave_decay_gives_viscosity(orc):
    ny = 32
    k = 2 * math.pi / ny
    tau_f = 0.8
    nu = (tau_f - 0.5) / 3.0
    Q = _uniform((1, ny, 1))
    y = np.arange(ny)
    amp = 1e-4
    Q[1, 0, :, 0] = amp * np.sin(k * y)
    n = 300
    out = orc.resistive_run(Q, tau_f, 0.9, (0, 0, 0), (0, 0, 0), 0, n)
    got = np.sum(out[1, 0, :, 0] * np.sin(k * y)) * 2 / ny
    # discrete-lattice decay factor per step for the diffusive mode
    rate = -math.log(got / amp) / n
    assert abs(rate / (nu * k * k) - 1) < 0.01


def test_magnetic_diffusion_gives_eta(orc):
    ny = 32
    k = 2 * math.pi / ny
    tau_m = 0.9
    eta = (tau_m - 0.5) / 4.0
    Q = _uniform((1, ny, 1))
    y = np.arange(ny)
    amp = 1e-3
    Q[4, 0, :, 0] = amp * np.sin(k * y)
    n = 300
    out = orc.resistive_run(Q, 0.7, tau_m, (0, 0, 0), (0, 0, 0), 0, n)
    got = np.sum(out[4, 0, :, 0] * np.sin(k * y)) * 2 / ny
    rate = -math.log(got / amp) / n
    assert abs(rate / (eta * k * k) - 1) < 0.01


def _channel_run(orc, Ha, ny=34, tau=1.0, steps=None):
    a = (ny - 2) / 2.0
    nu = (tau - 0.5) / 3.0
    eta = nu
    tau_m = 0.5 + 4.0 * eta
    B0 = Ha * math.sqrt(nu * eta) / a
    U_c = 0.02
    if Ha > 0:
        F = U_c * nu * Ha * math.tanh(Ha) / (a * a * (1 - 1 / math.cosh(Ha)))
    else:
        F = 2 * U_c * nu / (a * a)
    if steps is None:
        steps = int(5 * a * a / nu)
    Q = _uniform((1, ny, 1), B=(0, B0, 0))
    out = orc.resistive_run(Q, tau, tau_m, (F, 0, 0), (0, B0, 0), 1, steps)
    yc = np.arange(1, ny - 1) - (ny - 1) / 2.0
    u, b = out[1, 0, 1:ny - 1, 0], out[4, 0, 1:ny - 1, 0]
    return dict(u=u, b=b, yc=yc, a=a, nu=nu, eta=eta, B0=B0, F=F)


def test_poiseuille_profile(orc):
    r = _channel_run(orc, 0.0)
    u_ex, _ = fields.hartmann_profile(r["yc"], r["a"], r["F"], 1.0, r["nu"], r["eta"], 0.0)
    assert np.abs(r["u"] - u_ex).max() < 5e-3 * u_ex.max()
    assert np.abs(r["b"]).max() < 1e-14


def _hartmann_errors(r, Ha):
    u, b, yc, a = r["u"], r["b"], r["yc"], r["a"]
    # profile shape [1 - cosh(Ha y/a)/cosh Ha] does not depend on where the
    # magnetic wall sits (only the amplitude does, through the return current)
    shape = 1 - np.cosh(Ha * yc / a) / math.cosh(Ha)
    amp = (u @ shape) / (shape @ shape)
    shape_err = np.abs(u - amp * shape).max() / np.abs(u).max()
    bp = 0.5 * (b[2:] - b[:-2])
    # steady induction equation integrated once: eta b' + B0 u = const
    ind = r["eta"] * bp + r["B0"] * u[1:-1]
    ind_err = (ind.max() - ind.min()) / np.abs(ind).mean()
    # steady momentum equation: nu u'' + B0 b' + F = 0 holds exactly on the lattice
    upp = u[2:] - 2 * u[1:-1] + u[:-2]
    mom = np.abs(r["nu"] * upp + r["B0"] * bp + r["F"]).max() / r["F"]
    return shape_err, ind_err, mom


@pytest.mark.parametrize("Ha", [5.0, 10.0])
def test_hartmann_profile(orc, Ha):
    coarse = _hartmann_errors(_channel_run(orc, Ha, ny=34), Ha)
    fine = _hartmann_errors(_channel_run(orc, Ha, ny=66), Ha)
    assert coarse[2] < 1e-9 and fine[2] < 1e-9
    assert coarse[0] < 0.03 and coarse[1] < 0.06
    # the profile-shape error converges at second order, the induction balance
    # (limited by the node-located equilibrium wall of B) at least at first order
    assert fine[0] < coarse[0] / 3
    assert fine[1] < coarse[1] / 2
    r = _channel_run(orc, Ha, ny=34)
    b = r["b"]
    assert np.abs(b + b[::-1]).max() < 1e-10 * np.abs(b).max()


def test_c_oracle_matches_numpy_restatement_resistive(orc):
    from oracle import numpy_ref
    shape = (3, 6, 4)
    rng = np.random.default_rng(9)
    Q = _uniform(shape, B=(0.01, 0.03, 0.0))
    Q[0] += 0.02 * rng.uniform(-1, 1, size=shape)
    Q[1:4] = 0.01 * rng.uniform(-1, 1, size=(3,) + shape)
    Q[4:7] += 0.01 * rng.uniform(-1, 1, size=(3,) + shape)
    Q[1:4, :, 0, :] = 0
    Q[1:4, :, -1, :] = 0
    F = (2e-5, 1e-6, -1e-6)
    bw = (0.0, 0.03, 0.0)
    fa, ga = orc.resistive_init(Q, F)
    fb, gb = numpy_ref.resistive_init(Q, F)
    np.testing.assert_allclose(fa, fb, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(ga, gb, rtol=1e-14, atol=1e-16)
    for _ in range(25):
        fa, ga = orc.resistive_step(fa, ga, 0.62, 0.7, F, bw, 1)
        fb, gb = numpy_ref.resistive_step(fb, gb, 0.62, 0.7, F, bw, 1)
    Qa = orc.resistive_moments(fa, ga, F, bw, 1)
    Qb = numpy_ref.resistive_moments(fb, gb, F, bw, 1)
    np.testing.assert_allclose(Qa, Qb, rtol=1e-12, atol=1e-15)


def test_channel_update_is_symmetric_under_the_mirror_between_its_walls(orc):
    # y -> ny - 1 - y swaps the two walls; u turns as a vector (u_y flips) and B as a
    # pseudovector (B_x, B_z flip, B_y stays), which leaves the wall field (0, b, 0) and the
    # force along x unchanged, so the mirrored run is the run of the mirrored state
    shape = (3, 8, 5)
    rng = np.random.default_rng(21)
    Q = _uniform(shape, B=(0.01, 0.03, -0.02))
    Q[0] += 0.02 * rng.uniform(-1, 1, size=shape)
    Q[1:4] = 0.01 * rng.uniform(-1, 1, size=(3,) + shape)
    Q[4:7] += 0.01 * rng.uniform(-1, 1, size=(3,) + shape)
    Q[1:4, :, 0, :] = 0
    Q[1:4, :, -1, :] = 0
    F, bw = (2e-5, 0.0, 0.0), (0.0, 0.03, 0.0)

    def mirror(S):
        M = S[:, :, ::-1, :].copy()
        M[2] *= -1          # u_y
        M[4] *= -1          # B_x
        M[6] *= -1          # B_z
        return M

    a = mirror(orc.resistive_run(Q, 0.62, 0.7, F, bw, True, 9))
    b = orc.resistive_run(mirror(Q), 0.62, 0.7, F, bw, True, 9)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    assert np.abs(mirror(Q) - Q).max() > 1e-3   # the state itself is not symmetric


def test_channel_update_is_covariant_under_the_quarter_turn_about_y(orc):
    # (x, y, z) -> (z, y, -x) maps D3Q19 and D3Q7 onto themselves and keeps the walls; u, B,
    # the force and the wall field turn as vectors (v -> (v_z, v_y, -v_x)); square in x, z
    n, ny = 5, 8
    rng = np.random.default_rng(22)
    Q = _uniform((n, ny, n), B=(0.01, 0.03, -0.02))
    Q[0] += 0.02 * rng.uniform(-1, 1, size=(n, ny, n))
    Q[1:4] = 0.01 * rng.uniform(-1, 1, size=(3, n, ny, n))
    Q[4:7] += 0.01 * rng.uniform(-1, 1, size=(3, n, ny, n))
    Q[1:4, :, 0, :] = 0
    Q[1:4, :, -1, :] = 0
    Zi, Yi, Xi = np.meshgrid(np.arange(n), np.arange(ny), np.arange(n), indexing="ij")

    def turn(v):
        return np.array([v[2], v[1], -v[0]])

    def rotate(S):
        M = S[:, Xi, Yi, (-Zi) % n]      # the value at (x, y, z) lands at (z, y, -x)
        return np.concatenate([M[:1], turn(M[1:4]), turn(M[4:7])])

    F, bw = np.array([2e-5, 0.0, 1e-5]), np.array([0.01, 0.03, -0.02])
    a = rotate(orc.resistive_run(Q, 0.62, 0.7, F, bw, True, 9))
    b = orc.resistive_run(rotate(Q), 0.62, 0.7, turn(F), turn(bw), True, 9)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    assert np.abs(rotate(Q) - Q).max() > 1e-3
