"""Pins of the oracle's dissipative MHD with locally evolved gradients
(sec. 2.2.1 "Local Moments Evolution", sec. 2.3 "Evolution of the MHD equation
system", the full flux of the dissipative system), on the D2Q5 lattice.

The state carries G ~ tau_M grad B and W ~ tau_M grad u as lattices (flux
G u - I B, W u - I u, source -G/tau_M, -W/tau_M); the fluxes add the viscous
stress rho nu (grad u + grad u^T), eta(j) j x B and -eta grad B with
eta = eta0 (1 + |j|^2 / j_c^2).  Checked against: the pinned ideal scheme
(no dissipation), the quasi-steady balance G -> tau_M grad B, the decay rates
of shear and magnetic-diffusion modes (nu k^2, eta0 k^2 plus the lattice's
(tau - 1/2) cs^2 k^2), the Fourier projection of the current-dependent
resistivity, exact conservation, the local viscous and ohmic heating, a
closed-form uniform step with the Powell source, and the NumPy restatement.
"""
import numpy as np
import pytest

import oracle
from oracle import numpy_ref as R
from paper_2606_00641_gb300 import fields

GAMMA = 5.0 / 3.0
N = 64
K = 2 * np.pi / N
X = np.arange(N)
TAU_M = 2.0
TAU = 0.55
CS2 = 1.0 / 3.0


def _rest(ny=4, p=0.02):
    # gas at rest, c = 0.18 (below the D2Q5 lattice speed 0.577)
    Q = np.zeros((20, ny, N))
    Q[0] = 1.0
    Q[4] = p / (GAMMA - 1)
    return Q


def _amp(field):
    return 2 * np.mean(field[0] * np.sin(K * X))


def _shear(U):
    Q = _rest()
    Q[2] = U * np.sin(K * X)
    Q[4] += 0.5 * Q[2] ** 2
    Q[14 + 1] = TAU_M * U * K * np.cos(K * X)  # W_xy at its balance
    return Q


def _sheet(b):
    Q = _rest()
    Q[6] = b * np.sin(K * X)
    Q[4] += 0.5 * Q[6] ** 2
    Q[8 + 1] = TAU_M * b * K * np.cos(K * X)  # G_xy at its balance
    return Q


def _rate(Q, dp, t0, t1, field):
    a0 = _amp(oracle.diss_run(Q, GAMMA, TAU, dp, t0, tau_g=0.55)[field])
    a1 = _amp(oracle.diss_run(Q, GAMMA, TAU, dp, t1, tau_g=0.55)[field])
    return np.log(a0 / a1) / (t1 - t0), np.sqrt(a0 * a1)


@pytest.mark.parametrize("shape", [(12, 16), (8, 10)])
def test_without_dissipation_the_mhd_fields_follow_the_ideal_scheme(shape):
    # nu = eta0 = 0 and no Powell source: the gradient lattices evolve but feed nothing back
    f0 = fields.ideal_fields(shape, 71, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(3)
    Q = np.concatenate([f0.Q, 0.01 * rng.normal(size=(12,) + shape)])
    tau8 = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]
    got = oracle.diss_run(Q, f0.gamma, tau8, oracle.Dissipation(tau_m=1.5), 15, tau_g=0.7)
    ref = oracle.ideal_run(f0.Q, f0.gamma, tau8, 15)
    scale = np.abs(f0.Q).reshape(8, -1).max(1)
    assert (np.abs(got[:8] - ref).reshape(8, -1).max(1) / scale).max() < 1e-13


def test_gradient_lattices_relax_to_tau_m_times_the_gradients():
    # sec. 2.2.1: in the quasi-steady balance G = tau_M grad B (and W = tau_M grad u),
    # reached from G = W = 0 within a few tau_M
    Q = _rest()
    b, U = 1e-3, 1e-3
    Q[6] = b * np.sin(K * X)
    Q[3] = U * np.sin(K * X)  # u_z(x): a shear that does not move B_y
    Q[4] += 0.5 * Q[6] ** 2 + 0.5 * Q[3] ** 2
    out = oracle.diss_run(Q, GAMMA, TAU, oracle.Dissipation(tau_m=TAU_M), 20, tau_g=0.55)
    expect_g = TAU_M * b * K * np.cos(K * X)
    expect_w = TAU_M * U * K * np.cos(K * X)
    assert np.abs(out[8 + 1][0] - expect_g).max() < 0.02 * np.abs(expect_g).max()   # G_xy
    assert np.abs(out[14 + 2][0] - expect_w).max() < 0.02 * np.abs(expect_w).max()  # W_xz
    # no gradient along y: those components stay zero
    assert np.abs(out[8 + 3:8 + 6]).max() < 1e-15 and np.abs(out[14 + 3:14 + 6]).max() < 1e-15


@pytest.mark.parametrize("nu", [0.0, 0.01])
def test_shear_wave_decays_at_nu_plus_the_lattice_diffusion(nu):
    # u_y = U sin(kx): momentum diffuses at nu k^2 through the viscous stress, plus the
    # first-order equilibrium's (tau - 1/2) cs^2 k^2 (no characteristic speed: a = 0)
    rate, _ = _rate(_shear(1e-3), oracle.Dissipation(nu=nu, tau_m=TAU_M), 20, 200, 2)
    expect = (nu + (TAU - 0.5) * CS2) * K * K
    assert abs(rate / expect - 1) < 0.01, (rate, expect)


@pytest.mark.parametrize("eta0", [0.0, 0.01])
def test_magnetic_sheet_diffuses_at_eta_plus_the_lattice_diffusion(eta0):
    rate, _ = _rate(_sheet(1e-3), oracle.Dissipation(eta0=eta0, tau_m=TAU_M), 20, 200, 6)
    expect = (eta0 + (TAU - 0.5) * CS2) * K * K
    assert abs(rate / expect - 1) < 0.005, (rate, expect)


def test_current_dependent_resistivity_projects_onto_the_mode():
    # eta = eta0 (1 + (j/j_c)^2) with j = a k cos(kx): the flux -eta dB/dx projected on
    # cos(kx) gives eta0 (1 + 3/4 (a k / j_c)^2), so the mode decays faster than with a
    # constant eta0 by eta0 3/4 (a k / j_c)^2 k^2 at its current amplitude a
    b = 1e-3
    jc = b * K
    base, _ = _rate(_sheet(b), oracle.Dissipation(eta0=0.01, tau_m=TAU_M), 20, 40, 6)
    rate, a = _rate(_sheet(b), oracle.Dissipation(eta0=0.01, j_c=jc, tau_m=TAU_M), 20, 40, 6)
    expect = 0.01 * 0.75 * (a * K / jc) ** 2 * K * K
    assert abs((rate - base) / expect - 1) < 0.03, (rate - base, expect)


def test_conserved_fields_are_conserved_exactly():
    shape = (10, 12)
    f0 = fields.ideal_fields(shape, 72, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(4)
    Q = np.concatenate([f0.Q, 0.01 * rng.normal(size=(12,) + shape)])
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=0.05, tau_m=1.5)
    out = oracle.diss_run(Q, f0.gamma, 0.6, dp, 20, tau_g=0.7)
    s0 = Q[:8].reshape(8, -1).sum(1)
    s1 = out[:8].reshape(8, -1).sum(1)
    scale = np.abs(Q[:8]).reshape(8, -1).sum(1)
    assert (np.abs(s1 - s0) / scale).max() < 1e-13


@pytest.mark.parametrize("case", ["viscous", "ohmic"])
def test_heat_appears_where_the_dissipation_is(case):
    # Total energy is a conserved flux, so a wrong sign of u.tau or eta j x B in the
    # energy flux would still conserve it; locally the internal energy must rise as
    # mu (du_y/dx)^2 or eta j^2, i.e. like cos^2(kx), and gain what the mode loses
    if case == "viscous":
        Q, dp, field = _shear(2e-2), oracle.Dissipation(nu=0.05, tau_m=TAU_M), 2
    else:
        Q, dp, field = _sheet(2e-2), oracle.Dissipation(eta0=0.05, tau_m=TAU_M), 6

    def internal(S):
        return S[4] - 0.5 * (S[1:4] ** 2).sum(0) / S[0] - 0.5 * (S[5:8] ** 2).sum(0)

    out = oracle.diss_run(Q, GAMMA, TAU, dp, 30, tau_g=0.55)
    heat = (internal(out) - internal(Q))[0]
    c2 = np.cos(K * X) ** 2 - 0.5
    h = heat - heat.mean()
    assert np.dot(h, c2) / np.linalg.norm(h) / np.linalg.norm(c2) > 0.999
    lost = 0.5 * (Q[field] ** 2 - out[field] ** 2 / (out[0] if field == 2 else 1.0))[0]
    assert abs(heat.sum() / lost.sum() - 1) < 0.05


def test_uniform_step_with_the_powell_source_and_relaxing_gradients():
    # a uniform state does not stream; one step adds the source once:
    # G, W -> (1 - 1/tau_M) G, W and, with div B = (G_xx + G_yy) / tau_M, the
    # Powell terms -(div B)(0, B, u.B, u) on the MHD fields
    Q0 = np.zeros(20)
    Q0[0], Q0[1:4], Q0[4], Q0[5:8] = 1.1, [0.05, -0.02, 0.01], 0.1, [0.1, -0.05, 0.04]
    Q0[8:] = 0.01 * np.arange(1, 13)
    grid = np.broadcast_to(Q0[:, None, None], (20, 3, 4)).copy()
    tau_m = 2.5
    dp = oracle.Dissipation(nu=0.01, eta0=0.02, j_c=0.1, tau_m=tau_m, powell=True)
    one = oracle.diss_run(grid, GAMMA, 0.6, dp, 1, tau_g=0.7)[:, 0, 0]
    divB = (Q0[8] + Q0[12]) / tau_m
    u = Q0[1:4] / Q0[0]
    expect = Q0.copy()
    expect[1:4] -= divB * Q0[5:8]
    expect[4] -= divB * (u @ Q0[5:8])
    expect[5:8] -= divB * u
    expect[8:] *= 1 - 1 / tau_m
    np.testing.assert_allclose(one, expect, rtol=1e-12, atol=1e-16)


def test_low_mach_orszag_tang_set_up_carries_the_paper_parameters():
    # the generator's unit conversion against the numbers the paper prints (golden file):
    # Re = U L / nu with the peak speed component U and the box side L, eta0 = nu, j_c, the
    # 5 % stabilisation and tau_M, all recovered from the lattice values
    import math
    import os
    gold = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "low_mach_orszag_tang.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = (t.strip() for t in line.split("="))
                gold[k] = float(v)
    n = int(gold["finest_n"])
    s = fields.low_mach_orszag_tang(n)
    scale = s.dt / s.dx                      # lattice velocity per physical velocity
    nu_phys = s.nu * s.dx * s.dx / s.dt      # lattice to physical diffusivity
    assert abs(nu_phys / gold["nu"] - 1) < 1e-12
    assert abs(gold["u_peak_component"] * 2 * math.pi / nu_phys / gold["reynolds"] - 1) < 1e-12
    assert s.eta0 == s.nu
    assert abs(s.j_c / (scale * s.dx) / gold["j_c"] - 1) < 1e-12
    assert abs((s.tau - 0.5) * CS2 / s.nu / gold["stabilisation"] - 1) < 1e-12
    assert abs(s.tau_m * s.dt / gold["tau_m"] - 1) < 1e-12
    u = s.Q[1:3] / s.Q[0]
    assert abs(np.abs(u).max() / scale / gold["u_peak_component"] - 1) < 1e-6
    assert abs(np.abs(s.Q[5:7]).max() / scale / gold["B_peak_component"] - 1) < 1e-6
    # G and W start at tau_M times the field gradients (centred differences agree to O(dx^2))
    dBy_dx = 0.5 * (np.roll(s.Q[6], -1, 1) - np.roll(s.Q[6], 1, 1))
    assert np.abs(s.Q[8 + 1] - s.tau_m * dBy_dx).max() < 1e-5 * np.abs(s.Q[8 + 1]).max()


@pytest.mark.parametrize("powell", [False, True])
def test_oracle_matches_numpy_restatement(powell):
    shape = (10, 12)
    f0 = fields.ideal_fields(shape, 5, mach=0.8, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(0)
    Q = np.concatenate([f0.Q, 0.01 * rng.normal(size=(12,) + shape)])
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=0.05, tau_m=2.0, powell=powell)
    tau20 = np.array([0.6] * 8 + [0.7] * 12)
    a = oracle.diss_run(Q, f0.gamma, tau20, dp, 12)
    b = R.diss_run(Q, f0.gamma, tau20, 0.02, 0.03, 0.05, 2.0, powell, 12)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    # and the dissipation matters at this size (the comparison is not of two ideal runs)
    c = oracle.diss_run(Q, f0.gamma, tau20, oracle.Dissipation(tau_m=2.0, powell=powell), 12)
    assert np.abs(a - c).max() > 1e-6 * np.abs(a).max()



@pytest.mark.parametrize("powell", [False, True])
def test_update_is_covariant_under_the_quarter_turn_of_the_lattice(powell):
    # D2Q5 and the dissipative system are invariant under the quarter turn about z,
    # (x, y) -> (-y, x): positions move, rho u and B turn as vectors, G and W as tensors
    # (T' = R T R^T; their rows x, y map onto each other and the z row stays absent)
    from test_oracle_pins import _rotate_ideal
    n = 10
    Rm = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    Y, Xg = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")

    def move(A):  # the value at (x, y) lands at (-y, x)
        return A[..., (-Xg) % n, Y]

    def rotate(Q):
        out = np.empty_like(Q)
        out[:8] = _rotate_ideal(Q[:8])
        for lo in (8, 14):
            T = np.zeros((3, 3, n, n))
            T[:2] = Q[lo:lo + 6].reshape(2, 3, n, n)
            T = np.einsum("ik,jl,kl...->ij...", Rm, Rm, T)
            assert np.abs(T[2]).max() == 0.0
            out[lo:lo + 6] = move(T[:2].reshape(6, n, n))
        return out

    f0 = fields.ideal_fields((n, n), 91, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(92)
    Q = np.concatenate([f0.Q, 0.05 * rng.normal(size=(12, n, n))])
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=0.05, tau_m=1.5, powell=powell)
    tau = [0.6, 0.55, 0.55, 0.55, 0.7, 0.65, 0.65, 0.65]
    a = rotate(oracle.diss_run(Q, f0.gamma, tau, dp, 8, tau_g=0.7))
    b = oracle.diss_run(rotate(Q), f0.gamma, tau, dp, 8, tau_g=0.7)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    # four quarter turns are the identity
    R = Q
    for _ in range(4):
        R = rotate(R)
    np.testing.assert_array_equal(R, Q)
