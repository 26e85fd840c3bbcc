"""Pins of the oracle's dissipative MHD with locally evolved gradients on the
D3Q7 lattice (sec. 2.2.1 "Local Moments Evolution", sec. 2.3 "Evolution of the
MHD equation system"): 26 lattices, G_ab ~ tau_M d_a B_b at 8 + 3a + b and
W_ab ~ tau_M d_a u_b at 17 + 3a + b, with a = x, y, z.

What the 2-D pins cannot see is the third gradient row and the wider layout:
checked against the pinned 3-D ideal scheme (no dissipation), the covariance of
the whole update under the cyclic rotation x -> y -> z of positions, vectors
and tensors (the D3Q7 lattice and the MHD system are both invariant), the
decay of shear and magnetic-diffusion modes along z at nu k^2 and eta0 k^2 plus
the D3Q7 lattice's (tau - 1/2) k^2 / 4, the z-gradient balance G -> tau_M d_z B,
a closed-form uniform step whose Powell divergence is the full trace
G_xx + G_yy + G_zz, exact conservation, and the NumPy restatement.
"""
import numpy as np
import pytest

import oracle
from oracle import numpy_ref as R
from paper_2606_00641_gb300 import fields

GAMMA = 5.0 / 3.0
NV = 26
W0 = 17                 # first W_ab lattice in 3-D
N = 64
K = 2 * np.pi / N
Z = np.arange(N)
TAU_M = 2.0
TAU = 0.55
CS2 = 0.25              # D3Q7
TAU8 = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]


def _random_state(shape, seed, amp=0.01):
    f0 = fields.ideal_fields(shape, seed, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(seed)
    return f0, np.concatenate([f0.Q, amp * rng.normal(size=(18,) + shape)])


def _rotate(Q):
    """The cyclic rotation x -> y -> z: a value at position (x, y, z) moves to
    (z, x, y), vector component a to a + 1 (mod 3), and both indices of G and W."""
    sp = Q.shape[1:]
    out = np.empty((NV,) + (sp[1], sp[2], sp[0]))

    def pos(a):        # array axes (z, y, x) -> (z', y', x') with z' = y, y' = x, x' = z
        return np.moveaxis(a, -3, -1)

    out[0] = pos(Q[0])
    out[4] = pos(Q[4])
    out[1:4] = np.roll(pos(Q[1:4]), 1, axis=0)
    out[5:8] = np.roll(pos(Q[5:8]), 1, axis=0)
    for lo in (8, W0):
        T = pos(Q[lo:lo + 9]).reshape((3, 3) + out.shape[1:])
        out[lo:lo + 9] = np.roll(np.roll(T, 1, axis=0), 1, axis=1).reshape((9,) + out.shape[1:])
    return out


def test_without_dissipation_the_mhd_fields_follow_the_ideal_scheme():
    shape = (4, 5, 6)
    f0, Q = _random_state(shape, 81)
    got = oracle.diss_run(Q, f0.gamma, TAU8, oracle.Dissipation(tau_m=1.5), 12, tau_g=0.7)
    ref = oracle.ideal_run(f0.Q, f0.gamma, TAU8, 12)
    scale = np.abs(f0.Q).reshape(8, -1).max(1)
    assert (np.abs(got[:8] - ref).reshape(8, -1).max(1) / scale).max() < 1e-13


@pytest.mark.parametrize("powell", [False, True])
def test_update_is_covariant_under_the_cyclic_rotation_of_the_axes(powell):
    shape = (4, 5, 6)
    f0, Q = _random_state(shape, 82, amp=0.05)
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=0.05, tau_m=1.5, powell=powell)
    a = _rotate(oracle.diss_run(Q, f0.gamma, TAU8, dp, 8, tau_g=0.7))
    b = oracle.diss_run(_rotate(Q), f0.gamma, TAU8, dp, 8, tau_g=0.7)
    assert a.shape == b.shape == (NV, 5, 6, 4)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    # and the state is far from rotation-invariant, so the check has teeth
    assert np.abs(_rotate(Q)[:, :4, :4, :4] - Q[:, :4, :4, :4]).max() > 0.1


def _column(field, amp, lattice=None):
    """Gas at rest in a 2 x 2 x N column with one field = amp sin(k z), its
    gradient lattice (if given) at the balance tau_M d_z."""
    Q = np.zeros((NV, N, 2, 2))
    Q[0] = 1.0
    Q[4] = 0.02 / (GAMMA - 1)
    prof = amp * np.sin(K * Z)[:, None, None]
    Q[field] = prof
    Q[4] += 0.5 * prof ** 2
    if lattice is not None:
        Q[lattice] = TAU_M * amp * K * np.cos(K * Z)[:, None, None]
    return Q


def _amp(field):
    return 2 * np.mean(field[:, 0, 0] * np.sin(K * Z))


def _rate(Q, dp, t0, t1, field):
    a0 = _amp(oracle.diss_run(Q, GAMMA, TAU, dp, t0, tau_g=0.55)[field])
    a1 = _amp(oracle.diss_run(Q, GAMMA, TAU, dp, t1, tau_g=0.55)[field])
    return np.log(a0 / a1) / (t1 - t0)


@pytest.mark.parametrize("nu", [0.0, 0.01])
def test_shear_wave_along_z_decays_at_nu_plus_the_lattice_diffusion(nu):
    # u_x = U sin(kz) with W_zx at its balance
    rate = _rate(_column(1, 1e-3, W0 + 3 * 2 + 0), oracle.Dissipation(nu=nu, tau_m=TAU_M), 20, 200, 1)
    expect = (nu + (TAU - 0.5) * CS2) * K * K
    assert abs(rate / expect - 1) < 0.01, (rate, expect)


@pytest.mark.parametrize("eta0", [0.0, 0.01])
def test_magnetic_sheet_along_z_diffuses_at_eta_plus_the_lattice_diffusion(eta0):
    # B_y = b sin(kz) with G_zy at its balance
    rate = _rate(_column(6, 1e-3, 8 + 3 * 2 + 1), oracle.Dissipation(eta0=eta0, tau_m=TAU_M), 20, 200, 6)
    expect = (eta0 + (TAU - 0.5) * CS2) * K * K
    assert abs(rate / expect - 1) < 0.005, (rate, expect)


def test_z_gradient_lattices_relax_to_tau_m_times_the_gradients():
    # B_y(z) and u_x(z) from G = W = 0: G_zy and W_zx grow to tau_M d_z
    b, U = 1e-3, 1e-3
    Q = _column(6, b)
    Q[1] = U * np.sin(K * Z)[:, None, None]
    Q[4] += 0.5 * Q[1] ** 2
    out = oracle.diss_run(Q, GAMMA, TAU, oracle.Dissipation(tau_m=TAU_M), 20, tau_g=0.55)
    expect = TAU_M * 1e-3 * K * np.cos(K * Z)
    g_zy, w_zx = out[8 + 7][:, 0, 0], out[W0 + 6][:, 0, 0]
    assert np.abs(g_zy - expect).max() < 0.02 * np.abs(expect).max()
    assert np.abs(w_zx - expect).max() < 0.02 * np.abs(expect).max()
    # nothing varies along x or y, and B_x, B_z, u_y stay zero; W_zz is left free
    # (the magnetic pressure of B_y(z) drives a second-order u_z(z))
    zero = list(range(8, 14)) + list(range(W0, W0 + 6)) + [8 + 6, 8 + 8, W0 + 7]
    assert np.abs(out[zero]).max() < 1e-15
    assert 0 < np.abs(out[W0 + 8]).max() < 1e-2 * np.abs(expect).max()


def test_uniform_step_with_the_powell_source_and_relaxing_gradients():
    # a uniform state does not stream; one step adds the source once:
    # G, W -> (1 - 1/tau_M) G, W and, with div B = (G_xx + G_yy + G_zz) / tau_M,
    # the Powell terms -(div B)(0, B, u.B, u) on the MHD fields
    Q0 = np.zeros(NV)
    Q0[0], Q0[1:4], Q0[4], Q0[5:8] = 1.1, [0.05, -0.02, 0.01], 0.1, [0.1, -0.05, 0.04]
    Q0[8:] = 0.01 * np.arange(1, 19)
    grid = np.broadcast_to(Q0[:, None, None, None], (NV, 2, 3, 4)).copy()
    tau_m = 2.5
    dp = oracle.Dissipation(nu=0.01, eta0=0.02, j_c=0.1, tau_m=tau_m, powell=True)
    one = oracle.diss_run(grid, GAMMA, 0.6, dp, 1, tau_g=0.7)
    assert np.abs(one - one[:, :1, :1, :1]).max() == 0.0
    one = one[:, 0, 0, 0]
    divB = (Q0[8] + Q0[12] + Q0[16]) / tau_m
    u = Q0[1:4] / Q0[0]
    expect = Q0.copy()
    expect[1:4] -= divB * Q0[5:8]
    expect[4] -= divB * (u @ Q0[5:8])
    expect[5:8] -= divB * u
    expect[8:] *= 1 - 1 / tau_m
    np.testing.assert_allclose(one, expect, rtol=1e-12, atol=1e-16)


def test_flux_and_source_of_one_state_have_the_3d_layout():
    Q0 = np.zeros(NV)
    Q0[0], Q0[1:4], Q0[4], Q0[5:8] = 1.0, [0.1, 0.2, 0.3], 1.0, [0.3, 0.2, 0.1]
    Q0[8:] = 0.01 * np.arange(1, 19)
    dp = oracle.Dissipation(tau_m=2.0)
    phi = oracle.diss_flux(GAMMA, dp, Q0, dim=3)
    u, B = Q0[1:4], Q0[5:8]
    for a in range(3):
        for b in range(3):
            np.testing.assert_allclose(phi[8 + 3 * a + b], Q0[8 + 3 * a + b] * u - np.eye(3)[a] * B[b], rtol=1e-15)
            np.testing.assert_allclose(phi[W0 + 3 * a + b], Q0[W0 + 3 * a + b] * u - np.eye(3)[a] * u[b],
                                       rtol=1e-15)
    np.testing.assert_allclose(oracle.diss_source(dp, Q0, dim=3)[8:], -Q0[8:] / 2.0, rtol=1e-15)
    with pytest.raises(ValueError):
        oracle.diss_flux(GAMMA, dp, Q0[:20], dim=3)


def test_conserved_fields_are_conserved_exactly():
    shape = (4, 6, 5)
    f0, Q = _random_state(shape, 83)
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=0.05, tau_m=1.5, powell=False)
    out = oracle.diss_run(Q, f0.gamma, 0.6, dp, 15, tau_g=0.7)
    s0 = Q[:8].reshape(8, -1).sum(1)
    s1 = out[:8].reshape(8, -1).sum(1)
    scale = np.abs(Q[:8]).reshape(8, -1).sum(1)
    assert (np.abs(s1 - s0) / scale).max() < 1e-13


@pytest.mark.parametrize("powell", [False, True])
def test_oracle_matches_numpy_restatement(powell):
    shape = (4, 5, 6)
    f0, Q = _random_state(shape, 84)
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=0.05, tau_m=2.0, powell=powell)
    tau26 = np.array([0.6] * 8 + [0.7] * 18)
    a = oracle.diss_run(Q, f0.gamma, tau26, dp, 8)
    b = R.diss_run(Q, f0.gamma, tau26, 0.02, 0.03, 0.05, 2.0, powell, 8)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    c = oracle.diss_run(Q, f0.gamma, tau26, oracle.Dissipation(tau_m=2.0, powell=powell), 8)
    assert np.abs(a - c).max() > 1e-6 * np.abs(a).max()
