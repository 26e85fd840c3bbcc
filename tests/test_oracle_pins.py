"""Pins of the CPU oracle to things other than itself.

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's code: quadrature conditions of the
velocity sets, the textbook MHD wave speeds (eigenvalues of the flux
Jacobian), a sound speed the paper prints, exact discrete invariants
(uniform fixed point, conservation, centred div B), Chapman-Enskog decay
rates, closed-form Hartmann/Poiseuille profiles and an independent NumPy
restatement on tiny grids.
"""
import math
import os

import numpy as np
import pytest

from paper_2606_00641_gb300 import fields

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (t.strip() for t in line.split("=", 1))
            parts = v.split()
            vals[k] = float(parts[0]) if len(parts) == 1 else [float(t) for t in parts]
    return vals


def state(rho, u, p, B, gamma):
    u = np.asarray(u, float)
    B = np.asarray(B, float)
    e = p / (gamma - 1) + 0.5 * rho * u @ u + 0.5 * B @ B
    return np.array([rho, *(rho * u), e, *B])


def mhd_speeds(rho, u, p, B, gamma, axis):
    """Textbook ideal-MHD characteristic speeds along ``axis`` (conservative
    8-field system with the div-B flux row identically zero)."""
    a2 = gamma * p / rho
    b2 = float(np.dot(B, B)) / rho
    bn2 = B[axis] ** 2 / rho
    disc = math.sqrt(max((a2 + b2) ** 2 - 4 * a2 * bn2, 0.0))
    cf = math.sqrt(0.5 * (a2 + b2 + disc))
    cs = math.sqrt(max(0.5 * (a2 + b2 - disc), 0.0))
    ca = math.sqrt(bn2)
    un = u[axis]
    return np.sort([un - cf, un - ca, un - cs, un, 0.0, un + cs, un + ca, un + cf])


def flux_jacobian(orc, gamma, Q, axis, h=1e-6):
    J = np.zeros((8, 8))
    for j in range(8):
        dq = np.zeros(8)
        dq[j] = h * max(1.0, abs(Q[j]))
        fp = orc.ideal_flux(gamma, Q + dq)[:, axis]
        fm = orc.ideal_flux(gamma, Q - dq)[:, axis]
        J[:, j] = (fp - fm) / (2 * dq[j])
    return J


# --------------------------------------------------------------------------
# velocity sets
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q", [5, 7, 19])
def test_lattice_quadrature(orc, q):
    c, w, cs2, opp = orc.lattice(q)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs((w[:, None] * c).sum(0)).max() < 1e-15
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, cs2 * np.eye(3) * (np.abs(c).sum(0) > 0), atol=1e-15)
    third = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.abs(third).max() < 1e-15
    for i in range(q):
        assert (c[opp[i]] == -c[i]).all()
    if q == 19:
        # fourth-order isotropy needed by the second-order flow equilibrium
        fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
        d = np.eye(3)
        iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                          + np.einsum("ad,bc->abcd", d, d))
        assert np.allclose(fourth, iso, atol=1e-15)


# --------------------------------------------------------------------------
# flux (Eq. 12 + EOS Eq. 9): eigenvalues of its Jacobian = MHD wave speeds
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_flux_jacobian_eigenvalues_are_mhd_wave_speeds(orc, seed):
    rng = np.random.default_rng(seed)
    gamma = [5 / 3, 1.4, 2.0][seed % 3]
    rho = rng.uniform(0.5, 2.0)
    u = rng.normal(size=3) * 0.5
    B = rng.normal(size=3) * 0.7
    p = rng.uniform(0.2, 1.5)
    Q = state(rho, u, p, B, gamma)
    for axis in range(3):
        ev = np.linalg.eigvals(flux_jacobian(orc, gamma, Q, axis))
        assert np.abs(ev.imag).max() < 1e-5
        np.testing.assert_allclose(np.sort(ev.real), mhd_speeds(rho, u, p, B, gamma, axis),
                                   atol=2e-6)


def test_orszag_tang_sound_speed_printed_in_paper(orc):
    g = read_golden("orszag_tang_state.txt")
    Q = state(g["rho"], [0, 0, 0], g["p"], [0, 0, 0], g["gamma"])
    ev = np.sort(np.linalg.eigvals(flux_jacobian(orc, g["gamma"], Q, 0)).real)
    assert abs(ev[-1] - g["sound_speed"]) < 1e-6
    assert abs(ev[0] + g["sound_speed"]) < 1e-6


def test_flux_velocity_scaling_invariance(orc):
    # ideal MHD is invariant under u -> u/l, B -> B/l, p -> p/l^2 (sec. 2.2
    # "Unit conversion"): fluxes scale by l^-1 (rho), l^-2 (rho u, B), l^-3 (e)
    rng = np.random.default_rng(7)
    gamma = 5 / 3
    rho, u, B, p = 1.3, rng.normal(size=3), rng.normal(size=3), 0.9
    lam = 7.0
    F1 = orc.ideal_flux(gamma, state(rho, u, p, B, gamma))
    F2 = orc.ideal_flux(gamma, state(rho, u / lam, p / lam ** 2, B / lam, gamma))
    scale = np.array([lam, lam ** 2, lam ** 2, lam ** 2, lam ** 3, lam ** 2, lam ** 2, lam ** 2])
    np.testing.assert_allclose(F2 * scale[:, None], F1, rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------
# equilibrium moments (Eq. 3, Eq. 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_moments_return_state_and_flux(orc, dim):
    shape = (6, 5) if dim == 2 else (3, 4, 5)
    f0 = fields.ideal_fields(shape, 11, mach=1.5, beta=1.0, cfl=0.2)
    Q0 = f0.Q
    f = orc.ideal_init(Q0, f0.gamma)
    np.testing.assert_allclose(orc.ideal_moments(f), Q0, rtol=1e-14, atol=1e-16)
    c, w, cs2, _ = orc.lattice(5 if dim == 2 else 7)
    first = np.einsum("kixyz,ia->kaxyz".replace("xyz", "yx" if dim == 2 else "zyx"), f, c)
    cell = (2, 3) if dim == 2 else (1, 2, 3)
    phi = orc.ideal_flux(f0.gamma, Q0[(slice(None),) + cell])
    got = first[(slice(None), slice(None)) + cell]
    np.testing.assert_allclose(got[:, :dim], phi[:, :dim], rtol=1e-13, atol=1e-17)


# --------------------------------------------------------------------------
# exact discrete invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_state_is_fixed_point(orc, dim):
    shape = (7, 9) if dim == 2 else (4, 5, 6)
    gamma = 5 / 3
    Q = fields.uniform_ideal_state(shape, rho=1.2, u=(0.03, -0.02, 0.01), p=0.02,
                                   B=(0.05, 0.04, -0.03), gamma=gamma)
    out = orc.ideal_run(Q, gamma, 0.51, 60)
    np.testing.assert_allclose(out, Q, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("dim,tau", [(2, 0.51), (2, 0.9), (3, 0.51), (3, 0.7)])
def test_exact_conservation_periodic(orc, dim, tau):
    shape = (32, 32) if dim == 2 else (10, 12, 14)
    f0 = fields.ideal_fields(shape, 1001 + dim, mach=1.0, cfl=0.1 if dim == 2 else 0.2)
    n = 100
    out = orc.ideal_run(f0.Q, f0.gamma, tau, n)
    s0 = f0.Q.reshape(8, -1).sum(1)
    s1 = out.reshape(8, -1).sum(1)
    scale = np.abs(f0.Q).reshape(8, -1).sum(1) + 1e-300
    assert (np.abs(s1 - s0) / scale).max() < 1e-12


def test_direct_source_injection_adds_S_per_cell_per_step(orc):
    f0 = fields.ideal_fields((16, 16), 5, cfl=0.1)
    S = np.array([1e-4, 2e-5, -3e-5, 0.0, 5e-6, 1e-6, -2e-6, 0.0])
    n = 20
    out = orc.ideal_run(f0.Q, f0.gamma, 0.6, n, src=S)
    N = 16 * 16
    ds = out.reshape(8, -1).sum(1) - f0.Q.reshape(8, -1).sum(1)
    np.testing.assert_allclose(ds, n * N * S, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_centred_divB_stays_zero_with_tau_B_one(orc, dim):
    # derivation: with tau = 1 on the three B lattices,
    # sum_b d_b B_b^{n+1}(x) = sum_i w_i (d.B)^n(x - c_i), because the
    # induction flux is antisymmetric and centred differences commute.
    shape = (24, 24) if dim == 2 else (10, 10, 10)
    f0 = fields.ideal_fields(shape, 42, mach=1.5, beta=0.5, cfl=0.1 if dim == 2 else 0.2)
    tau = np.array([0.7] * 5 + [1.0] * 3)
    f = orc.ideal_init(f0.Q, f0.gamma)
    Bmax = np.abs(f0.Q[5:8]).max()
    for _ in range(40):
        f = orc.ideal_step(f, f0.gamma, tau)
    Q = orc.ideal_moments(f)
    div = fields.centred_divergence(Q[5], Q[6], Q[7] if dim == 3 else None)
    assert np.abs(div).max() < 1e-13 * Bmax
    # sensitivity: with tau_B != 1 the invariant is not exact
    f = orc.ideal_init(f0.Q, f0.gamma)
    for _ in range(40):
        f = orc.ideal_step(f, f0.gamma, 0.7)
    Q = orc.ideal_moments(f)
    div = fields.centred_divergence(Q[5], Q[6], Q[7] if dim == 3 else None)
    assert np.abs(div).max() > 1e-9 * Bmax


# --------------------------------------------------------------------------
# linear waves: speed = eigenvalue of the flux Jacobian, decay rate from the
# Chapman-Enskog expansion (Eq. 5 generalised): D = (tau - 1/2)(cs^2 - a^2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["sound", "alfven", "oblique"])
def test_linear_wave_speed_and_decay(orc, case):
    gamma = 5 / 3
    cs2_lat = 1.0 / 3.0
    # base states with distinct characteristic speeds along x
    if case == "sound":
        rho, u, p, B = 1.0, [0.02, 0, 0], 0.006, [0, 0, 0]
        targets = ["fast+", "fast-"]
    elif case == "alfven":
        rho, u, p, B = 1.0, [0.01, 0.01, 0], 0.006, [0.08, 0.02, 0]
        targets = ["alfven+", "fast+"]
    else:
        rho, u, p, B = 1.1, [0.015, -0.01, 0.005], 0.005, [0.06, 0.07, 0.02]
        targets = ["slow+", "fast-"]
    base = state(rho, u, p, B, gamma)
    J = flux_jacobian(orc, gamma, base, 0)
    ev, R = np.linalg.eig(J)
    assert np.abs(ev.imag).max() < 1e-6
    # make every eigenvector real (each is a real vector times a phase)
    for j in range(8):
        col = R[:, j]
        R[:, j] = col * np.exp(-1j * np.angle(col[np.argmax(np.abs(col))]))
    R = R.real
    L = np.linalg.inv(R)
    a2 = gamma * p / rho
    b2 = float(np.dot(B, B)) / rho
    bn2 = B[0] ** 2 / rho
    disc = math.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)
    want = {"fast+": u[0] + math.sqrt(0.5 * (a2 + b2 + disc)),
            "fast-": u[0] - math.sqrt(0.5 * (a2 + b2 + disc)),
            "slow+": u[0] + math.sqrt(0.5 * (a2 + b2 - disc)),
            "alfven+": u[0] + math.sqrt(bn2)}
    tau = 0.8
    nx, n, eps = 128, 1500, 1e-7
    x = np.arange(nx)
    k = 2 * math.pi / nx
    for name in targets:
        lam = want[name]
        j = int(np.argmin(np.abs(ev.real - lam)))
        assert abs(ev[j].real - lam) < 1e-6
        r = R[:, j] / np.abs(R[:, j]).max()
        Q = base[:, None] + eps * r[:, None] * np.cos(k * x)[None, :]
        f = orc.ideal_init(Q[:, None, :], gamma)
        for _ in range(n):
            f = orc.ideal_step(f, gamma, tau)
        Qn = orc.ideal_moments(f)[:, 0, :] - base[:, None]
        a_n = np.sum((L[j] @ Qn) * np.exp(-1j * k * x))
        a_0 = 0.5 * nx * eps * (L[j] @ r)
        phase = -np.angle(a_n / a_0)
        turns = round((lam * k * n - phase) / (2 * math.pi))
        speed = (phase + 2 * math.pi * turns) / (k * n)
        assert abs(speed - lam) < 3e-3 * abs(lam), (name, speed, lam)
        D = -math.log(abs(a_n / a_0)) / (k * k * n)
        D_ce = (tau - 0.5) * (cs2_lat - lam * lam)
        assert abs(D - D_ce) < 0.03 * D_ce, (name, D, D_ce)


# --------------------------------------------------------------------------
# the exact linearised scheme: one Fourier mode of a uniform state evolves by
# the 40 x 40 D2Q5 update operator M(kappa) = S(kappa) [(1 - W) + W E P]
# (BGK towards the first-order equilibrium, Eqs. 2-3, then streaming), so
# after n steps its moments are P M^n E r, to second order in the amplitude.
# --------------------------------------------------------------------------

def flux_jacobian_4th(orc, gamma, Q, axis, h=1e-3):
    """d Phi[:, axis] / dQ by the fourth-order central difference (truncation
    ~h^4, rounding ~1e-16/h: ~1e-12 here)."""
    J = np.zeros((8, 8))
    for j in range(8):
        d = np.zeros(8)
        d[j] = h
        fl = lambda s: orc.ideal_flux(gamma, Q + s * d)[:, axis]
        J[:, j] = (8 * (fl(1) - fl(-1)) - (fl(2) - fl(-2))) / (12 * h)
    return J


def linearised_operator(orc, gamma, base, tau, kappa):
    """M, E, P of the D2Q5 (len(kappa) == 2) or D3Q7 (3) scheme linearised about
    the uniform state `base` for the mode exp(i kappa . x): populations ordered
    (lattice, direction)."""
    dim = len(kappa)
    q = 5 if dim == 2 else 7
    n = 8 * q
    c, w, cs2, _ = orc.lattice(q)
    J = [flux_jacobian_4th(orc, gamma, base, a) for a in range(dim)]
    E = np.zeros((n, 8))  # d f_eq / d Q
    P = np.zeros((8, n))  # moments: sum over the directions of a lattice
    omega = np.zeros(n)
    shift = np.zeros(n, complex)
    for k in range(8):
        for i in range(q):
            row = q * k + i
            E[row, k] += w[i]
            for a in range(dim):
                E[row] += w[i] * c[i, a] * J[a][k] / cs2
            P[k, row] = 1.0
            omega[row] = 1.0 / tau[k]
            # pushed along c_i: the value at x came from x - c_i
            shift[row] = np.exp(-1j * sum(kappa[a] * c[i, a] for a in range(dim)))
    M = shift[:, None] * (np.diag(1 - omega) + omega[:, None] * (E @ P))
    return M, E, P


def test_linearised_update_operator_predicts_the_run(orc):
    gamma = 5 / 3
    base = state(1.05, [0.03, -0.02, 0.015], 0.05, [0.12, -0.09, 0.06], gamma)
    tau = np.array([0.62, 0.71, 0.66, 0.93, 0.58, 1.15, 0.77, 0.84])
    ny, nx, n = 16, 32, 120
    kappa = (2 * math.pi * 3 / nx, 2 * math.pi * 1 / ny)
    r = np.random.default_rng(7).normal(size=8)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    wave = np.exp(1j * (kappa[0] * x + kappa[1] * y))
    eps = 1e-5
    runs = []
    for s in (1, -1):
        Q0 = base[:, None, None] + s * eps * r[:, None, None] * np.cos(kappa[0] * x + kappa[1] * y)
        f = orc.ideal_init(Q0, gamma)
        for _ in range(n):
            f = orc.ideal_step(f, gamma, tau)
        runs.append(orc.ideal_moments(f))
    measured = (runs[0] - runs[1]) / (2 * eps)  # the quadratic term cancels
    M, E, P = linearised_operator(orc, gamma, base, tau, kappa)
    amp = P @ np.linalg.matrix_power(M, n) @ E @ r
    predicted = (amp[:, None, None] * wave[None]).real
    assert np.abs(predicted).max() > 0.05  # the mode is still there
    err = np.abs(measured - predicted).max() / np.abs(predicted).max()
    assert err < 1e-8, err


def test_linearised_d3q7_operator_predicts_the_3d_run(orc):
    # the same exact statement for the 3-D scheme: a mode oblique to all three axes
    # (every direction of D3Q7 streams it), per-lattice tau, 56 x 56 operator
    gamma = 5 / 3
    base = state(0.95, [-0.02, 0.025, 0.01], 0.04, [0.08, 0.1, -0.07], gamma)
    tau = np.array([0.56, 0.53, 0.6, 0.55, 0.7, 0.58, 0.8, 0.54])
    nz, ny, nx, n = 8, 12, 16, 30
    kappa = (2 * math.pi * 1 / nx, -2 * math.pi * 1 / ny, 2 * math.pi * 1 / nz)
    r = np.random.default_rng(9).normal(size=8)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phase = kappa[0] * x + kappa[1] * y + kappa[2] * z
    eps = 2e-6  # cubic remainder ~ (eps |r| / p)^2 ~ 2e-9 at p = 0.04; rounding ~ 1e-16 / eps
    runs = []
    for s in (1, -1):
        Q0 = base[:, None, None, None] + s * eps * r[:, None, None, None] * np.cos(phase)
        f = orc.ideal_init(Q0, gamma)
        for _ in range(n):
            f = orc.ideal_step(f, gamma, tau)
        runs.append(orc.ideal_moments(f))
    measured = (runs[0] - runs[1]) / (2 * eps)
    M, E, P = linearised_operator(orc, gamma, base, tau, kappa)
    amp = P @ np.linalg.matrix_power(M, n) @ E @ r
    predicted = (amp[:, None, None, None] * np.exp(1j * phase)[None]).real
    assert np.abs(predicted).max() > 0.05
    err = np.abs(measured - predicted).max() / np.abs(predicted).max()
    assert err < 1e-8, err


def test_linearised_operator_has_the_mhd_speeds_and_decay(orc):
    """The 8 slow eigenvalues of M approach exp(-i k lambda - D k^2) with the
    textbook speeds lambda and the Chapman-Enskog D = (tau - 1/2)(cs^2 - lambda^2)."""
    gamma = 5 / 3
    rho, u, p, B = 1.1, [0.02, -0.01, 0.01], 0.05, [0.12, 0.09, -0.05]
    base = state(rho, u, p, B, gamma)
    tau = 0.8
    _, _, cs2, _ = orc.lattice(5)
    k = 2 * math.pi / 512
    M, _, _ = linearised_operator(orc, gamma, base, np.full(8, tau), (k, 0.0))
    mu = np.linalg.eigvals(M)
    slow = mu[np.argsort(-np.abs(mu))[:8]]
    assert np.abs(mu[np.argsort(-np.abs(mu))[8:]]).max() < 0.5  # kinetic modes decay fast
    speed = np.sort(-np.angle(slow) / k)
    lam = mhd_speeds(rho, np.asarray(u), p, np.asarray(B), gamma, 0)
    np.testing.assert_allclose(speed, lam, atol=1e-4)
    order = np.argsort(-np.angle(slow) / k)
    D = -np.log(np.abs(slow[order])) / k ** 2
    np.testing.assert_allclose(D, (tau - 0.5) * (cs2 - lam ** 2), rtol=2e-3)


def test_first_order_self_convergence(orc):
    # Acoustic scaling (the lattice velocities do not change with N, so a fixed
    # physical time is N/2 steps) at fixed tau: the scheme's diffusion
    # (tau - 1/2)(cs^2 - A^2) dx vanishes linearly with dx, so the solution at N
    # differs from the one at 2N (sampled at the same points) by O(dx), and the
    # difference halves when N doubles -- for every field, B included.  A wrong
    # streaming distance, a time step that does not scale with dx or an input
    # that changes with the resolution breaks the ratio.
    runs = {}
    for n in (32, 64, 128, 256):
        f0 = fields.ideal_fields((n, n), 1001, mach=0.5, cfl=0.1)
        runs[n] = orc.ideal_run(f0.Q, f0.gamma, 0.6, n // 2, nthreads=4)
    err = {}
    for n in (32, 64, 128):
        coarse, fine = runs[n], runs[2 * n][:, ::2, ::2]
        err[n] = np.sqrt(((coarse - fine) ** 2).mean(axis=(1, 2)) / (coarse ** 2).mean(axis=(1, 2)))
    for n in (32, 64):
        ratio = err[n] / err[2 * n]
        assert ((ratio > 1.7) & (ratio < 2.6)).all(), (n, ratio)
    assert err[128].max() < 0.02


def test_brio_wu_states_smoke(orc):
    # the paper's Brio-Wu states (sec. 3.1): the run stays finite and
    # positive, conserves mass exactly, and the undisturbed far field ahead
    # of the fastest left-going wave keeps the left state.
    g = read_golden("brio_wu_states.txt")
    gamma = g["gamma"]
    nx = 400
    QL = state(g["left"][0], [g["left"][2], g["left"][3], 0], g["left"][1],
               [g["left"][4], g["left"][5], 0], gamma)
    QR = state(g["right"][0], [g["right"][2], g["right"][3], 0], g["right"][1],
               [g["right"][4], g["right"][5], 0], gamma)
    rhoL, pL, BL = g["left"][0], g["left"][1], np.array([g["left"][4], g["left"][5], 0])
    cfL = math.sqrt((gamma * pL + BL @ BL) / rhoL)
    lam = 2.0 * cfL / 0.1  # CFL 0.1 on the fastest speed (lattice units)
    scale = np.array([1, 1 / lam, 1 / lam, 1 / lam, 1 / lam ** 2, 1 / lam, 1 / lam, 1 / lam])
    Q = np.where(np.arange(nx)[None, :] < nx // 2, (QL * scale)[:, None], (QR * scale)[:, None])
    # make it periodic-safe: mirror so that both interfaces are far apart
    Q = np.concatenate([Q, Q[:, ::-1]], axis=1)[:, None, :]
    nsteps = 600
    out = orc.ideal_run(Q, gamma, 0.6, nsteps)
    assert np.isfinite(out).all()
    assert out[0].min() > 0
    p = np.array([orc.ideal_pressure(gamma, out[:, 0, i]) for i in range(out.shape[2])])
    assert p.min() > 0
    assert abs(out[0].sum() - Q[0].sum()) < 1e-11 * Q[0].sum()
    reach = int((cfL / lam) * nsteps) + 40  # fastest wave plus a diffusive margin
    far = slice(0, nx // 2 - reach)
    assert far.stop > 20
    np.testing.assert_allclose(out[0, 0, 10:far.stop], rhoL, rtol=1e-6)


# --------------------------------------------------------------------------
# brute force: C oracle vs the independent NumPy restatement
# --------------------------------------------------------------------------

def _rotate_ideal(Q):
    """The rotation of the whole state that the lattice maps onto itself: in 2-D the
    quarter turn about z, (x, y) -> (-y, x), on a square grid; in 3-D the cyclic
    x -> y -> z.  Positions and the vectors rho u and B turn together."""
    out = np.empty_like(Q)
    if Q.ndim == 3:  # [8, ny, nx], ny == nx
        n = Q.shape[-1]
        Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        moved = Q[:, (-X) % n, Y]          # value at (x, y) lands at (-y, x)
        out[:] = moved
        for v in (1, 5):                   # (v_x, v_y, v_z) -> (-v_y, v_x, v_z)
            out[v], out[v + 1] = -moved[v + 1], moved[v]
        return out
    moved = np.moveaxis(Q, -3, -1)         # value at (x, y, z) lands at (z, x, y)
    out = moved.copy()
    for v in (1, 5):                       # (v_x, v_y, v_z) -> (v_z, v_x, v_y)
        out[v:v + 3] = np.roll(moved[v:v + 3], 1, axis=0)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_update_is_covariant_under_the_rotations_of_the_lattice(orc, dim):
    # D2Q5 and D3Q7 are invariant under these rotations and so is ideal MHD: the run of the
    # rotated state is the rotated run (to rounding; the state itself is far from symmetric)
    shape = (12, 12) if dim == 2 else (4, 5, 6)
    f0 = fields.ideal_fields(shape, 333, mach=1.0, beta=1.0, cfl=0.2)
    tau = [0.6, 0.55, 0.55, 0.55, 0.7, 0.65, 0.65, 0.65]   # equal within each vector
    a = _rotate_ideal(orc.ideal_run(f0.Q, f0.gamma, tau, 9))
    b = orc.ideal_run(_rotate_ideal(f0.Q), f0.gamma, tau, 9)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    R = _rotate_ideal(f0.Q)
    corner = (slice(None),) + (slice(0, 4),) * dim
    assert np.abs(R[corner] - f0.Q[corner]).max() > 0.05 * np.abs(f0.Q).max()
    # four quarter turns (three cyclic rotations) are the identity
    for _ in range(3 if dim == 2 else 2):
        R = _rotate_ideal(R)
    np.testing.assert_array_equal(R, f0.Q)


@pytest.mark.parametrize("dim", [2, 3])
def test_c_oracle_matches_numpy_restatement(orc, dim):
    from oracle import numpy_ref
    shape = (8, 8) if dim == 2 else (4, 4, 4)
    f0 = fields.ideal_fields(shape, 77, mach=1.2, beta=1.0, cfl=0.15)
    tau = np.array([0.51, 0.6, 0.7, 0.8, 0.55, 0.9, 1.0, 0.65])
    S = np.array([1e-5, 0, 2e-6, 0, -1e-6, 0, 0, 3e-7])
    a = orc.ideal_run(f0.Q, f0.gamma, tau, 50, src=S)
    b = numpy_ref.ideal_run(f0.Q, f0.gamma, tau, 50, src=S)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)
