"""Seeded synthetic initial fields, in lattice units, for the VLBM workloads.

This module only builds inputs.  It contains none of the update arithmetic
(no equilibrium, no flux, no collision, no streaming); both the CUDA library
and the CPU oracle receive the arrays it returns.

Recipe (the same for every workload, parameters per workload):

* random-phase scalar modes: ``s(x) = sum_m cos(2 pi k_m . x / n + phi_m)``
  with integer wave vectors ``1 <= |k_m|_inf <= kmax`` and phases drawn from
  one ``numpy.random.default_rng(seed)`` stream in a fixed order;
* density ``rho = rho0 (1 + drho * s / max|s|)``;
* velocity: each component its own random-phase sum, scaled so that
  ``max |u| = mach * c_s0`` with ``c_s0 = sqrt(gamma p0 / mean(rho))``;
* magnetic field ``B = delta x A``, the discrete centred curl of a
  random-phase vector potential (differences divided by the cell size
  1/max(n); 2-D: ``A = A_z``, plus an independent ``B_z``), so that the
  centred divergence of B vanishes to round-off and the field is the same at
  every resolution up to O(dx^2); scaled so that ``max |B|^2 = 2 p0 / beta``;
* uniform gas pressure ``p0``; total energy from the ideal-gas relation of
  the paper's EOS (sec. 2.3) solved for e_tot;
* lattice scaling (sec. 2.2, "Unit conversion"): with the CFL reading
  ``CFL = (max|u| + max c_f) dt / dx`` -- it reproduces the rotor's
  ``dt ~ 1.3e-6`` at N = 2000, CFL = 0.01 (sec. 3.2) -- the velocity scale is
  ``lam = (max|u| + max c_f) / CFL`` and ideal MHD is invariant under
  ``u -> u/lam, B -> B/lam, p -> p/lam^2, e_tot -> e_tot/lam^2`` (mu_0 = 1).

Field order of the conserved state (ideal MHD, 8 fields):
``rho, rho u_x, rho u_y, rho u_z, e_tot, B_x, B_y, B_z``.
Resistive incompressible state (7 fields): ``rho, m_x, m_y, m_z, B_x, B_y, B_z``.
Arrays are C-ordered ``[field, (z,) y, x]`` (x fastest), float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field

import numpy as np

IDEAL_FIELDS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz")
RESISTIVE_FIELDS = ("rho", "mx", "my", "mz", "Bx", "By", "Bz")


def _wavevectors(rng, dim: int, kmax: int, count: int):
    ks = []
    while len(ks) < count:
        k = rng.integers(-kmax, kmax + 1, size=dim)
        if np.abs(k).max() >= 1:
            ks.append(k)
    return ks


class _Backend:
    """Array operations for NumPy (host) or torch (device) field building."""

    def __init__(self, device=None):
        self.device = device
        if device is None:
            self.t = None
        else:
            import torch
            self.t = torch

    def coords(self, shape):
        """1-D coordinate vectors x/n, shaped to broadcast, ordered (x, y, z)."""
        dim = len(shape)
        out = []
        for a in range(dim):
            n = shape[dim - 1 - a]
            if self.t is None:
                v = np.arange(n, dtype=np.float64) / n
            else:
                v = self.t.arange(n, dtype=self.t.float64, device=self.device) / n
            view = [1] * dim
            view[dim - 1 - a] = n
            out.append(v.reshape(view))
        return out

    def zeros(self, shape):
        if self.t is None:
            return np.zeros(shape)
        return self.t.zeros(shape, dtype=self.t.float64, device=self.device)

    def cos(self, a):
        return np.cos(a) if self.t is None else self.t.cos(a)

    def sqrt(self, a):
        return np.sqrt(a) if self.t is None else self.t.sqrt(a)

    def roll(self, a, shift, axis):
        return np.roll(a, shift, axis=axis) if self.t is None else self.t.roll(a, shift, dims=axis)

    def amax(self, a) -> float:
        return float(np.abs(a).max()) if self.t is None else float(a.abs().max())

    def mean(self, a) -> float:
        return float(a.mean())

    def stack(self, xs):
        return np.stack(xs) if self.t is None else self.t.stack(xs)

    def full(self, shape, v):
        if self.t is None:
            return np.full(shape, v, dtype=np.float64)
        return self.t.full(shape, v, dtype=self.t.float64, device=self.device)


def random_phase(rng, shape, kmax: int, count: int, backend: _Backend = None):
    """Sum of ``count`` unit cosines with random integer wave vectors and phases."""
    be = backend or _Backend()
    dim = len(shape)
    coords = be.coords(shape)
    out = be.zeros(shape)
    for k in _wavevectors(rng, dim, kmax, count):
        phase = rng.uniform(0.0, 2.0 * math.pi)
        arg = phase
        for a in range(dim):
            arg = arg + (2.0 * math.pi * float(k[a])) * coords[a]
        out = out + be.cos(arg)
    return out


def _cdiff(a, axis_xyz: int, backend: _Backend = None):
    """Centred periodic difference along x (0), y (1) or z (2)."""
    be = backend or _Backend()
    ax = a.ndim - 1 - axis_xyz
    return 0.5 * (be.roll(a, -1, ax) - be.roll(a, 1, ax))


def centred_divergence(Bx, By, Bz=None) -> np.ndarray:
    div = _cdiff(Bx, 0) + _cdiff(By, 1)
    if Bz is not None and Bx.ndim == 3:
        div = div + _cdiff(Bz, 2)
    return div


def signal_speed(rho, u, p, B, gamma) -> float:
    """max|u| + max c_f over the grid, with c_f^2 = (gamma p + |B|^2)/rho.

    This is the velocity in the CFL reading ``CFL = (max|u| + max c_f) dt/dx``
    (``u`` and ``B`` have a leading component axis of length 3).
    """
    u = np.asarray(u, dtype=float)
    B = np.asarray(B, dtype=float)
    cf = np.sqrt((gamma * np.asarray(p, dtype=float) + (B * B).sum(0)) / np.asarray(rho, dtype=float))
    return float(np.sqrt((u * u).sum(0)).max() + cf.max())


@dataclass
class IdealFields:
    Q: object                # [8, (nz,) ny, nx] float64 (numpy, or torch on `device`), lattice units
    gamma: float
    lam: float               # physical velocity per lattice velocity
    mach: float
    beta: float
    cfl: float
    seed: int
    meta: dict = dc_field(default_factory=dict)


def ideal_fields(shape, seed: int, *, gamma: float = 5.0 / 3.0, mach: float = 1.0,
                 beta: float = 10.0 / 3.0, p0: float = 0.6, rho0: float = 1.0,
                 drho: float = 0.1, cfl: float = 0.1, k_rho: int = 3, k_u: int = 2,
                 k_b: int = 2, device=None) -> IdealFields:
    """Smooth random-phase ideal-MHD state, scaled to lattice units.

    2-D ``shape = (ny, nx)``, 3-D ``shape = (nz, ny, nx)``.  The defaults are
    the 128^2 workload (peak Mach 1, beta 10/3, CFL 0.1, gamma 5/3).  With
    ``device`` (a torch device) the same recipe runs on that device and
    ``Q`` is a torch float64 tensor; the seeded wave vectors and phases are
    identical, values agree with the host build to rounding.
    """
    be = _Backend(device)
    shape = tuple(int(n) for n in shape)
    dim = len(shape)
    rng = np.random.default_rng(seed)
    s = random_phase(rng, shape, k_rho, 4, be)
    rho = rho0 * (1.0 + drho * s / be.amax(s))
    del s
    u = [random_phase(rng, shape, k_u, 2, be) for _ in range(3)]
    # centred differences divided by one cell size for all axes, 1/max(n) (the
    # lattice is isotropic: one factor keeps the centred divergence exactly zero),
    # so that the curl approximates the same field at every resolution
    inv_h = float(max(shape))

    def d(a, axis):
        return _cdiff(a, axis, be) * inv_h

    if dim == 2:
        Az = random_phase(rng, shape, k_b, 3, be)
        B = [d(Az, 1), -d(Az, 0), random_phase(rng, shape, k_b, 2, be)]
        del Az
    else:
        A = [random_phase(rng, shape, k_b, 3, be) for _ in range(3)]
        B = [d(A[2], 1) - d(A[1], 2), d(A[0], 2) - d(A[2], 0), d(A[1], 0) - d(A[0], 1)]
        del A
    cs0 = math.sqrt(gamma * p0 / be.mean(rho))
    umag = be.sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
    su = mach * cs0 / be.amax(umag)
    del umag
    u = [c * su for c in u]
    if beta > 0:
        bmag2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
        sb = math.sqrt((2.0 * p0 / beta) / be.amax(bmag2))
        del bmag2
        B = [c * sb for c in B]
    else:
        B = [c * 0.0 for c in B]
    # lattice scaling from the CFL reading (max |u| + max fast speed), p uniform
    u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
    vmax = be.amax(be.sqrt(u2)) + be.amax(be.sqrt((gamma * p0 + B2) / rho))
    lam = vmax / cfl
    u = [c / lam for c in u]
    B = [c / lam for c in B]
    p = p0 / lam ** 2
    e = p / (gamma - 1.0) + 0.5 * rho * (u2 / lam ** 2) + 0.5 * (B2 / lam ** 2)
    del u2, B2
    Q = be.stack([rho, rho * u[0], rho * u[1], rho * u[2], e, B[0], B[1], B[2]])
    if be.t is None:
        Q = np.ascontiguousarray(Q, dtype=np.float64)
    else:
        Q = Q.contiguous()
    return IdealFields(Q=Q, gamma=gamma, lam=lam, mach=mach, beta=beta, cfl=cfl, seed=seed,
                       meta={"p0_lattice": p, "vmax_phys": vmax})


def uniform_ideal_state(shape, rho=1.0, u=(0.0, 0.0, 0.0), p=0.01, B=(0.0, 0.0, 0.0),
                        gamma=5.0 / 3.0) -> np.ndarray:
    """Spatially constant conserved state in lattice units."""
    u = np.asarray(u, dtype=float)
    B = np.asarray(B, dtype=float)
    e = p / (gamma - 1.0) + 0.5 * rho * float(u @ u) + 0.5 * float(B @ B)
    vals = [rho, rho * u[0], rho * u[1], rho * u[2], e, B[0], B[1], B[2]]
    return np.stack([np.full(tuple(shape), v, dtype=np.float64) for v in vals])


# ----------------------------------------------------------------------------
# resistive incompressible channel (Hartmann set-up)
# ----------------------------------------------------------------------------

@dataclass
class HartmannSetup:
    Q: np.ndarray            # [7, nz, ny, nx]
    tau_f: float
    tau_m: float
    nu: float
    eta: float
    force: tuple
    b_wall: tuple
    B0: float
    Ha: float
    a: float
    U_c: float


def hartmann_profile(y, a, F, rho, nu, eta, B0):
    """Closed-form steady Hartmann flow with insulating walls at y = +-a.

    Returns (u_x(y), b_x(y)) with y measured from the channel centre.  From
    rho nu u'' + B0 b' + F = 0 and B0 u' + eta b'' = 0 with u(+-a) = b(+-a) = 0.
    """
    y = np.asarray(y, dtype=float)
    if B0 == 0.0:
        return F / (2.0 * rho * nu) * (a * a - y * y), np.zeros_like(y)
    Ha = B0 * a / math.sqrt(rho * nu * eta)
    u = F * a * a / (rho * nu * Ha * math.tanh(Ha)) * (1.0 - np.cosh(Ha * y / a) / math.cosh(Ha))
    K = F * a * a / (rho * nu * Ha * math.sinh(Ha))
    b = B0 * K * a / (eta * Ha) * (np.sinh(Ha * y / a) - (y / a) * math.sinh(Ha))
    return u, b


def hartmann_setup(shape, seed: int, *, Ha: float = 10.0, U_c: float = 0.05, Re: float = 100.0,
                   Pm: float = 1.0, noise: float = 0.01, rho0: float = 1.0) -> HartmannSetup:
    """Channel ``shape = (nz, ny, nx)`` with solid rows y = 0 and ny - 1.

    Half-width a = (ny - 2)/2 (halfway walls), nu = U_c a / Re, eta = nu / Pm,
    tau_f = 1/2 + 3 nu (D3Q19), tau_m = 1/2 + 4 eta (D3Q7),
    B0 = Ha sqrt(rho nu eta) / a along y, body force F_x chosen so that the
    closed-form centreline speed is U_c.  Initial velocity: uniform noise of
    relative size ``noise`` (times U_c) per component in the fluid rows.
    """
    nz, ny, nx = (int(n) for n in shape)
    a = (ny - 2) / 2.0
    nu = U_c * a / Re
    eta = nu / Pm
    tau_f = 0.5 + 3.0 * nu
    tau_m = 0.5 + 4.0 * eta
    B0 = Ha * math.sqrt(rho0 * nu * eta) / a
    if Ha > 0:
        F = U_c * rho0 * nu * Ha * math.tanh(Ha) / (a * a * (1.0 - 1.0 / math.cosh(Ha)))
    else:
        F = U_c * 2.0 * rho0 * nu / (a * a)
    rng = np.random.default_rng(seed)
    Q = np.zeros((7, nz, ny, nx))
    Q[0] = rho0
    Q[1:4] = rho0 * noise * U_c * rng.uniform(-1.0, 1.0, size=(3, nz, ny, nx))
    Q[5] = B0
    Q[1:4, :, 0, :] = 0.0
    Q[1:4, :, ny - 1, :] = 0.0
    return HartmannSetup(Q=np.ascontiguousarray(Q), tau_f=tau_f, tau_m=tau_m, nu=nu, eta=eta,
                         force=(F, 0.0, 0.0), b_wall=(0.0, B0, 0.0), B0=B0, Ha=Ha, a=a, U_c=U_c)


# ----------------------------------------------------------------------------
# batch of independent 2-D domains
# ----------------------------------------------------------------------------

BATCH_SIDES = (64, 128, 256, 512, 1024)


def batch_specs(count: int = 64, seed: int = 4004, sides=BATCH_SIDES):
    """Per-domain (side, gamma, mach, seed) drawn from one seeded stream."""
    rng = np.random.default_rng(seed)
    specs = []
    for d in range(count):
        side = int(rng.choice(np.asarray(sides)))
        gamma = float(rng.uniform(1.4, 5.0 / 3.0))
        mach = float(rng.uniform(0.5, 3.0))
        specs.append({"side": side, "gamma": gamma, "mach": mach, "seed": seed + d})
    return specs


# ----------------------------------------------------------------------------
# dissipative MHD with evolved gradients (low-Mach Orszag-Tang set-up)
# ----------------------------------------------------------------------------

DISSIPATIVE_FIELDS = IDEAL_FIELDS + tuple("G%s%s" % (a, b) for a in "xy" for b in "xyz") + \
    tuple("W%s%s" % (a, b) for a in "xy" for b in "xyz")


@dataclass
class DissipativeSetup:
    Q: np.ndarray            # [20, ny, nx]: the 8 MHD fields, G_ab at 8 + 3a + b, W_ab at 14 + 3a + b
    gamma: float
    tau: float               # BGK time of the eight MHD lattices
    tau_g: float             # BGK time of the twelve gradient lattices
    tau_m: float             # relaxation time of G and W, in steps
    nu: float                # kinematic viscosity, lattice units
    eta0: float              # resistivity at zero current, lattice units
    j_c: float               # current scale of eta(j), lattice units
    dx: float                # physical cell size
    dt: float                # physical time per step


def low_mach_orszag_tang(n: int, *, u_lat: float = 0.02, mach: float = 0.1, gamma: float = 5.0 / 3.0,
                         nu_phys: float = 1e-3, jc_phys: float = 25.0, tau_m_phys: float = 0.01,
                         stab: float = 0.05) -> DissipativeSetup:
    """The low-Mach resistive Orszag-Tang vortex (sec. 3.3, "Low compressible
    resistive Orszag-Tang vortex") on an n x n grid of
    the periodic box [0, 2 pi)^2, in lattice units.

    Physical state: rho = 1, u = (2 cos y, -2 sin x, 0), B = (-2 sin 2y, -2 sin x, 0),
    kinematic viscosity nu_phys, eta0 = nu, j_c = 25, relaxation time of the
    gradient tensors tau_M = 0.01, lattice diffusion ("stabilisation") stab * nu.
    Scaling: velocities and fields by s = u_lat / 2 (so the peak speed component
    is u_lat), dx = 2 pi / n, dt = s dx, uniform pressure from the sound speed
    u_lat / mach.  G and W start at their relaxed values tau_M grad B,
    tau_M grad u (analytic gradients of the profiles, scaled to the lattice).
    """
    n = int(n)
    s = 0.5 * u_lat
    dx = 2.0 * math.pi / n
    dt = s * dx
    x = dx * np.arange(n)[None, :]
    y = dx * np.arange(n)[:, None]
    one = np.ones((n, n))
    ux, uy = s * 2.0 * np.cos(y) * one, -s * 2.0 * np.sin(x) * one
    Bx, By = -s * 2.0 * np.sin(2.0 * y) * one, -s * 2.0 * np.sin(x) * one
    c = u_lat / mach
    p = c * c / gamma  # rho = 1
    nu = nu_phys * s / dx
    tau_m = tau_m_phys / dt
    g = tau_m * s * dx  # tau_M times the lattice derivative of a physical derivative
    Q = np.zeros((20, n, n))
    Q[0] = 1.0
    Q[1], Q[2] = ux, uy
    Q[4] = p / (gamma - 1.0) + 0.5 * (ux * ux + uy * uy) + 0.5 * (Bx * Bx + By * By)
    Q[5], Q[6] = Bx, By
    # G_ab = tau_M d_a B_b:  d_x B_y = -2 cos x,  d_y B_x = -4 cos 2y
    Q[8 + 1] = g * (-2.0 * np.cos(x)) * one
    Q[8 + 3] = g * (-4.0 * np.cos(2.0 * y)) * one
    # W_ab = tau_M d_a u_b:  d_x u_y = -2 cos x,  d_y u_x = -2 sin y
    Q[14 + 1] = g * (-2.0 * np.cos(x)) * one
    Q[14 + 3] = g * (-2.0 * np.sin(y)) * one
    tau = 0.5 + 3.0 * stab * nu  # (tau - 1/2) cs^2 = stab * nu on D2Q5
    return DissipativeSetup(Q=np.ascontiguousarray(Q), gamma=gamma, tau=tau, tau_g=tau, tau_m=tau_m, nu=nu,
                            eta0=nu, j_c=jc_phys * s * dx, dx=dx, dt=dt)


DISSIPATIVE3_FIELDS = IDEAL_FIELDS + tuple("G%s%s" % (a, b) for a in "xyz" for b in "xyz") + \
    tuple("W%s%s" % (a, b) for a in "xyz" for b in "xyz")


def low_mach_vortex_3d(n: int, *, u_lat: float = 0.02, mach: float = 0.1, gamma: float = 5.0 / 3.0,
                       nu_phys: float = 1e-3, jc_phys: float = 25.0, tau_m_phys: float = 0.01,
                       stab: float = 0.05) -> DissipativeSetup:
    """A 3-D companion of the low-Mach resistive Orszag-Tang set-up for the
    26-lattice D3Q7 form, on an n^3 grid of the periodic box [0, 2 pi)^3, in
    lattice units (same scalings, viscosity, resistivity and tau_M as
    low_mach_orszag_tang; a synthetic workload, the paper's dissipative case is
    2-D).  Physical state: rho = 1,
        u = (2 cos y + cos z, -2 sin x + sin z, sin x + cos y),
        B = (-2 sin 2y + sin z, -2 sin x + cos z, cos x + sin 2y),
    both free of divergence (no component depends on its own coordinate).
    Scaling by s = u_lat / 3 (the peak of a velocity component), dx = 2 pi / n,
    dt = s dx, uniform pressure from the sound speed u_lat / mach.  G_ab and W_ab
    (at 8 + 3a + b and 17 + 3a + b) start at tau_M times the analytic gradients."""
    n = int(n)
    s = u_lat / 3.0
    dx = 2.0 * math.pi / n
    dt = s * dx
    ax = dx * np.arange(n)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    u = [s * (2.0 * np.cos(y) + np.cos(z)), s * (-2.0 * np.sin(x) + np.sin(z)), s * (np.sin(x) + np.cos(y))]
    B = [s * (-2.0 * np.sin(2.0 * y) + np.sin(z)), s * (-2.0 * np.sin(x) + np.cos(z)),
         s * (np.cos(x) + np.sin(2.0 * y))]
    # physical gradients d_a u_b and d_a B_b (rows a = x, y, z)
    zero = np.zeros_like(x)
    du = [[zero, -2.0 * np.cos(x), np.cos(x)],
          [-2.0 * np.sin(y), zero, -np.sin(y)],
          [-np.sin(z), np.cos(z), zero]]
    dB = [[zero, -2.0 * np.cos(x), -np.sin(x)],
          [-4.0 * np.cos(2.0 * y), zero, 2.0 * np.cos(2.0 * y)],
          [np.cos(z), -np.sin(z), zero]]
    c = u_lat / mach
    p = c * c / gamma  # rho = 1
    nu = nu_phys * s / dx
    tau_m = tau_m_phys / dt
    g = tau_m * s * dx  # tau_M times the lattice derivative of a physical derivative
    Q = np.zeros((26, n, n, n))
    Q[0] = 1.0
    for b in range(3):
        Q[1 + b] = u[b]
        Q[5 + b] = B[b]
    Q[4] = p / (gamma - 1.0) + 0.5 * sum(v * v for v in u) + 0.5 * sum(v * v for v in B)
    for a in range(3):
        for b in range(3):
            Q[8 + 3 * a + b] = g * dB[a][b]
            Q[17 + 3 * a + b] = g * du[a][b]
    tau = 0.5 + 4.0 * stab * nu  # (tau - 1/2) cs^2 = stab * nu on D3Q7 (cs^2 = 1/4)
    return DissipativeSetup(Q=np.ascontiguousarray(Q), gamma=gamma, tau=tau, tau_g=tau, tau_m=tau_m, nu=nu,
                            eta0=nu, j_c=jc_phys * s * dx, dx=dx, dt=dt)
