"""Pins of the oracle's static equilibrium boundaries (sec. 2.4, "Static boundaries").

On an open face every state variable is Dirichlet (a set value) or Neumann (the
value of the next cell along the discrete normal), and the equilibrium of that
boundary state is assigned to the direction entering the domain.  Checked
against: a uniform state as an exact fixed point, exact agreement with the
periodic run until a disturbance reaches the faces (light cone), a supersonic
inflow that flushes the domain to the inflow state, a pulse that leaves through
zero-gradient faces, and the independent NumPy restatement.
"""
import numpy as np
import pytest

import oracle
from oracle import numpy_ref as R
from paper_2606_00641_gb300 import fields

GAMMA = 5.0 / 3.0
ALL = 0xFF


def _state(rho, u, p, B):
    Q = np.zeros(8)
    Q[0] = rho
    Q[1:4] = rho * np.asarray(u, dtype=float)
    Q[5:8] = B
    Q[4] = p / (GAMMA - 1) + 0.5 * rho * np.dot(u, u) + 0.5 * np.dot(B, B)
    return Q


def _uniform(Q, shape):
    return np.broadcast_to(Q.reshape((8,) + (1,) * len(shape)), (8,) + tuple(shape)).copy()


BG = _state(1.0, [0.05, -0.03, 0.02], 0.02, [0.04, 0.03, -0.02])


@pytest.mark.parametrize("shape,faces", [
    ((12, 16), [(ALL, BG), (0, None), (0b10110, BG), (0b01001, BG)]),
    ((6, 7, 8), [(0, None), (ALL, BG), (0b1100, BG), (0, None), (0b10000001, BG), (0, None)]),
])
def test_uniform_state_is_a_fixed_point(shape, faces):
    # Dirichlet values equal to the state, Neumann copies of it: every entering
    # population is the one the uniform state already carries
    Q = _uniform(BG, shape)
    out = oracle.open_run(Q, GAMMA, 0.6, faces, 40)
    assert np.abs(out - Q).max() < 1e-14 * np.abs(BG).max()


def _compact_bump(shape, centre, radius):
    grids = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    r = np.sqrt(sum((g - c) ** 2 for g, c in zip(grids, centre)))
    return np.where(r < radius, np.cos(0.5 * np.pi * r / radius) ** 2, 0.0)


@pytest.mark.parametrize("shape,faces,steps", [
    ((40, 40), [(ALL, BG), (0, None), (0b10110, BG), (0b01001, BG)], 12),
    ((24, 24, 24), [(0, None), (ALL, BG), (0b1100, BG), (0, None), (0b10000001, BG), (0, None)], 5),
])
def test_open_run_equals_the_periodic_run_inside_the_light_cone(shape, faces, steps):
    # A disturbance of radius 4 at the centre of a uniform moving, magnetised
    # background reaches at most 4 + steps cells; the boundary state is built from
    # the cells next to the faces, which stay at the background, so every entering
    # population equals the one the periodic run brings in (the background's
    # equilibrium) and the two runs agree everywhere
    centre = [0.5 * n for n in shape]
    b = _compact_bump(shape, centre, 4.0)
    assert 4 + steps + 1 < min(shape) / 2 - 1
    Q = _uniform(BG, shape)
    Q[0] += 0.05 * b
    Q[4] += 0.05 * b * 0.02 / (GAMMA - 1)
    Q[6] += 0.01 * b
    got = oracle.open_run(Q, GAMMA, 0.6, faces, steps)
    ref = oracle.ideal_run(Q, GAMMA, 0.6, steps)
    scale = np.abs(Q).reshape(8, -1).max(1)
    assert (np.abs(got - ref).reshape(8, -1).max(1) / scale).max() < 1e-13
    # and the disturbance did move (the comparison is not between two copies of Q)
    assert np.abs(ref - Q).max() > 1e-4


def test_supersonic_inflow_flushes_the_domain_to_the_inflow_state():
    # u = 0.2 along x with fast speed 0.107: every characteristic enters at x- and
    # leaves at x+, so a Dirichlet inflow and a zero-gradient outflow wash any
    # disturbance out and the domain converges to the inflow state
    Qin = _state(1.0, [0.2, 0.02, 0.0], 0.006, [0.03, 0.02, 0.01])
    shape = (4, 48)
    Q = _uniform(Qin, shape)
    x = np.arange(48)
    bump = 0.02 * np.exp(-((x - 20) / 4.0) ** 2)
    Q[0] += bump
    Q[4] += bump * 0.006 / (GAMMA - 1)
    faces = [(ALL, Qin), (0, None)]
    out = oracle.open_run(Q, GAMMA, 0.7, faces, 1200)
    assert np.abs(out - Qin.reshape(8, 1, 1)).max() < 1e-12


def test_zero_gradient_faces_let_a_pulse_leave():
    # a pressure pulse in gas at rest spreads as a fast wave; with zero-gradient
    # faces it leaves the 64^2 box, with periodic faces it keeps crossing it:
    # after 400 steps the open box holds a few percent of the periodic box's
    # deviation energy (a reversed or misplaced fill would reflect or inject it)
    bg = _state(1.0, [0.0, 0.0, 0.0], 0.02, [0.05, 0.0, 0.0])
    n = 64
    yy, xx = np.mgrid[0:n, 0:n]
    g = 0.01 * np.exp(-((xx - 31.5) ** 2 + (yy - 31.5) ** 2) / 16.0)
    Q = _uniform(bg, (n, n))
    Q[0] += g
    Q[4] += g * GAMMA * 0.02 / (GAMMA - 1)
    zero_gradient = [(0, None)] * 4
    opened = oracle.open_run(Q, GAMMA, 0.6, zero_gradient, 400, nthreads=4)
    periodic = oracle.ideal_run(Q, GAMMA, 0.6, 400, nthreads=4)
    e_open = ((opened - bg.reshape(8, 1, 1)) ** 2).sum()
    e_per = ((periodic - bg.reshape(8, 1, 1)) ** 2).sum()
    assert e_open < 0.05 * e_per, (e_open, e_per)


@pytest.mark.parametrize("shape", [(10, 12), (5, 6, 7)])
def test_oracle_matches_numpy_restatement(shape):
    # random smooth fields, both / all axes open, each face with its own mix of
    # Dirichlet and Neumann variables (edges and corners take the diagonal normal)
    f0 = fields.ideal_fields(shape, 7, mach=0.8, beta=1.0, cfl=0.2)
    v1 = f0.Q.reshape(8, -1).mean(1)
    v2 = f0.Q.reshape(8, -1)[:, 3]
    faces = [(0b10011, v1), (ALL, v2), (0, None), (0b100000, v1), (0b1001, v2), (0, None)][:2 * len(shape)]
    a = oracle.open_run(f0.Q, f0.gamma, 0.6, faces, 15)
    b = R.open_run(f0.Q, f0.gamma, 0.6, faces, 15)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


def test_face_specification_is_checked():
    Q = _uniform(BG, (6, 8))
    with pytest.raises(ValueError):
        oracle.open_run(Q, GAMMA, 0.6, [(0, None), None], 1)  # one face of an axis open
    with pytest.raises(Exception):
        oracle.open_run(_uniform(BG, (2, 8)), GAMMA, 0.6, [None, None, (0, None), (0, None)], 1)  # < 3 cells


def test_solids_inside_an_open_domain():
    # a homogenised body at the centre of the light-cone setup: the open run equals
    # the periodic run with the same body; with d = 1 everywhere it is the plain open run
    shape = (40, 40)
    faces = [(ALL, BG), (0, None), (0b10110, BG), (0b01001, BG)]
    yy, xx = np.mgrid[0:40, 0:40]
    phi = np.hypot(xx - 20.0, yy - 20.0) - 3.0
    solid = np.zeros((7,) + shape)
    solid[0] = oracle.hlbm_porosity(phi, 1.0)
    solid[1], solid[2] = 0.01, -0.02
    solid[4], solid[6] = 0.02, 0.01
    Q = _uniform(BG, shape)
    got = oracle.open_run(Q, GAMMA, 0.6, faces, 10, solid=solid)
    ref = oracle.hlbm_run(Q, GAMMA, 0.6, solid, 10)
    scale = np.abs(Q).reshape(8, -1).max(1)
    assert (np.abs(got - ref).reshape(8, -1).max(1) / scale).max() < 1e-13
    assert np.abs(ref - Q).max() > 1e-4
    fluid = solid.copy()
    fluid[0] = 1.0
    f0 = fields.ideal_fields(shape, 9, mach=0.8, beta=1.0, cfl=0.2)
    a = oracle.open_run(f0.Q, f0.gamma, 0.6, faces, 8, solid=fluid)
    b = oracle.open_run(f0.Q, f0.gamma, 0.6, faces, 8)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def test_update_is_symmetric_under_the_mirror_that_swaps_the_x_faces():
    # x -> nx - 1 - x swaps the x- and x+ faces; rho u turns as a vector (its x component
    # flips) and B as a pseudovector (B_y, B_z flip), Dirichlet values with the state and the
    # masks unchanged: the mirrored run with mirrored faces is the mirror of the run
    def mirror(S):
        M = S[..., ::-1].copy()
        for k in (1, 6, 7):
            M[k] *= -1
        return M

    f0 = fields.ideal_fields((14, 18), 666, mach=0.5, beta=1.0, cfl=0.2)
    Q = f0.Q
    inflow = Q[:, 5, 0].copy()
    inflow[1] = abs(inflow[1]) + 0.02 * Q[0, 5, 0]     # a state entering through x-
    faces = [(0b10110, inflow), (0, None)]               # mixed Dirichlet / Neumann, then Neumann
    mirrored = [(0, None), (0b10110, mirror(inflow[:, None])[:, 0])]
    a = mirror(oracle.open_run(Q, f0.gamma, 0.6, faces, 9))
    b = oracle.open_run(mirror(Q), f0.gamma, 0.6, mirrored, 9)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    assert np.abs(mirror(Q) - Q).max() > 1e-3
