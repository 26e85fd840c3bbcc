"""Independent NumPy restatement of the VLBM step for tiny grids.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  It restates the same
paper passages as ``vlbm_oracle.c`` in a different style (whole-array
algebra, ``np.roll`` streaming, primitive variables first) so that a coding
slip in either statement shows up as a disagreement on small grids:

* Eq. 2  -- BGK collision, direct source injection, streaming x -> x + c_i;
* Eq. 3  -- f_eq = w_i (Q_k + c_i . Phi_k / cs^2);
* Eq. 4  -- Q_k = sum_i f_ki;
* Eq. 9  -- p = (gamma - 1)(e_tot - rho|u|^2/2 - |B|^2/2);
* Eq. 12 -- ideal MHD flux.

The resistive model (D3Q19 + three D3Q7 magnetic lattices, Guo force,
halfway bounce-back, equilibrium magnetic walls) follows the same reading
as the C oracle.  Arrays use the layout [field, direction, (z,) y, x].
"""
from __future__ import annotations

import numpy as np


def _axis_dirs(dim: int):
    dirs = [(0, 0, 0)]
    for a in range(dim):
        e = [0, 0, 0]
        e[a] = 1
        dirs.append(tuple(e))
        dirs.append(tuple(-v for v in e))
    return np.array(dirs, dtype=int)


def vset(name: str):
    """Velocities, weights and cs^2 written out from the quadrature conditions."""
    if name == "D2Q5":
        c = _axis_dirs(2)
        w = np.array([1 / 3] + [1 / 6] * 4)
        return c, w, 1 / 3
    if name == "D3Q7":
        c = _axis_dirs(3)
        w = np.array([1 / 4] + [1 / 8] * 6)
        return c, w, 1 / 4
    if name == "D3Q19":
        c = list(_axis_dirs(3))
        for (a, b) in ((0, 1), (0, 2), (1, 2)):
            for (sa, sb) in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
                e = [0, 0, 0]
                e[a], e[b] = sa, sb
                c.append(np.array(e))
        w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
        return np.array(c, dtype=int), w, 1 / 3
    raise ValueError(name)


def _shift(a: np.ndarray, c, dim: int) -> np.ndarray:
    """Value at x moves to x + c (periodic).  Array axes are (z,) y, x."""
    out = a
    for ax in range(dim):
        if c[ax]:
            out = np.roll(out, c[ax], axis=a.ndim - 1 - ax)
    return out


def primitives(Q: np.ndarray, gamma: float):
    rho = Q[0]
    u = Q[1:4] / rho
    e = Q[4]
    B = Q[5:8]
    p = (gamma - 1.0) * (e - 0.5 * rho * (u * u).sum(0) - 0.5 * (B * B).sum(0))
    return rho, u, e, B, p


def ideal_flux(Q: np.ndarray, gamma: float) -> np.ndarray:
    """Phi[k, a, ...]: Eq. 12 assembled from primitive variables."""
    rho, u, e, B, p = primitives(Q, gamma)
    pt = p + 0.5 * (B * B).sum(0)
    phi = np.zeros((8, 3) + Q.shape[1:])
    phi[0] = rho * u
    for b in range(3):
        for a in range(3):
            phi[1 + b, a] = rho * u[a] * u[b] - B[a] * B[b] + (pt if a == b else 0.0)
            phi[5 + b, a] = u[a] * B[b] - B[a] * u[b]
    phi[4] = (e + pt) * u - B * (u * B).sum(0)
    return phi


def ideal_feq(Q: np.ndarray, gamma: float, dim: int) -> np.ndarray:
    c, w, cs2 = vset("D2Q5" if dim == 2 else "D3Q7")
    phi = ideal_flux(Q, gamma)
    feq = np.zeros((8, len(w)) + Q.shape[1:])
    for i in range(len(w)):
        cphi = sum(c[i, a] * phi[:, a] for a in range(3))
        feq[:, i] = w[i] * (Q + cphi / cs2)
    return feq


def ideal_step(f: np.ndarray, gamma: float, tau, dim: int, src=None) -> np.ndarray:
    c, w, _ = vset("D2Q5" if dim == 2 else "D3Q7")
    Q = f.sum(axis=1)
    feq = ideal_feq(Q, gamma, dim)
    tau = np.broadcast_to(np.asarray(tau, dtype=float), (8,))
    post = f + (feq - f) / tau[:, None].reshape((8, 1) + (1,) * (f.ndim - 2))
    if src is not None:
        s = np.asarray(src, dtype=float)
        post = post + w[None, :].reshape((1, len(w)) + (1,) * (f.ndim - 2)) * \
            s.reshape((8, 1) + (1,) * (f.ndim - 2))
    out = np.empty_like(f)
    for i in range(len(w)):
        out[:, i] = _shift(post[:, i], c[i], dim)
    return out


def ideal_run(Q0: np.ndarray, gamma: float, tau, nsteps: int, src=None) -> np.ndarray:
    dim = Q0.ndim - 1
    f = ideal_feq(Q0, gamma, dim)
    for _ in range(nsteps):
        f = ideal_step(f, gamma, tau, dim, src)
    return f.sum(axis=1)


def open_step(f: np.ndarray, gamma: float, tau, dim: int, faces, src=None) -> np.ndarray:
    """Static equilibrium boundaries (sec. 2.4): periodic streaming, then on every
    open face the direction entering across it is overwritten with the equilibrium
    of the boundary state (Dirichlet values where the mask bit is set, else the
    streamed moments of the cell one step along the discrete inward normal).
    faces[2a], faces[2a+1]: None (periodic) or (mask, values) for axis a's low and high face."""
    c, w, _ = vset("D2Q5" if dim == 2 else "D3Q7")
    out = ideal_step(f, gamma, tau, dim, src)
    shape = f.shape[2:]
    faces = list(faces) + [None] * (6 - len(faces))
    pos = np.indices(shape)  # pos[j] indexes array axis j, i.e. lattice axis dim - 1 - j
    size = [shape[dim - 1 - a] for a in range(dim)]
    coord = [pos[dim - 1 - a] for a in range(dim)]
    normal = [np.zeros(shape, dtype=int) for _ in range(dim)]
    for a in range(dim):
        if faces[2 * a] is not None:
            normal[a] = np.where(coord[a] == 0, 1, np.where(coord[a] == size[a] - 1, -1, 0))
    nb_index = tuple(coord[a] + normal[a] for a in range(dim))[::-1]
    Qs = out.sum(axis=1)
    Qn = Qs[(slice(None),) + nb_index]
    for a in range(dim):
        for side in (0, 1):
            spec = faces[2 * a + side]
            if spec is None:
                continue
            mask, vals = spec
            vals = np.zeros(8) if vals is None else np.asarray(vals, dtype=float)
            on = coord[a] == (0 if side == 0 else size[a] - 1)
            Qb = np.array([np.full(shape, vals[k]) if (int(mask) >> k) & 1 else Qn[k] for k in range(8)])
            feq = ideal_feq(Qb, gamma, dim)
            e = np.zeros(3, dtype=int)
            e[a] = 1 if side == 0 else -1
            din = [i for i in range(len(w)) if tuple(c[i]) == tuple(e[:c.shape[1]])][0]
            for k in range(8):
                out[k, din][on] = feq[k, din][on]
    return out


def open_run(Q0: np.ndarray, gamma: float, tau, faces, nsteps: int, src=None) -> np.ndarray:
    dim = Q0.ndim - 1
    f = ideal_feq(Q0, gamma, dim)
    for _ in range(nsteps):
        f = open_step(f, gamma, tau, dim, faces, src)
    return f.sum(axis=1)


# ----------------------------------------------------------------------------
# ideal MHD with the Powell correction (sec. 2.3): a ninth lattice carries
# D = tr G (sec. 2.2.1) with flux D u - B and source -D / tau_M; the other
# lattices receive S = -(D / tau_M) (0, B, u.B, u)
# ----------------------------------------------------------------------------

def powell_flux(Q: np.ndarray, gamma: float) -> np.ndarray:
    """phi[9, 3, ...] for Q[9, ...]."""
    rho, u, e, B, p = primitives(Q[:8], gamma)
    phi = np.zeros((9, 3) + Q.shape[1:])
    phi[:8] = ideal_flux(Q[:8], gamma)
    for a in range(3):
        phi[8, a] = Q[8] * u[a] - B[a]
    return phi


def powell_source(Q: np.ndarray, tau_m: float) -> np.ndarray:
    u = Q[1:4] / Q[0]
    B = Q[5:8]
    divB = Q[8] / tau_m
    S = np.zeros_like(Q)
    uB = (u * B).sum(0)
    for b in range(3):
        S[1 + b] = -divB * B[b]
        S[5 + b] = -divB * u[b]
    S[4] = -divB * uB
    S[8] = -Q[8] / tau_m
    return S


def powell_feq(Q: np.ndarray, gamma: float, dim: int) -> np.ndarray:
    c, w, cs2 = vset("D2Q5" if dim == 2 else "D3Q7")
    phi = powell_flux(Q, gamma)
    feq = np.zeros((9, len(w)) + Q.shape[1:])
    for i in range(len(w)):
        cphi = sum(c[i, a] * phi[:, a] for a in range(3))
        feq[:, i] = w[i] * (Q + cphi / cs2)
    return feq


def powell_step(f: np.ndarray, gamma: float, tau, tau_m: float, dim: int) -> np.ndarray:
    c, w, _ = vset("D2Q5" if dim == 2 else "D3Q7")
    Q = f.sum(axis=1)
    feq = powell_feq(Q, gamma, dim)
    S = powell_source(Q, tau_m)
    tau = np.broadcast_to(np.asarray(tau, dtype=float), (9,))
    shape1 = (9, 1) + (1,) * (f.ndim - 2)
    post = f + (feq - f) / tau.reshape(shape1)
    for i in range(len(w)):
        post[:, i] += w[i] * S
    out = np.empty_like(f)
    for i in range(len(w)):
        out[:, i] = _shift(post[:, i], c[i], dim)
    return out


def powell_run(Q0: np.ndarray, gamma: float, tau, tau_m: float, nsteps: int) -> np.ndarray:
    dim = Q0.ndim - 1
    f = powell_feq(Q0, gamma, dim)
    for _ in range(nsteps):
        f = powell_step(f, gamma, tau, tau_m, dim)
    return f.sum(axis=1)


# ----------------------------------------------------------------------------
# homogenised solids (HLBM, sec. 2.4): u and B blended with the solid's by the
# porosity d before the equilibrium; rho and the gas pressure kept
# ----------------------------------------------------------------------------

def hlbm_step(f: np.ndarray, gamma: float, tau, solid: np.ndarray, dim: int, src=None) -> np.ndarray:
    c, w, _ = vset("D2Q5" if dim == 2 else "D3Q7")
    Q = f.sum(axis=1)
    rho, u, e, B, p = primitives(Q, gamma)
    d = solid[0]
    uh = d * u + (1.0 - d) * solid[1:4]
    Bh = d * B + (1.0 - d) * solid[4:7]
    Qh = np.empty_like(Q)
    Qh[0] = rho
    Qh[1:4] = rho * uh
    Qh[5:8] = Bh
    Qh[4] = p / (gamma - 1.0) + 0.5 * rho * (uh * uh).sum(0) + 0.5 * (Bh * Bh).sum(0)
    feq = ideal_feq(Qh, gamma, dim)
    tau = np.broadcast_to(np.asarray(tau, dtype=float), (8,))
    shape1 = (8, 1) + (1,) * (f.ndim - 2)
    post = f + (feq - f) / tau.reshape(shape1)
    if src is not None:
        s = np.asarray(src, dtype=float)
        for i in range(len(w)):
            post[:, i] += w[i] * s.reshape((8,) + (1,) * (f.ndim - 2))
    out = np.empty_like(f)
    for i in range(len(w)):
        out[:, i] = _shift(post[:, i], c[i], dim)
    return out


def hlbm_run(Q0: np.ndarray, gamma: float, tau, solid: np.ndarray, nsteps: int, src=None) -> np.ndarray:
    dim = Q0.ndim - 1
    f = ideal_feq(Q0, gamma, dim)
    for _ in range(nsteps):
        f = hlbm_step(f, gamma, tau, solid, dim, src)
    return f.sum(axis=1)


# ----------------------------------------------------------------------------
# resistive incompressible reading: D3Q19 flow + three D3Q7 B lattices
# ----------------------------------------------------------------------------

def _flow_feq(rho, j, B):
    c, w, cs2 = vset("D3Q19")
    u = j / rho
    B2 = (B * B).sum(0)
    feq = np.zeros((19,) + rho.shape)
    for i in range(19):
        cu = sum(c[i, a] * u[a] for a in range(3))
        cB = sum(c[i, a] * B[a] for a in range(3))
        c2 = float((c[i] * c[i]).sum())
        uu = (u * u).sum(0)
        # (c c - cs2 I) : (rho u u + B^2/2 I - B B)
        second = rho * (cu * cu - cs2 * uu) + 0.5 * B2 * (c2 - 3 * cs2) - (cB * cB - cs2 * B2)
        feq[i] = w[i] * (rho + rho * cu / cs2 + second / (2 * cs2 * cs2))
    return feq


def _mag_feq(u, B):
    c, w, cs2 = vset("D3Q7")
    geq = np.zeros((3, 7) + B.shape[1:])
    for b in range(3):
        for i in range(7):
            cphi = sum(c[i, a] * (u[a] * B[b] - B[a] * u[b]) for a in range(3))
            geq[b, i] = w[i] * (B[b] + cphi / cs2)
    return geq


def resistive_init(Q0, force):
    rho = Q0[0]
    m = Q0[1:4]
    B = Q0[4:7]
    F = np.asarray(force, dtype=float).reshape(3, 1, 1, 1)
    f = _flow_feq(rho, m - 0.5 * F, B)
    g = _mag_feq(m / rho, B)
    return f, g


def resistive_step(f, g, tau_f, tau_m, force, b_wall, walls_y):
    c19, w19, cs2 = vset("D3Q19")
    c7, w7, _ = vset("D3Q7")
    F = np.asarray(force, dtype=float).reshape(3, 1, 1, 1)
    ny = f.shape[2]
    wall = np.zeros(f.shape[1:], dtype=bool)
    if walls_y:
        wall[:, 0, :] = True
        wall[:, ny - 1, :] = True
    rho = f.sum(0)
    j = np.stack([sum(c19[i, a] * f[i] for i in range(19)) for a in range(3)])
    m = j + 0.5 * F
    u = m / rho
    B = g.sum(1)
    feq = _flow_feq(rho, m, B)
    geq = _mag_feq(u, B)
    fo = f.copy()
    go = g.copy()
    for i in range(19):
        cu = sum(c19[i, a] * u[a] for a in range(3))
        cF = sum(c19[i, a] * F[a] for a in range(3))
        uF = (u * F).sum(0)
        guo = (1 - 0.5 / tau_f) * w19[i] * ((cF - uF) / cs2 + cu * cF / cs2 ** 2)
        post = f[i] - (f[i] - feq[i]) / tau_f + guo
        # a population whose destination is a wall returns in the opposite direction
        dest_wall = _shift(wall, -c19[i], 3)  # dest_wall[x] = wall[x + c_i]
        opp = [k for k in range(19) if (c19[k] == -c19[i]).all()][0]
        moved = _shift(np.where(wall | dest_wall, np.nan, post), c19[i], 3)
        keep = ~np.isnan(moved)
        fo[i] = np.where(keep, moved, fo[i])
        fo[opp] = np.where(dest_wall & ~wall, post, fo[opp])
    for b in range(3):
        for i in range(7):
            post = np.where(wall, w7[i] * b_wall[b], g[b, i] - (g[b, i] - geq[b, i]) / tau_m)
            go[b, i] = _shift(post, c7[i], 3)
    return fo, go


def resistive_moments(f, g, force, b_wall, walls_y):
    c19, _, _ = vset("D3Q19")
    F = np.asarray(force, dtype=float).reshape(3, 1, 1, 1)
    rho = f.sum(0)
    m = np.stack([sum(c19[i, a] * f[i] for i in range(19)) for a in range(3)]) + 0.5 * F
    B = g.sum(1)
    Q = np.concatenate([rho[None], m, B])
    if walls_y:
        ny = f.shape[2]
        for y in (0, ny - 1):
            Q[0, :, y, :] = 1.0
            Q[1:4, :, y, :] = 0.0
            for b in range(3):
                Q[4 + b, :, y, :] = b_wall[b]
    return Q


# ----------------------------------------------------------------------------
# dissipative MHD with locally evolved gradients (sec. 2.2.1, 2.3), D2Q5 / D3Q7:
# Q[8 + 3a + b] = G_ab ~ tau_M d_a B_b, Q[8 + 3 dim + 3a + b] = W_ab ~ tau_M d_a u_b,
# a over the dim lattice axes; dim = Q.ndim - 1
# ----------------------------------------------------------------------------

def diss_flux(Q: np.ndarray, gamma: float, nu: float, eta0: float, j_c: float, tau_m: float) -> np.ndarray:
    """phi[8 + 6 dim, 3, ...] of the full system: ideal flux plus viscous stress, eta(j) j x B
    and -eta grad B, and the gradient lattices' G u - I B, W u - I u."""
    dim = Q.ndim - 1
    nvar, w0 = 8 + 6 * dim, 8 + 3 * dim
    rho, u, e, B, p = primitives(Q[:8], gamma)
    shape = Q.shape[1:]
    pt = p + 0.5 * (B * B).sum(0)
    grad_B = np.zeros((3, 3) + shape)
    grad_u = np.zeros((3, 3) + shape)
    grad_B[:dim] = Q[8:w0].reshape((dim, 3) + shape) / tau_m
    grad_u[:dim] = Q[w0:nvar].reshape((dim, 3) + shape) / tau_m
    visc = rho * nu * (grad_u + np.swapaxes(grad_u, 0, 1))
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    j = np.einsum("abc,bc...->a...", eps, grad_B)  # curl B
    eta = eta0 * (1.0 + ((j * j).sum(0) / j_c ** 2 if j_c > 0 else 0.0))
    jxB = np.cross(j, B, axis=0)
    eye = np.eye(3).reshape((3, 3) + (1,) * len(shape))
    phi = np.zeros((nvar, 3) + shape)
    phi[0] = rho * u
    phi[1:4] = np.einsum("c...,b...->bc...", rho * u, u) + pt * eye - np.einsum("c...,b...->bc...", B, B) \
        - np.swapaxes(visc, 0, 1)
    phi[4] = (e + pt) * u - B * (u * B).sum(0) - np.einsum("b...,bc...->c...", u, visc) + eta * jxB
    phi[5:8] = np.einsum("c...,b...->bc...", u, B) - np.einsum("c...,b...->bc...", B, u) \
        - eta * np.swapaxes(grad_B, 0, 1)
    for a in range(dim):
        for b in range(3):
            phi[8 + 3 * a + b] = Q[8 + 3 * a + b] * u - eye[a] * B[b]
            phi[w0 + 3 * a + b] = Q[w0 + 3 * a + b] * u - eye[a] * u[b]
    return phi


def diss_source(Q: np.ndarray, tau_m: float, powell: bool) -> np.ndarray:
    dim = Q.ndim - 1
    S = np.zeros_like(Q)
    S[8:] = -Q[8:] / tau_m
    if powell:
        rho = Q[0]
        u = Q[1:4] / rho
        divB = sum(Q[8 + 4 * a] for a in range(dim)) / tau_m   # trace of G over the lattice axes
        S[1:4] = -divB * Q[5:8]
        S[4] = -divB * (u * Q[5:8]).sum(0)
        S[5:8] = -divB * u
    return S


def diss_feq(Q: np.ndarray, gamma: float, nu, eta0, j_c, tau_m) -> np.ndarray:
    dim = Q.ndim - 1
    c, w, cs2 = vset("D2Q5" if dim == 2 else "D3Q7")
    phi = diss_flux(Q, gamma, nu, eta0, j_c, tau_m)
    feq = np.zeros((Q.shape[0], len(w)) + Q.shape[1:])
    for i in range(len(w)):
        feq[:, i] = w[i] * (Q + sum(c[i, a] * phi[:, a] for a in range(dim)) / cs2)
    return feq


def diss_step(f: np.ndarray, gamma: float, tau20, nu, eta0, j_c, tau_m, powell) -> np.ndarray:
    dim = f.ndim - 2
    c, w, _ = vset("D2Q5" if dim == 2 else "D3Q7")
    Q = f.sum(axis=1)
    feq = diss_feq(Q, gamma, nu, eta0, j_c, tau_m)
    S = diss_source(Q, tau_m, powell)
    t = np.asarray(tau20, dtype=float).reshape((-1, 1) + (1,) * dim)
    post = f + (feq - f) / t + w.reshape((1, -1) + (1,) * dim) * S[:, None]
    out = np.empty_like(f)
    for i in range(len(w)):
        out[:, i] = _shift(post[:, i], c[i], dim)
    return out


def diss_run(Q0: np.ndarray, gamma: float, tau20, nu, eta0, j_c, tau_m, powell, nsteps: int) -> np.ndarray:
    f = diss_feq(Q0, gamma, nu, eta0, j_c, tau_m)
    for _ in range(nsteps):
        f = diss_step(f, gamma, tau20, nu, eta0, j_c, tau_m, powell)
    return f.sum(axis=1)
