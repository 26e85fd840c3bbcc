"""Plain FP64 CPU oracle of the vectorial LBM for MHD.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA path; the product
library never loads it.

Two independent statements of the method live here:

* ``vlbm_oracle.c`` -- plain C, two population arrays, push streaming,
  compiled with ``-ffp-contract=off`` (the oracle proper);
* ``numpy_ref.py`` -- a NumPy restatement for tiny grids, used to
  brute-force check the C code.

Equation numbers follow the order in which the paper displays them
(Eq. 2 update, Eq. 3 equilibrium, Eq. 4 moments, Eq. 9 EOS, Eq. 12 ideal
MHD flux); see the header of ``vlbm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NVAR_IDEAL = 8
NVAR_RESISTIVE = 7


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _configure(L):
    d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    L.orc_ideal_flux.argtypes = [d, p, p]
    L.orc_ideal_flux.restype = None
    L.orc_ideal_pressure.argtypes = [d, p]
    L.orc_ideal_pressure.restype = d
    L.orc_lattice_info.argtypes = [i, p, p, p, p]
    L.orc_ideal_collide_cell.argtypes = [i, d, p, p, p, p]
    L.orc_ideal_init.argtypes = [i, i, i, i, d, p, p]
    L.orc_ideal_step.argtypes = [i, i, i, i, d, p, p, p, p, i]
    L.orc_ideal_moments.argtypes = [i, i, i, i, p, p]
    L.orc_ideal_run.argtypes = [i, i, i, i, d, p, p, p, i, p, i]
    L.orc_resistive_init.argtypes = [i, i, i, p, p, p, p]
    L.orc_resistive_step.argtypes = [i, i, i, d, d, p, p, i, p, p, p, p, i]
    L.orc_resistive_moments.argtypes = [i, i, i, p, p, i, p, p, p]
    L.orc_resistive_run.argtypes = [i, i, i, d, d, p, p, i, p, i, p, i]
    L.orc_resistive_collide_cell.argtypes = [d, d, p, p, p]
    L.orc_powell_flux.argtypes = [d, p, p]
    L.orc_powell_flux.restype = None
    L.orc_powell_source.argtypes = [d, p, p]
    L.orc_powell_source.restype = None
    L.orc_powell_collide_cell.argtypes = [i, d, p, d, p, p, p]
    L.orc_powell_init.argtypes = [i, i, i, i, d, p, p]
    L.orc_powell_step.argtypes = [i, i, i, i, d, p, d, p, p, p, i]
    L.orc_powell_moments.argtypes = [i, i, i, i, p, p]
    L.orc_powell_run.argtypes = [i, i, i, i, d, p, d, p, p, i, p, i]
    L.orc_hlbm_porosity.argtypes = [d, d]
    L.orc_hlbm_porosity.restype = ctypes.c_double
    L.orc_hlbm_target.argtypes = [d, p, d, p, p, p]
    L.orc_hlbm_target.restype = None
    L.orc_hlbm_step.argtypes = [i, i, i, i, d, p, p, p, p, p, i]
    L.orc_hlbm_run.argtypes = [i, i, i, i, d, p, p, p, p, i, p, i]
    L.orc_diss_flux.argtypes = [d, d, d, d, d, p, p]
    L.orc_diss_flux.restype = None
    L.orc_diss_source.argtypes = [d, i, p, p]
    L.orc_diss_source.restype = None
    L.orc_diss_init.argtypes = [i, i, d, d, d, d, d, p, p]
    L.orc_diss_step.argtypes = [i, i, d, p, d, d, d, d, i, p, p, i]
    L.orc_diss_moments.argtypes = [i, i, p, p]
    L.orc_diss_run.argtypes = [i, i, d, p, d, d, d, d, i, p, i, p, i]
    L.orc_diss_flux_d.argtypes = [i, d, d, d, d, d, p, p]
    L.orc_diss_flux_d.restype = None
    L.orc_diss_source_d.argtypes = [i, d, i, p, p]
    L.orc_diss_source_d.restype = None
    L.orc_diss_init_d.argtypes = [i, i, i, i, d, d, d, d, d, p, p]
    L.orc_diss_step_d.argtypes = [i, i, i, i, d, p, d, d, d, d, i, p, p, i]
    L.orc_diss_moments_d.argtypes = [i, i, i, i, p, p]
    L.orc_diss_run_d.argtypes = [i, i, i, i, d, p, d, d, d, d, i, p, i, p, i]
    L.orc_open_step.argtypes = [i, i, i, i, d, p, p, p, p, p, p, p, p, i]
    L.orc_open_run.argtypes = [i, i, i, i, d, p, p, p, p, p, p, p, i, p, i]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of the
    oracle source (used by the mutation test, which plants mistakes in a copy
    of ``vlbm_oracle.c`` to show that the pins catch them)."""

    def __init__(self, path: str):
        self._new = _configure(ctypes.CDLL(path))

    def __enter__(self):
        global _lib
        lib()
        self._old = _lib
        _lib = self._new
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._old
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source with the oracle's flags."""
    c_path = out_path + ".c"
    with open(c_path, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                    "-shared", "-std=c99", c_path, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle %s failed (rc=%d)" % (what, rc))


def lattice(q: int):
    """(c[q,3] int, w[q], cs2, opp[q]) of D2Q5 / D3Q7 / D3Q19."""
    c = np.zeros(3 * q, dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    cs2 = ctypes.c_double(0.0)
    _check(lib().orc_lattice_info(q, c.ctypes.data_as(ctypes.c_void_p), _ptr(w),
                                  ctypes.byref(cs2), opp.ctypes.data_as(ctypes.c_void_p)),
           "lattice_info")
    return c.reshape(q, 3), w, cs2.value, opp


def ideal_flux(gamma: float, Q) -> np.ndarray:
    """Flux tensor phi[k, a] of ideal MHD (Eq. 12) at one state Q[8]."""
    Q = _f64(Q)
    phi = np.zeros(24)
    lib().orc_ideal_flux(gamma, _ptr(Q), _ptr(phi))
    return phi.reshape(8, 3)


def ideal_pressure(gamma: float, Q) -> float:
    return lib().orc_ideal_pressure(gamma, _ptr(_f64(Q)))


def _dims(shape):
    if len(shape) == 2:
        ny, nx = shape
        return 2, nx, ny, 1
    nz, ny, nx = shape
    return 3, nx, ny, nz


def ideal_init(Q0: np.ndarray, gamma: float) -> np.ndarray:
    """Populations f[8, q, *shape] = f_eq(Q0); Q0 has shape [8, (nz,) ny, nx]."""
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _dims(Q0.shape[1:])
    q = 5 if dim == 2 else 7
    f = np.zeros((8, q) + Q0.shape[1:])
    _check(lib().orc_ideal_init(dim, nx, ny, nz, gamma, _ptr(Q0), _ptr(f)), "init")
    return f


def ideal_step(f: np.ndarray, gamma: float, tau, src=None, nthreads: int = 1) -> np.ndarray:
    f = _f64(f)
    dim, nx, ny, nz = _dims(f.shape[2:])
    out = np.empty_like(f)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (8,)))
    s = _f64(src) if src is not None else None
    _check(lib().orc_ideal_step(dim, nx, ny, nz, gamma, _ptr(tau),
                                _ptr(s) if s is not None else None, _ptr(f), _ptr(out),
                                nthreads), "step")
    return out


def ideal_moments(f: np.ndarray) -> np.ndarray:
    f = _f64(f)
    dim, nx, ny, nz = _dims(f.shape[2:])
    Q = np.zeros((8,) + f.shape[2:])
    _check(lib().orc_ideal_moments(dim, nx, ny, nz, _ptr(f), _ptr(Q)), "moments")
    return Q


def ideal_collide_cell(dim: int, gamma: float, tau, fin, src=None) -> np.ndarray:
    """Post-collision populations [8, q] of one cell from its pre-collision ones."""
    fin = _f64(fin)
    out = np.zeros_like(fin)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (8,)))
    s = _f64(src) if src is not None else None
    _check(lib().orc_ideal_collide_cell(dim, gamma, _ptr(tau), _ptr(s) if s is not None else None,
                                        _ptr(fin), _ptr(out)), "collide_cell")
    return out


def ideal_run(Q0: np.ndarray, gamma: float, tau, nsteps: int, src=None,
              nthreads: int = 1) -> np.ndarray:
    """Moments after nsteps steps of the ideal-MHD VLBM started from f_eq(Q0)."""
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _dims(Q0.shape[1:])
    out = np.zeros_like(Q0)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (8,)))
    s = _f64(src) if src is not None else None
    _check(lib().orc_ideal_run(dim, nx, ny, nz, gamma, _ptr(tau),
                               _ptr(s) if s is not None else None, _ptr(Q0), nsteps,
                               _ptr(out), nthreads), "run")
    return out


# ---- ideal MHD with the Powell correction: nine fields, the ninth D ~ tau_M div B ----

def powell_flux(gamma: float, Q) -> np.ndarray:
    """Flux phi[k, a] of the nine Powell-form fields at one state Q[9]."""
    phi = np.zeros(27)
    lib().orc_powell_flux(gamma, _ptr(_f64(Q)), _ptr(phi))
    return phi.reshape(9, 3)


def powell_source(tau_m: float, Q) -> np.ndarray:
    """Source S[9] at one state: Powell's term with div B = D / tau_M, and -D / tau_M."""
    S = np.zeros(9)
    lib().orc_powell_source(tau_m, _ptr(_f64(Q)), _ptr(S))
    return S


def _tau9(tau):
    return _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (9,)))


def powell_init(Q0: np.ndarray, gamma: float) -> np.ndarray:
    """Populations f[9, q, *shape] = f_eq(Q0); Q0 has shape [9, (nz,) ny, nx]."""
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _dims(Q0.shape[1:])
    q = 5 if dim == 2 else 7
    f = np.zeros((9, q) + Q0.shape[1:])
    _check(lib().orc_powell_init(dim, nx, ny, nz, gamma, _ptr(Q0), _ptr(f)), "powell_init")
    return f


def powell_step(f: np.ndarray, gamma: float, tau, tau_m: float, src=None, nthreads: int = 1) -> np.ndarray:
    f = _f64(f)
    dim, nx, ny, nz = _dims(f.shape[2:])
    out = np.empty_like(f)
    s = _f64(src) if src is not None else None
    _check(lib().orc_powell_step(dim, nx, ny, nz, gamma, _ptr(_tau9(tau)), tau_m,
                                 _ptr(s) if s is not None else None, _ptr(f), _ptr(out), nthreads),
           "powell_step")
    return out


def powell_moments(f: np.ndarray) -> np.ndarray:
    f = _f64(f)
    dim, nx, ny, nz = _dims(f.shape[2:])
    Q = np.zeros((9,) + f.shape[2:])
    _check(lib().orc_powell_moments(dim, nx, ny, nz, _ptr(f), _ptr(Q)), "powell_moments")
    return Q


def powell_collide_cell(dim: int, gamma: float, tau, tau_m: float, fin, src=None) -> np.ndarray:
    """Post-collision populations [9, q] of one cell from its pre-collision ones."""
    fin = _f64(fin)
    out = np.zeros_like(fin)
    s = _f64(src) if src is not None else None
    _check(lib().orc_powell_collide_cell(dim, gamma, _ptr(_tau9(tau)), tau_m,
                                         _ptr(s) if s is not None else None, _ptr(fin), _ptr(out)),
           "powell_collide_cell")
    return out


def powell_run(Q0: np.ndarray, gamma: float, tau, tau_m: float, nsteps: int, src=None,
               nthreads: int = 1) -> np.ndarray:
    """Moments [9, ...] after nsteps steps of the Powell form started from f_eq(Q0)."""
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _dims(Q0.shape[1:])
    out = np.zeros_like(Q0)
    s = _f64(src) if src is not None else None
    _check(lib().orc_powell_run(dim, nx, ny, nz, gamma, _ptr(_tau9(tau)), tau_m,
                                _ptr(s) if s is not None else None, _ptr(Q0), nsteps, _ptr(out),
                                nthreads), "powell_run")
    return out


# ---- homogenised solids (HLBM, sec. 2.4): porosity d, solid velocity uB and field BB per cell ----

def hlbm_porosity(phi, eps_h: float) -> np.ndarray:
    """d(phi) for an array of signed distances (positive in the fluid)."""
    phi = np.asarray(phi, dtype=np.float64)
    return np.vectorize(lambda v: lib().orc_hlbm_porosity(float(v), float(eps_h)), otypes=[float])(phi)


def hlbm_target(gamma: float, Q, d: float, uB, BB) -> np.ndarray:
    """Blended state Q_hat[8] of one cell."""
    out = np.zeros(8)
    lib().orc_hlbm_target(gamma, _ptr(_f64(Q)), float(d), _ptr(_f64(uB)), _ptr(_f64(BB)), _ptr(out))
    return out


def _solid(solid, shape):
    solid = _f64(solid)
    assert solid.shape == (7,) + tuple(shape)
    return solid


def hlbm_step(f: np.ndarray, gamma: float, tau, solid, src=None, nthreads: int = 1) -> np.ndarray:
    """One step with homogenised solids; solid = [d, uB_x, uB_y, uB_z, BB_x, BB_y, BB_z] per cell."""
    f = _f64(f)
    dim, nx, ny, nz = _dims(f.shape[2:])
    out = np.empty_like(f)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (8,)))
    s = _f64(src) if src is not None else None
    _check(lib().orc_hlbm_step(dim, nx, ny, nz, gamma, _ptr(tau), _ptr(s) if s is not None else None,
                               _ptr(_solid(solid, f.shape[2:])), _ptr(f), _ptr(out), nthreads), "hlbm_step")
    return out


def hlbm_run(Q0: np.ndarray, gamma: float, tau, solid, nsteps: int, src=None, nthreads: int = 1) -> np.ndarray:
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _dims(Q0.shape[1:])
    out = np.zeros_like(Q0)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (8,)))
    s = _f64(src) if src is not None else None
    _check(lib().orc_hlbm_run(dim, nx, ny, nz, gamma, _ptr(tau), _ptr(s) if s is not None else None,
                              _ptr(_solid(solid, Q0.shape[1:])), _ptr(Q0), nsteps, _ptr(out), nthreads),
           "hlbm_run")
    return out


def resistive_init(Q0: np.ndarray, force):
    Q0 = _f64(Q0)
    nz, ny, nx = Q0.shape[1:]
    f = np.zeros((19,) + Q0.shape[1:])
    g = np.zeros((3, 7) + Q0.shape[1:])
    _check(lib().orc_resistive_init(nx, ny, nz, _ptr(Q0), _ptr(_f64(force)), _ptr(f), _ptr(g)),
           "resistive_init")
    return f, g


def resistive_step(f, g, tau_f, tau_m, force, b_wall, walls_y, nthreads: int = 1):
    f, g = _f64(f), _f64(g)
    nz, ny, nx = f.shape[1:]
    fo, go = f.copy(), g.copy()
    _check(lib().orc_resistive_step(nx, ny, nz, tau_f, tau_m, _ptr(_f64(force)),
                                    _ptr(_f64(b_wall)), int(walls_y), _ptr(f), _ptr(g),
                                    _ptr(fo), _ptr(go), nthreads), "resistive_step")
    return fo, go


def resistive_moments(f, g, force, b_wall, walls_y):
    f, g = _f64(f), _f64(g)
    nz, ny, nx = f.shape[1:]
    Q = np.zeros((7,) + f.shape[1:])
    _check(lib().orc_resistive_moments(nx, ny, nz, _ptr(_f64(force)), _ptr(_f64(b_wall)),
                                       int(walls_y), _ptr(f), _ptr(g), _ptr(Q)),
           "resistive_moments")
    return Q


def resistive_collide_cell(tau_f, tau_m, force, fin) -> np.ndarray:
    """Post-collision populations [40] (19 flow, then 3 x 7 magnetic) of one fluid cell."""
    fin = _f64(fin)
    out = np.zeros(40)
    _check(lib().orc_resistive_collide_cell(tau_f, tau_m, _ptr(_f64(force)), _ptr(fin), _ptr(out)),
           "resistive_collide_cell")
    return out


def resistive_run(Q0, tau_f, tau_m, force, b_wall, walls_y, nsteps, nthreads: int = 1):
    Q0 = _f64(Q0)
    nz, ny, nx = Q0.shape[1:]
    out = np.zeros_like(Q0)
    _check(lib().orc_resistive_run(nx, ny, nz, tau_f, tau_m, _ptr(_f64(force)),
                                   _ptr(_f64(b_wall)), int(walls_y), _ptr(Q0), nsteps,
                                   _ptr(out), nthreads), "resistive_run")
    return out


# ---- static equilibrium boundaries (sec. 2.4, "Static boundaries") ----

def _faces(faces, dim):
    """faces: up to six entries for x-, x+, y-, y+, z-, z+, each None (periodic) or
    (mask, values): bit k of mask set = Q_k Dirichlet at values[k], clear = Neumann."""
    faces = list(faces) + [None] * (6 - len(faces))
    open_ = np.zeros(3, dtype=np.int32)
    mask = np.zeros(6, dtype=np.uint32)
    vals = np.zeros(48)
    for a in range(3):
        lo, hi = faces[2 * a], faces[2 * a + 1]
        if (lo is None) != (hi is None):
            raise ValueError("both faces of an axis are open or both periodic")
        if lo is None:
            continue
        if a >= dim:
            raise ValueError("face beyond the grid's dimension")
        open_[a] = 1
        for f, spec in ((2 * a, lo), (2 * a + 1, hi)):
            m, v = spec
            mask[f] = int(m)
            vals[8 * f:8 * f + 8] = np.asarray(v if v is not None else np.zeros(8), dtype=np.float64)
    return open_, mask, vals


def open_step(f: np.ndarray, gamma: float, tau, faces, src=None, solid=None, nthreads: int = 1) -> np.ndarray:
    """One step with open faces (equilibrium Dirichlet / Neumann boundaries), optionally
    with homogenised solids in the domain."""
    f = _f64(f)
    dim, nx, ny, nz = _dims(f.shape[2:])
    open_, mask, vals = _faces(faces, dim)
    out = np.zeros_like(f)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (8,)))
    s = _f64(src) if src is not None else None
    sd = _solid(solid, f.shape[2:]) if solid is not None else None
    _check(lib().orc_open_step(dim, nx, ny, nz, gamma, _ptr(tau), _ptr(s) if s is not None else None,
                               _ptr(sd) if sd is not None else None,
                               open_.ctypes.data_as(ctypes.c_void_p), mask.ctypes.data_as(ctypes.c_void_p),
                               _ptr(vals), _ptr(f), _ptr(out), nthreads), "open_step")
    return out


def open_run(Q0: np.ndarray, gamma: float, tau, faces, nsteps: int, src=None, solid=None,
             nthreads: int = 1) -> np.ndarray:
    """Moments [8, ...] after nsteps steps with open faces, started from f_eq(Q0)."""
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _dims(Q0.shape[1:])
    open_, mask, vals = _faces(faces, dim)
    out = np.zeros_like(Q0)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (8,)))
    s = _f64(src) if src is not None else None
    sd = _solid(solid, Q0.shape[1:]) if solid is not None else None
    _check(lib().orc_open_run(dim, nx, ny, nz, gamma, _ptr(tau), _ptr(s) if s is not None else None,
                              _ptr(sd) if sd is not None else None,
                              open_.ctypes.data_as(ctypes.c_void_p), mask.ctypes.data_as(ctypes.c_void_p),
                              _ptr(vals), _ptr(Q0), nsteps, _ptr(out), nthreads), "open_run")
    return out


# ---- dissipative MHD with locally evolved gradients (sec. 2.2.1, 2.3), D2Q5 and D3Q7 ----
# Q[8 + 6 dim]: rho, rho u (3), e, B (3), G_ab = Q[8 + 3a + b] ~ tau_M d_a B_b,
# W_ab = Q[8 + 3 dim + 3a + b] ~ tau_M d_a u_b, with a over the dim lattice axes and b over x, y, z.

NVAR_DISS = 20      # 2-D
NVAR_DISS_3D = 26


def diss_nvar(dim: int) -> int:
    return 8 + 6 * dim


class Dissipation:
    """Physical parameters of the dissipative model: kinematic viscosity nu,
    resistivity eta0 (1 + |j|^2 / j_c^2) (j_c <= 0: constant), tau_M in steps,
    Powell source on or off."""

    def __init__(self, nu=0.0, eta0=0.0, j_c=0.0, tau_m=1.0, powell=False):
        self.nu, self.eta0, self.j_c, self.tau_m, self.powell = float(nu), float(eta0), float(j_c), float(tau_m), bool(powell)


def _tau_diss(tau, tau_g=None, dim: int = 2):
    nvar = diss_nvar(dim)
    t = np.asarray(tau, dtype=np.float64).reshape(-1)
    if t.size == nvar:
        return _f64(t)
    t8 = np.broadcast_to(t, (8,)) if t.size in (1, 8) else None
    if t8 is None:
        raise ValueError(f"tau: 1, 8 or {nvar} values")
    g = float(t8[0]) if tau_g is None else float(tau_g)
    return _f64(np.concatenate([t8, np.full(nvar - 8, g)]))


def _tau20(tau, tau_g=None):
    return _tau_diss(tau, tau_g, 2)


def _diss_grid(a: np.ndarray, lead: int):
    """(dim, nx, ny, nz) of an array [lead..., ny, nx] (2-D) or [lead..., nz, ny, nx] (3-D)."""
    spatial = a.shape[lead:]
    if len(spatial) == 2:
        return 2, spatial[1], spatial[0], 1
    if len(spatial) == 3:
        return 3, spatial[2], spatial[1], spatial[0]
    raise ValueError("dissipative fields: [nvar, ny, nx] or [nvar, nz, ny, nx]")


def diss_flux(gamma: float, dp: Dissipation, Q, dim: int = 2) -> np.ndarray:
    """Flux tensor phi[nvar, 3] of one state (nvar = 20 in 2-D, 26 in 3-D)."""
    nvar = diss_nvar(dim)
    Q = _f64(Q)
    if Q.size != nvar:
        raise ValueError(f"{dim}-D state: {nvar} values")
    out = np.zeros(3 * nvar)
    lib().orc_diss_flux_d(dim, gamma, dp.nu, dp.eta0, dp.j_c, dp.tau_m, _ptr(Q), _ptr(out))
    return out.reshape(nvar, 3)


def diss_source(dp: Dissipation, Q, dim: int = 2) -> np.ndarray:
    nvar = diss_nvar(dim)
    Q = _f64(Q)
    if Q.size != nvar:
        raise ValueError(f"{dim}-D state: {nvar} values")
    out = np.zeros(nvar)
    lib().orc_diss_source_d(dim, dp.tau_m, int(dp.powell), _ptr(Q), _ptr(out))
    return out


def diss_init(Q0: np.ndarray, gamma: float, dp: Dissipation) -> np.ndarray:
    """Populations f[nvar, q, (nz,) ny, nx] = f_eq(Q0); Q0 [20, ny, nx] (D2Q5) or [26, nz, ny, nx] (D3Q7)."""
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _diss_grid(Q0, 1)
    f = np.zeros((diss_nvar(dim), 2 * dim + 1) + Q0.shape[1:])
    _check(lib().orc_diss_init_d(dim, nx, ny, nz, gamma, dp.nu, dp.eta0, dp.j_c, dp.tau_m, _ptr(Q0), _ptr(f)),
           "diss_init")
    return f


def diss_step(f: np.ndarray, gamma: float, tau, dp: Dissipation, tau_g=None, nthreads: int = 1) -> np.ndarray:
    f = _f64(f)
    dim, nx, ny, nz = _diss_grid(f, 2)
    out = np.empty_like(f)
    _check(lib().orc_diss_step_d(dim, nx, ny, nz, gamma, _ptr(_tau_diss(tau, tau_g, dim)), dp.nu, dp.eta0, dp.j_c,
                                 dp.tau_m, int(dp.powell), _ptr(f), _ptr(out), nthreads), "diss_step")
    return out


def diss_moments(f: np.ndarray) -> np.ndarray:
    f = _f64(f)
    dim, nx, ny, nz = _diss_grid(f, 2)
    Q = np.zeros((diss_nvar(dim),) + f.shape[2:])
    _check(lib().orc_diss_moments_d(dim, nx, ny, nz, _ptr(f), _ptr(Q)), "diss_moments")
    return Q


def diss_run(Q0: np.ndarray, gamma: float, tau, dp: Dissipation, nsteps: int, tau_g=None,
             nthreads: int = 1) -> np.ndarray:
    """Moments [nvar, (nz,) ny, nx] after nsteps steps started from f_eq(Q0)."""
    Q0 = _f64(Q0)
    dim, nx, ny, nz = _diss_grid(Q0, 1)
    out = np.zeros_like(Q0)
    _check(lib().orc_diss_run_d(dim, nx, ny, nz, gamma, _ptr(_tau_diss(tau, tau_g, dim)), dp.nu, dp.eta0, dp.j_c,
                                dp.tau_m, int(dp.powell), _ptr(Q0), nsteps, _ptr(out), nthreads), "diss_run")
    return out
