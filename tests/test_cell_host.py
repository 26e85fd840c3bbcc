"""The step kernels' own per-cell arithmetic (ideal_cell.cuh), compiled for the
host from the same source, against the oracle cell by cell -- a check of the
kernel code's moments (Eq. 4), pressure (Eq. 9), fluxes (Eq. 12) and BGK update
with direct source injection (Eq. 2, 3) that needs no GPU.

The host build differs from the device build only in where it runs (and in
FMA contraction, off here), so it checks the formulas as the kernels write
them; the GPU parity tests check the kernels themselves, streaming included.
Covered: FP64 and FP32 plain storage, the Powell form (nine lattices), the
homogenised-solid blend, the FP16/BF16 deviation form (collision on stored
deviations, sources divided by the scale) with and without the FP64 pressure
recovery, and the non-physical flag, on D2Q5 and D3Q7 with uniform sources;
and the dissipative system's fluxes and sources (diss_cell.cuh: viscous
stress, eta(j), the gradient lattices, the Powell source) state by state.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "cell_host.cu")
LIB = os.path.join(HERE, "_build", "libcellhost.so")
W = {2: (1.0 / 3.0, 1.0 / 6.0), 3: (1.0 / 4.0, 1.0 / 8.0)}
FLAG_NONPHYSICAL = 1
F32_TOL = 1e-5   # relative to the lattice's largest population: ~80 FP32 ulps


def _deps():
    csrc = os.path.join(ROOT, "paper_2606_00641_gb300", "csrc")
    return [SRC, os.path.join(csrc, "ideal_cell.cuh"), os.path.join(csrc, "diss_cell.cuh"),
            os.path.join(csrc, "vlbm_internal.cuh"), os.path.join(ROOT, "include", "vlbm.h")]


@pytest.fixture(scope="module")
def H():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    if not os.path.exists(LIB) or any(os.path.getmtime(p) > os.path.getmtime(LIB) for p in _deps()):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "--expt-relaxed-constexpr",
               "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
               "-I", os.path.join(ROOT, "paper_2606_00641_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
               "-shared", SRC, "-o", tmp]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stdout + res.stderr
        os.replace(tmp, LIB)
    L = ctypes.CDLL(LIB)
    i, d, f, p = ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_void_p
    L.hc_ideal_f64.argtypes = [i, d, p, p, p, p, p]
    L.hc_ideal_f32.argtypes = [i, f, p, p, p, p, p]
    L.hc_ideal_dev.argtypes = [i, f, p, p, p, p, p, p, p, f, p, p]
    L.hc_powell_f64.argtypes = [i, d, p, p, p, d, p, p]
    L.hc_powell_f32.argtypes = [i, f, p, p, p, f, p, p]
    L.hc_hom_f64.argtypes = [i, d, p, p, p, d, p, p, p, p]
    L.hc_hom_f32.argtypes = [i, f, p, p, p, f, p, p, p, p]
    L.hc_diss_f64.argtypes = [p, d, d, d, d, d, i, p, p, p]
    L.hc_diss_f32.argtypes = [p, f, f, f, f, f, i, p, p, p]
    L.hc_diss3_f64.argtypes = [p, d, d, d, d, d, i, p, p, p]
    L.hc_diss3_f32.argtypes = [p, f, f, f, f, f, i, p, p, p]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cells(dim, seed, nl=8, amp=0.02):
    """Pre-collision populations [ncell, nl, q]: equilibria of random MHD states
    (the seeded generator), pushed off equilibrium by a seeded perturbation."""
    shape = (6, 7) if dim == 2 else (3, 4, 5)
    f0 = fields.ideal_fields(shape, seed, mach=1.0, beta=1.0, cfl=0.2)
    Q = f0.Q
    if nl == 9:
        rng = np.random.default_rng(seed)
        Q = np.concatenate([Q, 0.05 * rng.normal(size=(1,) + shape)])
        feq = oracle.powell_init(Q, f0.gamma)
    else:
        feq = oracle.ideal_init(Q, f0.gamma)
    q = 2 * dim + 1
    cells = np.moveaxis(feq.reshape(nl, q, -1), -1, 0).copy()
    rng = np.random.default_rng(seed + 1)
    cells += amp * np.abs(cells).max(axis=2, keepdims=True) * rng.normal(size=cells.shape)
    return f0.gamma, cells


def _inputs(dim, nl, dtype, S, scale=None):
    tau = np.linspace(0.55, 0.9, nl)
    w0, w1 = W[dim]
    s = np.ones(nl) if scale is None else scale
    omega = (1.0 / tau).astype(dtype)
    src0 = (w0 * S / s).astype(dtype)
    src1 = (w1 * S / s).astype(dtype)
    return tau, omega, src0, src1


def _check(got, ref, tol):
    scale = np.abs(ref).max(axis=-1, keepdims=True) + 1e-300
    err = np.abs(got - ref) / scale
    assert err.max() < tol, err.max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ideal_collision_matches_the_oracle(H, dim, prec):
    gamma, cells = _cells(dim, 11 + dim)
    S = np.array([0.0, 1e-3, -2e-3, 5e-4, 1e-4, 2e-4, -1e-4, 3e-4])
    dtype = np.float64 if prec == "f64" else np.float32
    tau, omega, src0, src1 = _inputs(dim, 8, dtype, S)
    fn = H.hc_ideal_f64 if prec == "f64" else H.hc_ideal_f32
    flags = np.zeros(1, np.uint32)
    for c in cells:
        got = c.astype(dtype)
        assert fn(dim, gamma - 1.0, _p(omega), _p(src0), _p(src1), _p(got), _p(flags)) == 0
        ref = oracle.ideal_collide_cell(dim, gamma, tau, c, src=S)
        _check(got.astype(np.float64), ref, 1e-13 if prec == "f64" else F32_TOL)
    assert flags[0] == 0


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_powell_collision_matches_the_oracle(H, dim, prec):
    gamma, cells = _cells(dim, 21 + dim, nl=9)
    S = np.array([0.0, 1e-3, -2e-3, 5e-4, 1e-4, 2e-4, -1e-4, 3e-4, 0.0])
    tau_m = 3.0
    dtype = np.float64 if prec == "f64" else np.float32
    tau, omega, src0, src1 = _inputs(dim, 9, dtype, S)
    fn = H.hc_powell_f64 if prec == "f64" else H.hc_powell_f32
    flags = np.zeros(1, np.uint32)
    for c in cells:
        got = c.astype(dtype)
        assert fn(dim, gamma - 1.0, _p(omega), _p(src0), _p(src1), 1.0 / tau_m, _p(got), _p(flags)) == 0
        ref = oracle.powell_collide_cell(dim, gamma, tau, tau_m, c, src=S)
        _check(got.astype(np.float64), ref, 1e-13 if prec == "f64" else F32_TOL)
    assert flags[0] == 0


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_homogenised_solid_collision_matches_the_oracle(H, dim, prec):
    # the oracle's HLBM step on a one-cell periodic grid streams every population
    # back onto its own slot, so it is the collision alone
    gamma, cells = _cells(dim, 31 + dim)
    S = np.array([0.0, 1e-3, -2e-3, 5e-4, 1e-4, 2e-4, -1e-4, 3e-4])
    dtype = np.float64 if prec == "f64" else np.float32
    tau, omega, src0, src1 = _inputs(dim, 8, dtype, S)
    fn = H.hc_hom_f64 if prec == "f64" else H.hc_hom_f32
    rng = np.random.default_rng(7)
    flags = np.zeros(1, np.uint32)
    one = (1,) * dim
    for n, c in enumerate(cells):
        d = [0.0, 1.0, 0.3, 0.75][n % 4]
        uB = (0.05 * rng.normal(size=3)).astype(dtype)
        BB = (0.1 * rng.normal(size=3)).astype(dtype)
        got = c.astype(dtype)
        assert fn(dim, gamma - 1.0, _p(omega), _p(src0), _p(src1), d, _p(uB), _p(BB), _p(got), _p(flags)) == 0
        solid = np.concatenate([[d], uB.astype(np.float64), BB.astype(np.float64)]).reshape((7,) + one)
        ref = oracle.hlbm_step(c.reshape(c.shape + one), gamma, tau, solid, src=S).reshape(c.shape)
        _check(got.astype(np.float64), ref, 1e-13 if prec == "f64" else F32_TOL)
    assert flags[0] == 0


def _dev_setup(dim, cells):
    Q = cells.sum(axis=2)                                  # [ncell, 8]
    r = Q.mean(axis=0)
    s = np.maximum(np.abs(Q - r).max(axis=0), 1e-3)
    q = 2 * dim + 1
    w = np.array([W[dim][0]] + [W[dim][1]] * (q - 1))
    return r, s, w


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("codec", [np.float16, "bf16"])
def test_deviation_form_collides_the_stored_deviations_like_the_oracle(H, dim, codec):
    # g = (f - w_i r_k) / s_k as stored (rounded to 16 bits, as the decode sees it), collided
    # in FP32, decoded f* = w_i r_k + s_k g*, against the oracle on the decoded f
    gamma, cells = _cells(dim, 41 + dim)
    r, s, w = _dev_setup(dim, cells)
    S = np.array([0.0, 1e-3, -2e-3, 5e-4, 1e-4, 2e-4, -1e-4, 3e-4])
    tau, omega, src0, src1 = _inputs(dim, 8, np.float32, S, scale=s)
    ref32, scale32, inv32 = r.astype(np.float32), s.astype(np.float32), (1.0 / s).astype(np.float32)
    refscale = np.concatenate([r, s])
    flags = np.zeros(1, np.uint32)

    def round16(x):
        if codec is np.float16:
            return x.astype(np.float16).astype(np.float32)
        b = x.astype(np.float32).view(np.uint32)            # round to nearest even on the upper 16 bits
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32)

    for c in cells:
        g = round16((c - w[None, :] * r[:, None]) / s[:, None]).astype(np.float32)
        f_dec = w[None, :] * r[:, None] + s[:, None] * g.astype(np.float64)
        got = g.copy()
        assert H.hc_ideal_dev(dim, gamma - 1.0, _p(omega), _p(src0), _p(src1), _p(ref32), _p(scale32), _p(inv32),
                              _p(refscale), 0.01, _p(got), _p(flags)) == 0
        f_new = w[None, :] * r[:, None] + s[:, None] * got.astype(np.float64)
        ref = oracle.ideal_collide_cell(dim, gamma, tau, f_dec, src=S)
        _check(f_new, ref, 2e-5)
    assert flags[0] == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_deviation_form_recovers_the_pressure_of_a_cold_plasma_in_fp64(H, dim):
    # beta = 5e-9: e_tot - |B|^2/2 is below the FP32 ulp of e_tot, so the FP32
    # pressure is not positive; with p_theta > 0 the cell takes p in FP64 from
    # r_k + s_k G_k and stays physical, with p_theta = 0 it raises the flag
    gamma, B0, p0 = 5.0 / 3.0, 0.2, 1e-10
    Q = np.zeros((8,) + (1,) * dim)
    Q[0], Q[4], Q[7] = 1.0, p0 / (gamma - 1) + 0.5 * B0 * B0, B0
    feq = oracle.ideal_init(Q, gamma).reshape(8, 2 * dim + 1)
    r = Q.reshape(8).copy()
    s = np.array([1.0, 0.01, 0.01, 0.01, 1.0, 1.0, 1.0, 1.0])
    w = np.array([W[dim][0]] + [W[dim][1]] * (2 * dim))
    g0 = ((feq - w[None, :] * r[:, None]) / s[:, None]).astype(np.float32)
    tau, omega, src0, src1 = _inputs(dim, 8, np.float32, np.zeros(8), scale=s)
    args = (_p(omega), _p(src0), _p(src1), _p(r.astype(np.float32)), _p(s.astype(np.float32)),
            _p((1.0 / s).astype(np.float32)), _p(np.concatenate([r, s])))
    ok, bad = np.zeros(1, np.uint32), np.zeros(1, np.uint32)
    g = g0.copy()
    assert H.hc_ideal_dev(dim, gamma - 1.0, *args, 0.01, _p(g), _p(ok)) == 0
    assert ok[0] == 0
    # the state at rest is a fixed point: every lattice keeps its sum
    np.testing.assert_allclose(g.astype(np.float64).sum(1), g0.astype(np.float64).sum(1), atol=1e-7)
    g = g0.copy()
    assert H.hc_ideal_dev(dim, gamma - 1.0, *args, 0.0, _p(g), _p(bad)) == 0
    assert bad[0] & FLAG_NONPHYSICAL


@pytest.mark.parametrize("dim", [2, 3])
def test_non_physical_cell_raises_the_flag(H, dim):
    gamma, cells = _cells(dim, 51)
    c = cells[0].copy()
    c[4] *= -1.0   # negative total energy: p < 0
    tau, omega, src0, src1 = _inputs(dim, 8, np.float64, np.zeros(8))
    flags = np.zeros(1, np.uint32)
    assert H.hc_ideal_f64(dim, gamma - 1.0, _p(omega), _p(src0), _p(src1), _p(c), _p(flags)) == 0
    assert flags[0] & FLAG_NONPHYSICAL
    assert H.hc_ideal_f64(4, gamma - 1.0, _p(omega), _p(src0), _p(src1), _p(c), _p(flags)) == -1


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("powell", [False, True])
@pytest.mark.parametrize("j_c", [0.0, 0.08])
def test_dissipative_fluxes_and_sources_match_the_oracle(H, prec, powell, j_c):
    shape = (6, 7)
    f0 = fields.ideal_fields(shape, 61, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(62)
    Q = np.concatenate([f0.Q, 0.05 * rng.normal(size=(12,) + shape)]).reshape(20, -1).T
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=j_c, tau_m=1.7, powell=powell)
    dtype = np.float64 if prec == "f64" else np.float32
    fn = H.hc_diss_f64 if prec == "f64" else H.hc_diss_f32
    inv_jc2 = 1.0 / (j_c * j_c) if j_c > 0 else 0.0
    tol = 1e-13 if prec == "f64" else F32_TOL
    flags = np.zeros(1, np.uint32)
    for q in Q:
        phi = np.zeros(40, dtype)
        S = np.zeros(20, dtype)
        assert fn(_p(q.astype(dtype)), f0.gamma - 1.0, dp.nu, dp.eta0, inv_jc2, 1.0 / dp.tau_m, int(powell),
                  _p(phi), _p(S), _p(flags)) == 0
        ref_phi = oracle.diss_flux(f0.gamma, dp, q)[:, :2]
        ref_S = oracle.diss_source(dp, q)
        # each lattice's fluxes against the largest flux of the state's MHD part (the terms
        # a flux is made of are of that size), sources against the largest source
        pscale = np.abs(ref_phi).max()
        assert np.abs(phi.reshape(20, 2).astype(np.float64) - ref_phi).max() < tol * pscale
        sscale = np.abs(ref_S).max()
        assert np.abs(S.astype(np.float64) - ref_S).max() < tol * sscale
    assert flags[0] == 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("powell", [False, True])
@pytest.mark.parametrize("j_c", [0.0, 0.08])
def test_dissipative_3d_fluxes_and_sources_match_the_oracle(H, prec, powell, j_c):
    # the 26-lattice D3Q7 form: every lattice's flux along x, y, z and its source
    shape = (3, 4, 5)
    f0 = fields.ideal_fields(shape, 63, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(64)
    Q = np.concatenate([f0.Q, 0.05 * rng.normal(size=(18,) + shape)]).reshape(26, -1).T
    dp = oracle.Dissipation(nu=0.02, eta0=0.03, j_c=j_c, tau_m=1.7, powell=powell)
    dtype = np.float64 if prec == "f64" else np.float32
    fn = H.hc_diss3_f64 if prec == "f64" else H.hc_diss3_f32
    inv_jc2 = 1.0 / (j_c * j_c) if j_c > 0 else 0.0
    tol = 1e-13 if prec == "f64" else F32_TOL
    flags = np.zeros(1, np.uint32)
    for q in Q:
        phi = np.zeros(78, dtype)
        S = np.zeros(26, dtype)
        assert fn(_p(q.astype(dtype)), f0.gamma - 1.0, dp.nu, dp.eta0, inv_jc2, 1.0 / dp.tau_m, int(powell),
                  _p(phi), _p(S), _p(flags)) == 0
        ref_phi = oracle.diss_flux(f0.gamma, dp, q, dim=3)
        ref_S = oracle.diss_source(dp, q, dim=3)
        pscale = np.abs(ref_phi).max()
        assert np.abs(phi.reshape(26, 3).astype(np.float64) - ref_phi).max() < tol * pscale
        sscale = np.abs(ref_S).max()
        assert np.abs(S.astype(np.float64) - ref_S).max() < tol * sscale
    assert flags[0] == 0
