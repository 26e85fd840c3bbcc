"""Slab decomposition of one periodic domain on the GPU (vlbm_set_slab,
vlbm_halo_pack / vlbm_halo_unpack, vlbm_slabs_step).

P slabs of one domain, each a context on this GPU, exchange the population
planes that wrapped inside them after every step.  Every element moves
unchanged and every cell runs the same arithmetic as in the undivided domain,
so the decomposed run must equal the single-context run bit for bit (moments
and populations), at both AA parities, for every model and storage that the
exchange serves, and the oracle to the usual tolerances (FP64 1e-12, FP32
1e-5).  The exchange through the public pack/unpack calls, routed by
``slabs.route`` as the one-process-per-GPU driver routes it, must equal the
library's own group step.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


@pytest.fixture(scope="module")
def S():
    from paper_2606_00641_gb300 import slabs
    return slabs


def ideal_scales(Q0):
    rho = np.abs(Q0[0]).max()
    mom = np.abs(Q0[1:4]).max()
    B = np.abs(Q0[5:8]).max()
    return np.array([rho, mom, mom, mom, np.abs(Q0[4]).max(), B, B, B])


def rel_err(got, ref, scales):
    nv = got.shape[0]
    g, r = got.reshape(nv, -1), ref.reshape(nv, -1)
    return np.abs(g - r).max(1) / (np.maximum(np.abs(r).max(1), scales) + 1e-300)


def dev_ref_scale(Q):
    flat = Q.reshape(Q.shape[0], -1)[:8]
    ref = flat.mean(1)
    return ref, np.maximum(np.abs(flat - ref[:, None]).max(1), 1e-30)


def single_run(V, params, Q0, steps):
    with V.Context(params) as ctx:
        assert ctx.init_fields(Q0) == V.VLBM_OK
        ctx.step(steps)
        out = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    return out


def slab_run(V, S, make, shape, parts, Q0, steps):
    with S.LocalSlabs(make, shape, parts) as g:
        assert g.init_fields(Q0) == V.VLBM_OK
        assert g.step(steps) == V.VLBM_OK
        out = g.moments()
        sums = g.conservation()
        assert g.sync() == V.VLBM_OK
    return out, sums


# ---------------------------------------------------------------------------
# ideal MHD, every storage
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ["f64", "f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("parts", [2, 4])
@pytest.mark.parametrize("steps", [6, 7])
def test_ideal_slabs_equal_the_single_domain_bit_for_bit(V, S, storage, parts, steps):
    shape = (16, 10, 24)  # nx % 8 == 0: the 16-bit forms run the bulk-copy pairs kernel
    f0 = fields.ideal_fields(shape, 515, mach=1.2, beta=1.0, cfl=0.2)
    qref, qscale = dev_ref_scale(f0.Q)
    tau = [0.51, 0.6, 0.7, 0.8, 0.55, 0.9, 1.0, 0.65]

    def make(sub):
        return V.make_params(shape=sub, storage=storage, gamma=f0.gamma, tau=tau, q_ref=qref, q_scale=qscale)

    ref = single_run(V, make(shape), f0.Q, steps)
    got, sums = slab_run(V, S, make, shape, parts, f0.Q, steps)
    assert np.array_equal(got, ref)
    with V.Context(make(shape)) as ctx:
        ctx.init_fields(f0.Q)
        ctx.step(steps)
        whole = ctx.conservation()
    assert (np.abs(sums - whole) / np.abs(f0.Q).reshape(8, -1).sum(1)).max() < 1e-13
    if storage in ("f64", "f32"):
        orc = oracle.ideal_run(f0.Q, f0.gamma, tau, steps)
        tol = 1e-12 if storage == "f64" else 1e-5
        assert rel_err(got, orc, ideal_scales(f0.Q)).max() < tol


@pytest.mark.parametrize("shape,parts,storage", [
    ((16, 6, 8), 16, "f32"),        # one layer per slab: both faces are the same layer
    ((10, 7, 9), 3, "f64"),         # uneven slabs (4, 3, 3 layers), ragged x
    ((12, 5, 20), 3, "f16dev"),     # 16-bit one-cell-per-thread kernel (nx % 8 != 0)
    ((24, 40), 2, "f64"),           # 2-D: slabs along y, D2Q5
    ((30, 17), 3, "f32"),
    ((24, 16), 4, "bf16dev"),
])
@pytest.mark.parametrize("steps", [4, 5])
def test_ideal_slab_shapes_equal_the_single_domain(V, S, shape, parts, storage, steps):
    f0 = fields.ideal_fields(shape, 516, mach=1.0, beta=1.0, cfl=0.1 if len(shape) == 2 else 0.2)
    qref, qscale = dev_ref_scale(f0.Q)

    def make(sub):
        return V.make_params(shape=sub, storage=storage, gamma=f0.gamma, tau=0.6, q_ref=qref, q_scale=qscale)

    ref = single_run(V, make(shape), f0.Q, steps)
    got, _ = slab_run(V, S, make, shape, parts, f0.Q, steps)
    assert np.array_equal(got, ref)


def test_slab_populations_at_odd_parity(V, S):
    # the gathered pre-collision populations of every slab cell equal the single domain's
    shape, parts, steps = (8, 5, 16), 2, 3
    f0 = fields.ideal_fields(shape, 517, mach=1.0, cfl=0.2)

    def make(sub):
        return V.make_params(shape=sub, storage="f64", gamma=f0.gamma, tau=0.7)

    with V.Context(make(shape)) as ctx:
        ctx.init_fields(f0.Q)
        ctx.step(steps)
        whole = ctx.populations(np.arange(np.prod(shape)))
    with S.LocalSlabs(make, shape, parts) as g:
        g.init_fields(f0.Q)
        g.step(steps)
        got = np.concatenate([c.populations(np.arange(np.prod(c.shape()))) for c in g.ctxs])
    assert np.array_equal(got, whole)


# ---------------------------------------------------------------------------
# other models
# ---------------------------------------------------------------------------

def test_powell_slabs_equal_the_single_domain(V, S):
    shape = (12, 6, 16)
    f0 = fields.ideal_fields(shape, 518, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(518)
    D = 0.01 * np.abs(f0.Q[5:8]).max() * rng.normal(size=shape)
    Q0 = np.concatenate([f0.Q, D[None]])

    def make(sub):
        return V.make_params(model=V.VLBM_IDEAL_POWELL, shape=sub, storage="f32", gamma=f0.gamma, tau=0.6,
                             tau_d=0.6, tau_m=2.0)

    for steps in (4, 5):
        ref = single_run(V, make(shape), Q0, steps)
        got, _ = slab_run(V, S, make, shape, 3, Q0, steps)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("walls", [True, False])
def test_resistive_channel_slabs_equal_the_single_domain(V, S, walls):
    shape = (8, 12, 20)
    setup = fields.hartmann_setup(shape, 2002, Ha=10.0, U_c=0.05, Re=10.0)
    Q0 = setup.Q.copy()
    rng = np.random.default_rng(2)
    Q0[4:7] += 0.01 * rng.uniform(-1, 1, size=(3,) + shape)

    def make(sub):
        return V.make_params(model=V.VLBM_RESISTIVE, shape=sub, storage="f32",
                             tau=[setup.tau_f, setup.tau_m, setup.tau_m, setup.tau_m],
                             force=setup.force, b_wall=setup.b_wall, walls_y=walls)

    for steps in (6, 7):
        ref = single_run(V, make(shape), Q0, steps)
        got, _ = slab_run(V, S, make, shape, 2, Q0, steps)
        assert np.array_equal(got, ref)
        orc = oracle.resistive_run(Q0, setup.tau_f, setup.tau_m, setup.force, setup.b_wall, walls, steps)
        cs = math.sqrt(1 / 3)
        scales = np.array([1.0, cs, cs, cs] + [np.abs(Q0[4:7]).max()] * 3)
        assert rel_err(got, orc, scales).max() < 1e-5


def test_dissipative_slabs_equal_the_single_domain(V, S):
    shape = (12, 20)
    f0 = fields.ideal_fields(shape, 519, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(519)
    G = 0.01 * rng.normal(size=(12,) + shape)
    Q0 = np.concatenate([f0.Q, G])

    def make(sub):
        return V.make_params(model=V.VLBM_DISSIPATIVE, shape=sub, storage="f64", gamma=f0.gamma, tau=0.6,
                             tau_g=0.7, tau_m=3.0, nu=0.02, eta0=0.03, j_c=0.05, powell=True)

    for steps in (4, 5):
        ref = single_run(V, make(shape), Q0, steps)
        got, _ = slab_run(V, S, make, shape, 3, Q0, steps)
        assert np.array_equal(got, ref)


def test_dissipative_3d_slabs_equal_the_single_domain(V, S):
    shape = (9, 6, 16)
    f0 = fields.ideal_fields(shape, 522, mach=1.0, beta=1.0, cfl=0.2)
    rng = np.random.default_rng(522)
    Q0 = np.concatenate([f0.Q, 0.01 * rng.normal(size=(18,) + shape)])

    def make(sub):
        return V.make_params(model=V.VLBM_DISSIPATIVE, shape=sub, storage="f32", gamma=f0.gamma, tau=0.6,
                             tau_g=0.7, tau_m=3.0, nu=0.02, eta0=0.03, j_c=0.05, powell=True)

    for steps in (4, 5):
        ref = single_run(V, make(shape), Q0, steps)
        got, _ = slab_run(V, S, make, shape, 3, Q0, steps)
        assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------
# the public pack / unpack calls, routed as the one-process-per-GPU driver does
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ["f32", "bf16dev"])
def test_pack_unpack_routed_by_hand_equals_the_group_step(V, S, storage):
    import torch
    shape, parts, steps = (12, 8, 16), 3, 7
    f0 = fields.ideal_fields(shape, 520, mach=1.0, cfl=0.2)
    qref, qscale = dev_ref_scale(f0.Q)
    stream = torch.cuda.Stream()

    def make(sub):
        return V.make_params(shape=sub, storage=storage, gamma=f0.gamma, tau=0.6, q_ref=qref, q_scale=qscale,
                             stream=stream.cuda_stream)

    ref, _ = slab_run(V, S, make, shape, parts, f0.Q, steps)
    ranges = S.split_layers(shape[0], parts)
    ctxs = [V.Context(make((z1 - z0,) + shape[1:])) for z0, z1 in ranges]
    try:
        for c, (z0, z1) in zip(ctxs, ranges):
            assert c.init_fields(np.ascontiguousarray(f0.Q[:, z0:z1])) == V.VLBM_OK
            c.set_slab(True)
        nb = ctxs[0].halo_bytes
        elem = {"f32": 4, "bf16dev": 2}[storage]
        assert nb == 8 * shape[1] * shape[2] * elem  # one slot per lattice per face cell
        send = [(torch.empty(nb, dtype=torch.uint8, device="cuda"), torch.empty(nb, dtype=torch.uint8, device="cuda"))
                for _ in ctxs]
        recv = [(torch.empty(nb, dtype=torch.uint8, device="cuda"), torch.empty(nb, dtype=torch.uint8, device="cuda"))
                for _ in ctxs]
        with torch.cuda.stream(stream):
            for s in range(steps):
                for c in ctxs:
                    assert c.step(1) == V.VLBM_OK
                    # nothing reads a slab before its exchange is unpacked
                    sums = np.empty(8)
                    assert V.load().vlbm_conservation(c.ptr, 0, sums.ctypes.data) == V.VLBM_ERR_STATE
                for r, c in enumerate(ctxs):
                    c.halo_pack(send[r][0].data_ptr(), send[r][1].data_ptr())
                for r in range(parts):
                    hi_to, lo_to, _, _ = S.route(r, parts, s + 1)
                    recv[hi_to][1].copy_(send[r][1])
                    recv[lo_to][0].copy_(send[r][0])
                for r, c in enumerate(ctxs):
                    c.halo_unpack(recv[r][0].data_ptr(), recv[r][1].data_ptr())
        got = np.concatenate([c.moments() for c in ctxs], axis=1)
    finally:
        for c in ctxs:
            c.close()
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------
# the contract
# ---------------------------------------------------------------------------

def test_slab_contract(V, S):
    shape = (8, 6, 16)
    f0 = fields.ideal_fields(shape, 521, mach=1.0, cfl=0.2)
    L = V.load()
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.6)
    with V.Context(p) as ctx:
        ctx.init_fields(f0.Q)
        ctx.step(1)
        assert L.vlbm_set_slab(ctx.ptr, 1) == V.VLBM_ERR_STATE   # mark at an even step count
        ctx.step(1)
        ctx.set_slab(True)
        assert L.vlbm_step(ctx.ptr, 2) == V.VLBM_ERR_STATE       # one step at a time
        assert ctx.step(1) == V.VLBM_OK
        assert L.vlbm_step(ctx.ptr, 1) == V.VLBM_ERR_STATE       # exchange first
        out = np.empty((8,) + shape)
        assert L.vlbm_moments(ctx.ptr, 0, out.ctypes.data) == V.VLBM_ERR_STATE
        assert L.vlbm_set_slab(ctx.ptr, 0) == V.VLBM_ERR_STATE
        # an open face on the decomposed axis is refused; the other axes may open
        assert L.vlbm_set_boundary(ctx.ptr, 4, V.VLBM_BC_EQUILIBRIUM, 0, None) == V.VLBM_ERR_UNSUPPORTED
        assert L.vlbm_set_boundary(ctx.ptr, 0, V.VLBM_BC_EQUILIBRIUM, 0, None) == V.VLBM_OK
        assert L.vlbm_set_boundary(ctx.ptr, 1, V.VLBM_BC_EQUILIBRIUM, 0, None) == V.VLBM_OK
        # re-initialising clears the pending exchange
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        assert ctx.step(1) == V.VLBM_OK
    # slabs that do not fit together are refused before any device work
    a = V.Context(V.make_params(shape=(4, 6, 16), storage="f32", gamma=f0.gamma, tau=0.6))
    b = V.Context(V.make_params(shape=(4, 6, 8), storage="f32", gamma=f0.gamma, tau=0.6))
    try:
        for c in (a, b):
            c.init_fields(np.ascontiguousarray(fields.ideal_fields(c.shape(), 1, mach=1.0, cfl=0.2).Q))
            c.set_slab(True)
        assert L.vlbm_slabs_step((ctypes.c_void_p * 2)(a.ptr, b.ptr), 2, 1) == V.VLBM_ERR_ARG
        assert L.vlbm_slabs_step((ctypes.c_void_p * 2)(a.ptr, a.ptr), 2, 1) == V.VLBM_ERR_ARG
    finally:
        a.close()
        b.close()


def test_slabs_with_open_x_faces_and_solids_equal_the_single_domain(V, S):
    # open faces on the axes the decomposition keeps whole (x here), and homogenised
    # solids given per slab, compose with the exchange: still bit for bit
    import torch
    shape, parts = (12, 8, 16), 3
    f0 = fields.ideal_fields(shape, 523, mach=0.5, beta=10.0, cfl=0.2)
    solid = np.zeros((7,) + shape, dtype=np.float32)
    z, y, x = np.meshgrid(*[np.arange(v) for v in shape], indexing="ij")
    r = np.sqrt((x - 8.0) ** 2 + (y - 4.0) ** 2 + (z - 6.0) ** 2)
    solid[0] = np.clip((r - 3.0) / 1.0 + 0.5, 0.0, 1.0)
    solid[1] = 0.01
    solid[6] = 0.002
    mean = f0.Q.reshape(8, -1).mean(1)

    def make(sub):
        return V.make_params(shape=sub, storage="f64", gamma=f0.gamma, tau=0.6)

    def dress(c, sl):
        c.set_boundary("x-", V.VLBM_BC_EQUILIBRIUM, 0xFF, mean)
        c.set_boundary("x+", V.VLBM_BC_EQUILIBRIUM)
        c.set_solid(sl.data_ptr())

    steps = 7
    sd = torch.from_numpy(solid.reshape(7, -1)).cuda().contiguous()
    with V.Context(make(shape)) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        dress(ctx, sd)
        ctx.step(steps)
        ref = ctx.moments()
    ranges = S.split_layers(shape[0], parts)
    parts_solid = [torch.from_numpy(np.ascontiguousarray(solid[:, z0:z1]).reshape(7, -1)).cuda().contiguous()
                   for z0, z1 in ranges]
    with S.LocalSlabs(make, shape, parts) as g:
        assert g.init_fields(f0.Q) == V.VLBM_OK
        for c, sl in zip(g.ctxs, parts_solid):
            dress(c, sl)
        torch.cuda.synchronize()
        assert g.step(steps) == V.VLBM_OK
        got = g.moments()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("shape", [(24, 20), (10, 12, 16)])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("steps", [5, 6])
def test_slabs_with_open_faces_on_both_kept_axes_equal_the_single_domain(V, S, shape, storage, steps):
    # open faces with mixed Dirichlet / Neumann masks on both x faces (and both y faces in 3-D,
    # whose edges with the x faces give diagonal normals), at both parities and both storages:
    # the slabs fill them after the exchange, the single domain after its step -- bit for bit
    f0 = fields.ideal_fields(shape, 529, mach=0.5, beta=1.0, cfl=0.2)
    mean = f0.Q.reshape(8, -1).mean(1)
    tau = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]

    def make(sub):
        return V.make_params(shape=sub, storage=storage, gamma=f0.gamma, tau=tau)

    def dress(c):
        c.set_boundary("x-", V.VLBM_BC_EQUILIBRIUM, 0b00010011, mean)
        c.set_boundary("x+", V.VLBM_BC_EQUILIBRIUM)
        if len(shape) == 3:  # edges: the x faces' normals turn diagonal there
            c.set_boundary("y-", V.VLBM_BC_EQUILIBRIUM, 0b11100001, mean)
            c.set_boundary("y+", V.VLBM_BC_EQUILIBRIUM)

    with V.Context(make(shape)) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        dress(ctx)
        ctx.step(steps)
        ref = ctx.moments()
    with S.LocalSlabs(make, shape, 2) as g:
        assert g.init_fields(f0.Q) == V.VLBM_OK
        for c in g.ctxs:
            dress(c)
        assert g.step(steps) == V.VLBM_OK
        got = g.moments()
    assert np.array_equal(got, ref)
