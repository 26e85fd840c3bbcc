"""Static equilibrium boundaries (sec. 2.4, "Static boundaries") on the GPU
against the FP64 oracle: open faces with Dirichlet / Neumann boundary states,
alone and with homogenised solids, through plain launches and captured graphs,
at both AA parities (boundary cells, edges and corners included).

Tolerances as for the ideal model: FP64 storage 1e-12, FP32 storage 1e-5,
relative to each field's maximum.
"""
import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu

TAU = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]
ALL = 0xFF


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def _faces(Q, dim, open_axes):
    # each open face its own mix: x- Dirichlet inflow of the mean state, x+ zero
    # gradient, y- Dirichlet rho and B only, y+ Dirichlet e only, z- / z+ mixed
    mean = Q.reshape(8, -1).mean(1)
    corner = Q.reshape(8, -1)[:, 0]
    spec = [(ALL, mean), (0, None), (0b11100001, mean), (0b10000, corner), (0b1001, corner), (0b100110, mean)]
    return [spec[f] if (f // 2) in open_axes else None for f in range(2 * dim)]


def _apply(ctx, V, faces):
    for f, sp in enumerate(faces):
        if sp is not None:
            ctx.set_boundary(f, V.VLBM_BC_EQUILIBRIUM, sp[0], sp[1])


def field_errors(got, ref):
    scale = np.maximum(np.abs(ref).reshape(8, -1).max(1), 1e-300)
    return np.abs(got - ref).reshape(8, -1).max(1) / scale


@pytest.mark.parametrize("shape,open_axes", [((24, 40), (0, 1)), ((12, 40), (0,)), ((8, 12, 20), (0, 1, 2)),
                                             ((6, 9, 16), (2,)), ((5, 7, 12), (0, 2))])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("steps", [4, 5])
def test_open_faces_match_oracle(V, shape, open_axes, storage, tol, steps):
    f0 = fields.ideal_fields(shape, 61, mach=0.5, beta=1.0, cfl=0.2)
    faces = _faces(f0.Q, len(shape), open_axes)
    p = V.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=TAU)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        _apply(ctx, V, faces)
        ctx.step(steps)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    ref = oracle.open_run(f0.Q, f0.gamma, TAU, faces, steps)
    err = field_errors(got, ref)
    assert err.max() < tol, err


def test_boundary_and_corner_populations_at_odd_parity(V):
    shape = (6, 8, 10)
    f0 = fields.ideal_fields(shape, 62, mach=0.5, beta=1.0, cfl=0.2)
    faces = _faces(f0.Q, 3, (0, 1, 2))
    f = oracle.ideal_init(f0.Q, f0.gamma)
    for _ in range(3):
        f = oracle.open_step(f, f0.gamma, TAU, faces)
    nx, ny, nz = 10, 8, 6
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, 4, 3), (nx - 1, 0, 2), (5, 0, 0), (4, 3, 2), (5, ny - 1, 3)]
    cells = np.array([x + nx * (y + ny * z) for (x, y, z) in pts], dtype=np.int64)
    p = V.make_params(shape=shape, storage="f64", gamma=f0.gamma, tau=TAU)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        _apply(ctx, V, faces)
        ctx.step(3)
        got = ctx.populations(cells)
    ref = f.reshape(8 * 7, -1)[:, cells].T
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_open_faces_with_solids_match_oracle(V, storage, tol):
    import torch
    shape = (8, 12, 20)
    f0 = fields.ideal_fields(shape, 63, mach=0.5, beta=1.0, cfl=0.2)
    faces = _faces(f0.Q, 3, (0, 1))
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    phi = np.sqrt((x - 10.0) ** 2 + (y - 5.5) ** 2 + (z - 3.5) ** 2) - 2.5
    solid = np.zeros((7,) + shape)
    solid[0] = oracle.hlbm_porosity(phi, 1.0)
    solid[1] = -0.002 * (y - 5.5)
    solid[2] = 0.002 * (x - 10.0)
    solid[4] = 0.02
    solid = solid.astype(np.float32)
    sd = torch.from_numpy(solid).cuda()
    p = V.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=TAU)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        _apply(ctx, V, faces)
        ctx.set_solid(sd.data_ptr())
        ctx.step(5)
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    ref = oracle.open_run(f0.Q, f0.gamma, TAU, faces, 5, solid=solid.astype(np.float64))
    assert field_errors(got, ref).max() < tol


def test_captured_graphs_match_oracle_and_count_two_launches_per_step(V):
    # on a torch stream the steps run as captured 32-step graphs; the fill pass is
    # captured with the step (two kernels per step) and the launch count says so
    import torch
    shape = (10, 16, 24)
    f0 = fields.ideal_fields(shape, 64, mach=0.5, beta=1.0, cfl=0.2)
    faces = _faces(f0.Q, 3, (0, 2))
    stream = torch.cuda.Stream()
    p = V.make_params(shape=shape, storage="f64", gamma=f0.gamma, tau=TAU, stream=stream.cuda_stream)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        _apply(ctx, V, faces)
        before = V.vlbm_launch_count(ctx.ptr)
        ctx.step(1)
        ctx.step(64)  # an odd start: both parities of graph
        launched = V.vlbm_launch_count(ctx.ptr) - before
        got = ctx.moments()
        assert ctx.sync() == V.VLBM_OK
    assert launched == 2 * 65
    ref = oracle.open_run(f0.Q, f0.gamma, TAU, faces, 65, nthreads=4)
    assert field_errors(got, ref).max() < 1e-12


def test_closing_the_faces_returns_to_the_periodic_scheme_and_api_checks(V):
    shape = (12, 16)
    f0 = fields.ideal_fields(shape, 65, mach=0.5, beta=1.0, cfl=0.2)
    p = V.make_params(shape=shape, storage="f64", gamma=f0.gamma, tau=TAU)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        ctx.set_boundary("x-", V.VLBM_BC_EQUILIBRIUM, ALL, f0.Q[:, 0, 0])
        ctx.set_boundary("x+", V.VLBM_BC_EQUILIBRIUM)
        ctx.set_boundary("x-", V.VLBM_BC_PERIODIC)
        ctx.set_boundary("x+", V.VLBM_BC_PERIODIC)
        ctx.step(6)
        got = ctx.moments()
    assert field_errors(got, oracle.ideal_run(f0.Q, f0.gamma, TAU, 6)).max() < 1e-12
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        ctx.set_boundary("y-", V.VLBM_BC_EQUILIBRIUM)
        with pytest.raises(V.VlbmError):
            ctx.step(1)  # y+ still periodic
    with V.Context(p) as ctx:
        for bad in (lambda: ctx.set_boundary(4, V.VLBM_BC_EQUILIBRIUM),  # no z faces in 2-D
                    lambda: ctx.set_boundary("x-", 7),
                    lambda: ctx.set_boundary("x-", V.VLBM_BC_EQUILIBRIUM, 0x100, np.ones(8)),
                    lambda: ctx.set_boundary("x-", V.VLBM_BC_EQUILIBRIUM, 1, None)):
            with pytest.raises(V.VlbmError):
                bad()
    thin = V.make_params(shape=(2, 16), storage="f64")
    with V.Context(thin) as ctx:
        with pytest.raises(V.VlbmError):
            ctx.set_boundary("y-", V.VLBM_BC_EQUILIBRIUM)  # fewer than 3 cells
    for params in (V.make_params(shape=(4, 8, 16), storage="f16dev"),
                   V.make_params(model=V.VLBM_IDEAL_POWELL, shape=(4, 8, 16))):
        with V.Context(params) as ctx:
            with pytest.raises(V.VlbmError):
                ctx.set_boundary("x-", V.VLBM_BC_EQUILIBRIUM)


def test_full_size_open_box_sampled_against_light_cones(V):
    # The 512^3 benchmark run with open faces (x- a Dirichlet reservoir at the mean
    # state, the other faces zero-gradient), on its own stream (captured graphs),
    # 4 + 20 steps.  Per step a cell depends on cells within L-inf distance 1 (the
    # streaming, and the fill's copy along the discrete normal), so the oracle on
    # the box of half-width n around a sample, clipped to the domain, gives the
    # sample exactly: a clipped side keeps the domain's face, the opposite side of
    # that axis is an artificial zero-gradient face n cells away.
    import torch
    n, steps = 512, 24
    shape = (n, n, n)
    f0 = fields.ideal_fields(shape, 3003, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4,
                             device=torch.device("cuda"))
    Q = f0.Q
    mean = Q.reshape(8, -1).mean(1).cpu().numpy()
    scale = Q.abs().reshape(8, -1).amax(1).cpu().numpy()
    spec = [(ALL, mean)] + [(0, None)] * 5
    samples = [(0, 256, 256), (n - 1, 100, 300), (0, 0, 0), (n - 1, n - 1, n - 1), (0, 0, 200),
               (300, n - 3, 40), (17, 480, 2), (256, 256, 256)]  # (x, y, z)
    boxes = []
    for s in samples:
        lo = [max(0, v - steps) for v in s]
        hi = [min(n - 1, v + steps) for v in s]
        faces = []
        for a in range(3):
            if lo[a] == 0 or hi[a] == n - 1:
                faces += [spec[2 * a] if lo[a] == 0 else (0, None), spec[2 * a + 1] if hi[a] == n - 1 else (0, None)]
            else:
                faces += [None, None]
        Qb = Q[:, lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1].cpu().numpy()
        boxes.append((Qb, faces, [s[a] - lo[a] for a in range(3)]))

    stream = torch.cuda.Stream()
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.51, stream=stream.cuda_stream)
    with V.Context(p) as ctx:
        assert V.vlbm_init_fields_device(ctx.ptr, 0, Q.data_ptr()) == V.VLBM_OK
        _apply(ctx, V, spec)
        ctx.step(4)
        ctx.step(steps - 4)
        assert ctx.sync() == V.VLBM_OK
        got = ctx.populations([x + n * (y + n * z) for (x, y, z) in samples])
    del Q

    for (Qb, faces, at), g in zip(boxes, got):
        fb = oracle.ideal_init(Qb, f0.gamma)
        for _ in range(steps):
            fb = oracle.open_step(fb, f0.gamma, 0.51, faces, nthreads=8)
        ref = fb[:, :, at[2], at[1], at[0]].reshape(-1)
        tol = 1e-5 * np.repeat(scale, 7)
        assert np.all(np.abs(g - ref) <= tol), np.abs(g - ref).reshape(8, 7).max(1) / scale
