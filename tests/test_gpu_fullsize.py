"""Parity at the full workload sizes, on outputs the oracle computes cell by cell.

* 512^3 ideal MHD, 8 x D3Q7, FP32 (the benchmark's workload and launch
  configuration): the populations of sampled cells after one step equal the
  oracle's collision of the gathered pre-step populations of their upstream
  neighbours, at both AA parities; domain sums stay conserved.  The same
  one-step check for the FP16 and BF16 deviation forms at 512^3, up to the
  storage rounding of the deviations.
* 256 x 128 x 128 resistive channel (D3Q19 + 3 x D3Q7, walls): the same
  one-step check, including cells next to the walls (bounce-back and the
  magnetic wall equilibrium); mass stays conserved.
* 64 batched 2-D domains: whole-domain moments of a subset against the
  oracle after several steps.
* Both full-size workloads over many steps, through the launch configuration
  the benchmark uses (own stream, so 32-step chunks replay a captured graph):
  the populations of sampled cells after n steps against the oracle run on the
  cell's light cone.  On D3Q7 a cell after n steps depends only on the cells
  within L1 distance n, on D3Q19 within L-infinity distance n, so the oracle
  on the periodic (2n+1) box centred on the cell (for the channel: the full
  wall-to-wall height, the walls being part of the box) gives that cell
  exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu

D3Q7 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
D3Q19 = D3Q7 + [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
                (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def shifted(cell, c, shape, sign=-1):
    nz, ny, nx = shape
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    x = (x + sign * c[0]) % nx
    y = (y + sign * c[1]) % ny
    z = (z + sign * c[2]) % nz
    return x + nx * (y + ny * z)


def sample_cells(shape, rng, n):
    nz, ny, nx = shape
    N = nx * ny * nz
    corners = [0, nx - 1, (ny - 1) * nx, N - 1, N - nx, nx * ny * (nz - 1), nx // 2 + nx * (ny // 2)]
    return np.unique(np.concatenate([rng.choice(N, size=n, replace=False), corners])).astype(np.int64)


@pytest.fixture(scope="module")
def ideal512(V):
    import torch
    shape = (512, 512, 512)
    f0 = fields.ideal_fields(shape, 3003, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4,
                             device=torch.device("cuda"))
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.51)
    ctx = V.Context(p)
    assert V.vlbm_init_fields_device(ctx.ptr, 0, f0.Q.data_ptr()) == V.VLBM_OK
    sums0 = ctx.conservation()
    del f0
    torch.cuda.empty_cache()
    yield ctx, shape, p.gamma, sums0
    ctx.close()


@pytest.mark.parametrize("parity", [1, 0])
def test_ideal_512cubed_sampled_step(V, ideal512, parity):
    ctx, shape, gamma, _ = ideal512
    if (ctx.step_count & 1) != parity:
        ctx.step(1)
    rng = np.random.default_rng(11 + parity)
    cells = sample_cells(shape, rng, 48)
    src = {x: [shifted(int(x), c, shape) for c in D3Q7] for x in cells}
    uniq = np.array(sorted({s for v in src.values() for s in v}), dtype=np.int64)
    pre = dict(zip(uniq.tolist(), ctx.populations(uniq)))
    ctx.step(1)
    post = ctx.populations(cells)
    assert ctx.sync() == V.VLBM_OK
    post_coll = {s: oracle.ideal_collide_cell(3, gamma, 0.51, pre[s].reshape(8, 7)) for s in uniq.tolist()}
    expect = np.zeros_like(post)
    for r, x in enumerate(cells):
        for k in range(8):
            for i in range(7):
                expect[r, k * 7 + i] = post_coll[src[x][i]][k, i]
    scale = np.abs(expect).reshape(len(cells), 8, 7).max(axis=(0, 2))
    err = np.abs(post - expect).reshape(len(cells), 8, 7).max(axis=(0, 2)) / scale
    assert err.max() < 1e-5, err


@pytest.mark.parametrize("storage,ulp", [("f16dev", 2.0 ** -11), ("bf16dev", 2.0 ** -8)])
def test_deviation_storage_512cubed_sampled_step(V, storage, ulp):
    # the 16-bit forms at the benchmark's size and launch configuration (the persistent
    # bulk-copy pairs kernel, 912 CTAs walking 2M row tiles): one step of sampled cells
    # at both parities equals the oracle collision of the gathered upstream populations
    # up to the storage rounding of the deviations (as at the small sizes)
    import torch
    shape = (512, 512, 512)
    f0 = fields.ideal_fields(shape, 3003, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4,
                             device=torch.device("cuda"))
    flat = f0.Q.reshape(8, -1)
    qref = flat.mean(1).cpu().numpy()
    qscale = (flat - flat.mean(1, keepdim=True)).abs().amax(1).clamp_min(1e-30).cpu().numpy()
    p = V.make_params(shape=shape, storage=storage, gamma=f0.gamma, tau=0.51, q_ref=qref, q_scale=qscale)
    w = np.array([1 / 4] + [1 / 8] * 6)
    with V.Context(p) as ctx:
        assert V.vlbm_init_fields_device(ctx.ptr, 0, f0.Q.data_ptr()) == V.VLBM_OK
        del f0, flat
        torch.cuda.empty_cache()
        ctx.step(3)
        for parity in (1, 0):
            rng = np.random.default_rng(21 + parity)
            cells = sample_cells(shape, rng, 40)
            src = {x: [shifted(int(x), c, shape) for c in D3Q7] for x in cells}
            uniq = np.array(sorted({u for v in src.values() for u in v}), dtype=np.int64)
            pre = dict(zip(uniq.tolist(), ctx.populations(uniq)))
            assert (ctx.step_count & 1) == parity
            ctx.step(1)
            post = ctx.populations(cells)
            assert ctx.sync() == V.VLBM_OK
            coll = {u: oracle.ideal_collide_cell(3, p.gamma, 0.51, pre[u].reshape(8, 7)) for u in uniq.tolist()}
            for r, x in enumerate(cells.tolist()):
                exp = np.array([[coll[src[x][i]][k, i] for i in range(7)] for k in range(8)])
                g_exp = (exp - w[None, :] * qref[:, None]) / qscale[:, None]
                g_got = (post[r].reshape(8, 7) - w[None, :] * qref[:, None]) / qscale[:, None]
                tol = ulp * np.abs(g_exp) + 2e-3 * ulp * 64 * np.abs(g_exp).max()
                assert (np.abs(g_got - g_exp) <= tol).all(), (storage, parity, x, np.abs(g_got - g_exp).max())


def test_ideal_512cubed_conservation(V, ideal512):
    ctx, shape, gamma, sums0 = ideal512
    ctx.step(10)
    assert ctx.sync() == V.VLBM_OK
    s = ctx.conservation()
    # FP32 storage: every population is rounded each step; the sums of the
    # conserved fields drift only by that rounding (relative to sum |Q|)
    scale = np.array([abs(v) for v in sums0])
    scale[1:4] = max(scale[1:4].max(), 1e-3 * scale[0])
    scale[5:8] = max(scale[5:8].max(), 1e-3 * scale[0])
    assert (np.abs(s - sums0) / scale).max() < 1e-5


def test_channel_full_size_sampled_step(V):
    import torch
    shape = (128, 128, 256)  # nz, ny, nx: 256 x 128 x 128 channel, walls at y = 0, 127
    setup = fields.hartmann_setup(shape, 2002, Ha=10.0)
    p = V.make_params(model=V.VLBM_RESISTIVE, shape=shape, storage="f32",
                      tau=[setup.tau_f, setup.tau_m, setup.tau_m, setup.tau_m], force=setup.force,
                      b_wall=setup.b_wall, walls_y=True)
    nz, ny, nx = shape
    with V.Context(p) as ctx:
        Qd = torch.from_numpy(setup.Q).cuda()
        assert V.vlbm_init_fields_device(ctx.ptr, 0, Qd.data_ptr()) == V.VLBM_OK
        del Qd
        sums0 = ctx.conservation()
        ctx.step(37)  # develop the flow a little; the next kernel has odd parity
        rng = np.random.default_rng(3)
        cells = list(sample_cells(shape, rng, 40))
        # add cells next to both walls
        for _ in range(12):
            x, z = int(rng.integers(nx)), int(rng.integers(nz))
            for y in (1, ny - 2):
                cells.append(x + nx * (y + ny * z))
        cells = np.array(sorted(set(c for c in cells if 0 < (c // nx) % ny < ny - 1)), dtype=np.int64)

        def is_wall(c):
            return (c // nx) % ny in (0, ny - 1)

        need = set(cells.tolist())
        for x in cells:
            for c in D3Q19:
                s = shifted(int(x), c, shape)
                if not is_wall(s):
                    need.add(s)
        uniq = np.array(sorted(need), dtype=np.int64)
        pre = dict(zip(uniq.tolist(), ctx.populations(uniq)))
        ctx.step(1)
        post = ctx.populations(cells)
        assert ctx.sync() == V.VLBM_OK
        s1 = ctx.conservation()
    coll = {s: oracle.resistive_collide_cell(setup.tau_f, setup.tau_m, setup.force, pre[s])
            for s in uniq.tolist()}
    w7 = [0.25] + [0.125] * 6
    expect = np.zeros_like(post)
    for r, x in enumerate(cells.tolist()):
        for i, c in enumerate(D3Q19):
            s = shifted(x, c, shape)
            if is_wall(s):  # halfway bounce-back: own post-collision, opposite direction
                opp = D3Q19.index(tuple(-v for v in c))
                expect[r, i] = coll[x][opp]
            else:
                expect[r, i] = coll[s][i]
        for b in range(3):
            for i, c in enumerate(D3Q7):
                s = shifted(x, c, shape)
                j = 19 + 7 * b + i
                expect[r, j] = w7[i] * setup.b_wall[b] if is_wall(s) else coll[s][j]
    scale = np.array([np.abs(expect[:, :19]).max()] * 19 + [np.abs(expect[:, 19:]).max()] * 21)
    err = (np.abs(post - expect) / scale).max(0)
    assert err.max() < 1e-5, err
    assert abs(s1[0] - sums0[0]) < 1e-5 * sums0[0]


def test_batched_64_domains_subset(V):
    import torch
    specs = fields.batch_specs(64, 4004)
    params, inits = [], []
    for sp in specs:
        n = sp["side"]
        f0 = fields.ideal_fields((n, n), sp["seed"], gamma=sp["gamma"], mach=sp["mach"], cfl=0.1,
                                 device=torch.device("cuda"))
        inits.append(f0)
        params.append(V.make_params(shape=(n, n), storage="f32", gamma=sp["gamma"], tau=0.51))
    steps = 6
    with V.Context(params, batch=True) as ctx:
        for d, f0 in enumerate(inits):
            assert V.vlbm_init_fields_device(ctx.ptr, d, f0.Q.data_ptr()) == V.VLBM_OK
        ctx.autotune(4)
        ctx.step(steps)
        assert ctx.sync() == V.VLBM_OK
        by_size = {}
        for d, sp in enumerate(specs):
            by_size.setdefault(sp["side"], d)
        for side, d in sorted(by_size.items()):
            got = ctx.moments(d)
            Q0 = inits[d].Q.cpu().numpy()
            ref = oracle.ideal_run(Q0, specs[d]["gamma"], 0.51, steps, nthreads=8)
            scl = np.array([np.abs(Q0[0]).max()] + [np.abs(Q0[1:4]).max()] * 3 + [np.abs(Q0[4]).max()]
                           + [np.abs(Q0[5:8]).max()] * 3)
            err = np.abs(got - ref).reshape(8, -1).max(1) / scl
            assert err.max() < 1e-5, (side, err)


def test_ideal_512cubed_light_cones_after_40_steps(V):
    # The benchmark's workload and launch configuration: 512^3, 8 x D3Q7, FP32,
    # Mach 2, beta 1, own stream; 5 single steps then 35 (one captured 32-step
    # graph and three single launches).  Eight sampled cells (corners, faces,
    # interior) against the oracle on their periodic 81^3 light-cone boxes.
    import torch
    n, warm, steps = 512, 5, 35
    total = warm + steps
    shape = (n, n, n)
    f0 = fields.ideal_fields(shape, 3003, mach=2.0, beta=1.0, cfl=0.2, k_rho=4, k_u=4, k_b=4,
                             device=torch.device("cuda"))
    Q, gamma = f0.Q, f0.gamma
    del f0
    scale = Q.abs().reshape(8, -1).amax(1).cpu().numpy()
    samples = [(0, 0, 0), (n - 1, n - 1, n - 1), (n // 2, n // 2, n // 2), (7, 300, 511), (511, 0, 256),
               (123, 456, 78), (400, 17, 3), (256, 511, 0)]
    h = total
    boxes = []
    for (zc, yc, xc) in samples:
        idx = [torch.arange(v - h, v + h + 1, device="cuda") % n for v in (zc, yc, xc)]
        boxes.append(Q[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]].cpu().numpy())
    stream = torch.cuda.Stream()
    p = V.make_params(shape=shape, storage="f32", gamma=gamma, tau=0.51, stream=stream.cuda_stream)
    with V.Context(p) as ctx:
        assert V.vlbm_init_fields_device(ctx.ptr, 0, Q.data_ptr()) == V.VLBM_OK
        del Q
        torch.cuda.empty_cache()
        ctx.step(warm)
        l0 = ctx.launches
        ctx.step(steps)
        assert ctx.launches - l0 == steps
        assert ctx.sync() == V.VLBM_OK
        got = ctx.populations([xc + n * (yc + n * zc) for (zc, yc, xc) in samples])
    for Qb, g in zip(boxes, got):
        fb = oracle.ideal_init(Qb, gamma)
        for _ in range(total):
            fb = oracle.ideal_step(fb, gamma, 0.51, nthreads=8)
        expect = fb[:, :, h, h, h].reshape(-1)
        tol = 1e-5 * np.repeat(scale, 7)
        assert np.all(np.abs(g - expect) <= tol), np.abs(g - expect).reshape(8, 7).max(1) / scale


def test_channel_full_size_light_cones_after_40_steps(V):
    # 256 x 128 x 128 channel (walls at y = 0, 127), the benchmark's fields and
    # launch configuration (own stream), 4 + 36 steps; sampled cells on the walls,
    # next to them and inside, against the oracle on boxes of 81 x 128 x 81 cells
    # (periodic in x and z, the whole height in y).
    import torch
    shape = (128, 128, 256)
    nz, ny, nx = shape
    setup = fields.hartmann_setup(shape, 2002, Ha=10.0)
    warm, steps = 4, 36
    total = warm + steps
    h = total
    stream = torch.cuda.Stream()
    p = V.make_params(model=V.VLBM_RESISTIVE, shape=shape, storage="f32",
                      tau=[setup.tau_f, setup.tau_m, setup.tau_m, setup.tau_m], force=setup.force,
                      b_wall=setup.b_wall, walls_y=True, stream=stream.cuda_stream)
    samples = [(0, 0, 0), (5, 1, 200), (127, 126, 255), (64, 64, 128), (100, 2, 7), (31, 125, 99),
               (64, 127, 31), (10, 70, 250)]
    with V.Context(p) as ctx:
        Qd = torch.from_numpy(setup.Q).cuda()
        assert V.vlbm_init_fields_device(ctx.ptr, 0, Qd.data_ptr()) == V.VLBM_OK
        del Qd
        ctx.step(warm)
        ctx.step(steps)
        assert ctx.sync() == V.VLBM_OK
        got = ctx.populations([xc + nx * (yc + ny * zc) for (zc, yc, xc) in samples])
    for (zc, yc, xc), g in zip(samples, got):
        iz = (np.arange(zc - h, zc + h + 1)) % nz
        ix = (np.arange(xc - h, xc + h + 1)) % nx
        Qb = np.ascontiguousarray(setup.Q[:, iz][:, :, :, ix])
        f, gm = oracle.resistive_init(Qb, setup.force)
        for _ in range(total):
            f, gm = oracle.resistive_step(f, gm, setup.tau_f, setup.tau_m, setup.force, setup.b_wall, True,
                                          nthreads=8)
        if yc in (0, ny - 1):
            # a wall cell: its flow slots are never used, its magnetic populations are the wall equilibrium
            expect_g = gm[:, :, h, yc, h].reshape(-1)
            err = np.abs(g[19:] - expect_g).max() / np.abs(setup.b_wall).max()
            assert err < 1e-5, (zc, yc, xc, err)
            continue
        expect = np.concatenate([f[:, h, yc, h], gm[:, :, h, yc, h].reshape(-1)])
        scale = np.array([np.abs(f[:, h]).max()] * 19 + [max(np.abs(gm).max(), 1e-30)] * 21)
        err = (np.abs(g - expect) / scale).max()
        assert err < 1e-5, (zc, yc, xc, err)
