"""Learned flux closure on the GPU against the FP64 reference.

The kernels' type contract, which the reference is evaluated under: BF16
weights and input features; hidden activations (a1, a2) and hidden-layer
gradients (gz2, gz1) kept in BF16 between layers; every sum accumulated in
FP32 (the reference: FP64).  The reference takes the same BF16-rounded
weights, features and output gradient, and rounds its hidden activations and
gradients to BF16 where the kernels store them (``store=bf16_round``).
Tolerances: network outputs and parameter gradients within 1e-2 of the
largest magnitude of that reference; the corrected lattice Boltzmann step
(FP32 storage) within 1e-5 like every FP32 step.
"""
import numpy as np
import pytest

import oracle
from oracle import closure_ref as C
from paper_2606_00641_gb300 import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_00641_gb300 import vlbm
    vlbm.load()
    return vlbm


def bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def flat_params(p):
    return np.concatenate([p[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def unflat(flat):
    shapes = [("W1", (32, 8, 27)), ("b1", (32,)), ("W2", (32, 32, 27)), ("b2", (32,)),
              ("W3", (24, 32, 27)), ("b3", (24,))]
    out, off = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = flat[off:off + n].reshape(shp).astype(np.float64)
        off += n
    return out


def setup_closure(V, shape, seed, last_scale=1.0):
    import torch
    f0 = fields.ideal_fields(shape, seed, mach=1.5, beta=1.0, cfl=0.2)
    Q = f0.Q
    mu = Q.reshape(8, -1).mean(1)
    sigma = Q.reshape(8, -1).std(1) + 1e-3 * np.abs(Q).reshape(8, -1).max(1) + 1e-12
    out_scale = 1e-3 * np.abs(Q).reshape(8, -1).max(1) + 1e-12
    cl = V.Closure(shape, f0.gamma, 0.55, mu, sigma, out_scale, lr=1e-3)
    rng = np.random.default_rng(seed)
    p = C.init_params(rng, hidden=32, last_scale=last_scale)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(size=p[k].shape) * 0.05
    cl.set_weights(flat_params(p))
    pw = unflat(np.asarray(bf16_round(flat_params(p))))
    Qd = torch.from_numpy(Q).cuda()
    return cl, f0, Qd, pw, mu, sigma, out_scale


# grids per convolution kernel: tcgen05/TMEM (nx % 8, ny % 16, nz % 4; weight
# gradient nz % 2), shared-memory mma.sync (nx % 16, ny % 8), global-load
# mma.sync (anything with nx % 16).  (12, 80, 96) has 180 convolution tiles
# of 8 x 16 x 4 cells and 360 weight-gradient tiles of 8 x 16 x 2: more than
# one tile per persistent CTA, so the staging pipelines run.
CONV_SHAPES = [(4, 16, 16), (2, 32, 48), (6, 8, 32), (4, 6, 16), (12, 80, 96)]


@pytest.mark.parametrize("shape", CONV_SHAPES)
def test_closure_forward_matches_reference(V, shape):
    import torch
    cl, f0, Qd, pw, mu, sigma, out_scale = setup_closure(V, shape, 51)
    dphi = torch.empty((np.prod(shape), 24), dtype=torch.float32, device="cuda")
    cl.forward(Qd.data_ptr(), dphi.data_ptr())
    got = dphi.cpu().numpy().T.reshape((24,) + shape)
    x = bf16_round(C.features(f0.Q, mu, sigma))
    y, _ = C.net_forward(pw, x, store=bf16_round)
    ref = C.dphi_from_output(y, out_scale).reshape((24,) + shape)
    for k in range(8):
        g, r = got[3 * k:3 * k + 3], ref[3 * k:3 * k + 3]
        assert np.abs(g - r).max() < 1e-2 * np.abs(r).max(), (k, np.abs(g - r).max() / np.abs(r).max())
    cl.close()


@pytest.mark.parametrize("shape", CONV_SHAPES)
def test_closure_backward_matches_reference(V, shape):
    import torch
    cl, f0, Qd, pw, mu, sigma, out_scale = setup_closure(V, shape, 52)
    N = int(np.prod(shape))
    rng = np.random.default_rng(9)
    gy = rng.normal(size=(N, 24)).astype(np.float32)
    got = unflat(cl.backward(Qd.data_ptr(), torch.from_numpy(gy).cuda().data_ptr()))
    x = bf16_round(C.features(f0.Q, mu, sigma))
    y, cache = C.net_forward(pw, x, store=bf16_round)
    ref = C.net_backward(pw, cache, bf16_round(gy).T.reshape((24,) + shape), store=bf16_round)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.abs(got[name] - ref[name]).max() / np.abs(ref[name]).max()
        assert err < 1e-2, (name, err)
    cl.close()


@pytest.mark.parametrize("shape", [(6, 8, 32), (4, 16, 16)])
def test_corrected_step_matches_reference(V, shape):
    import torch
    cl, f0, Qd, pw, mu, sigma, out_scale = setup_closure(V, shape, 53)
    N = int(np.prod(shape))
    dphi = torch.empty((N, 24), dtype=torch.float32, device="cuda")
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.55)
    with V.Context(p) as ctx:
        assert ctx.init_fields(f0.Q) == V.VLBM_OK
        ctx.step(3)                      # an odd parity for the corrected step
        Q3 = ctx.moments()
        s3 = ctx.conservation()
        cl.forward(torch.from_numpy(Q3).cuda().data_ptr(), dphi.data_ptr())
        V.vlbm_set_closure(ctx.ptr, cl)
        f3 = ctx.populations(np.arange(N)).T.reshape((8, 7) + shape)
        ctx.step(1)
        V.vlbm_set_closure(ctx.ptr, None)
        got = ctx.moments()
        s4 = ctx.conservation()
        assert ctx.sync() == V.VLBM_OK
    dp = dphi.cpu().numpy().astype(np.float64).T.reshape((8, 3) + shape)
    f4 = C.corrected_step(f3, f0.gamma, 0.55, dp, lambda a, g, t: oracle.ideal_step(a, g, t))
    ref = f4.sum(1)
    scale = np.abs(f0.Q).reshape(8, -1).max(1)
    assert (np.abs(got - ref).reshape(8, -1).max(1) / scale).max() < 1e-5
    # the correction moves fluxes only: every domain sum stays put
    assert (np.abs(s4 - s3) / np.abs(f0.Q).reshape(8, -1).sum(1)).max() < 1e-6
    cl.close()


def test_restriction_is_a_block_average(V):
    import torch
    rng = np.random.default_rng(3)
    Qf = rng.normal(size=(8, 8, 12, 16))
    Qc = torch.zeros((8, 2, 3, 4), dtype=torch.float64, device="cuda")
    V.vlbm_restrict(torch.from_numpy(Qf).cuda().data_ptr(), (8, 12, 16), 4, Qc.data_ptr())
    torch.cuda.synchronize()
    ref = Qf.reshape(8, 2, 4, 3, 4, 4, 4).mean(axis=(2, 4, 6))
    np.testing.assert_allclose(Qc.cpu().numpy(), ref, rtol=1e-14, atol=1e-15)


def test_training_learns_a_representable_flux(V):
    # target: one plain step followed by an extra flux divergence that is a
    # smooth function of the state, which the network can represent
    import torch
    shape = (8, 16, 16)
    N = int(np.prod(shape))
    f0 = fields.ideal_fields(shape, 54, mach=1.0, beta=1.0, cfl=0.2)
    Q0 = f0.Q
    mu = Q0.reshape(8, -1).mean(1)
    sigma = Q0.reshape(8, -1).std(1) + 1e-12
    out_scale = 0.02 * sigma
    target_phi = np.zeros((8, 3) + shape)
    for k in range(8):
        for a in range(3):
            target_phi[k, a] = 0.01 * sigma[k] * np.tanh((Q0[(k + a + 1) % 8] - mu[(k + a + 1) % 8])
                                                          / sigma[(k + a + 1) % 8])
    f = oracle.ideal_init(Q0, f0.gamma)
    plain = oracle.ideal_step(f, f0.gamma, 0.55).sum(1)
    Qt = plain - np.stack([C.centred_divergence3(target_phi[k]) for k in range(8)])
    cl = V.Closure(shape, f0.gamma, 0.55, mu, sigma, out_scale, lr=3e-3)
    rng = np.random.default_rng(0)
    cl.set_weights(flat_params(C.init_params(rng, last_scale=0.1)))
    Q0d = torch.from_numpy(Q0).cuda()
    Qtd = torch.from_numpy(Qt).cuda()
    losses = [cl.train_step(Q0d.data_ptr(), Qtd.data_ptr()) for _ in range(300)]
    assert np.isfinite(losses).all()
    assert np.mean(losses[-10:]) < 0.2 * losses[0], (losses[0], losses[-10:])
    cl.close()


def test_trained_closure_beats_plain_coarse_run(V):
    # fine 128^3 runs restricted 4x to 32^3; in-the-loop training with early
    # stopping on seed 5100; two held-out seeds must show a lower error of the
    # corrected coarse run than of the plain coarse run after 32 coarse steps
    from paper_2606_00641_gb300 import closure
    r = closure.run_experiment(fine_shape=(128, 128, 128), train_seeds=tuple(range(5000, 5008)),
                               val_seed=5100, test_seeds=(5101, 5102), episodes=120)
    try:
        assert r["best_val"] <= r["history"][0][1]
        for t in r["tests"]:
            assert t["status"] == [0, 0], t
            assert t["rel_l2_closure_coarse"] < 0.95 * t["rel_l2_plain_coarse"], t
    finally:
        r["closure"].close()


def _dp_problem(V, seed, lr=1e-3):
    import torch
    shape = (4, 16, 16)
    f0 = fields.ideal_fields(shape, seed, mach=1.0, beta=1.0, cfl=0.2)
    Q0 = f0.Q
    mu = Q0.reshape(8, -1).mean(1)
    sigma = Q0.reshape(8, -1).std(1) + 1e-3 * np.abs(Q0).reshape(8, -1).max(1) + 1e-12
    out_scale = 1e-2 * sigma
    rng = np.random.default_rng(seed)
    Qt = Q0 * (1.0 + 1e-3 * rng.normal(size=Q0.shape))  # any target: the loss has a gradient
    w0 = flat_params(C.init_params(rng, last_scale=0.1))
    make_cl = lambda: V.Closure(shape, f0.gamma, 0.55, mu, sigma, out_scale, lr=lr)
    p = V.make_params(shape=shape, storage="f32", gamma=f0.gamma, tau=0.55)
    return shape, Q0, torch.from_numpy(Qt).cuda(), w0, make_cl, p


def test_gradient_and_update_halves_equal_the_fused_train_step(V):
    # data-parallel training splits each step into vlbm_closure_grad_step_ctx and
    # vlbm_closure_apply_grads around the all-reduce; with one process (nothing averaged)
    # the halves must reproduce the fused step exactly: losses, weights, coarse state
    import torch
    shape, Q0, Qtd, w0, make_cl, p = _dp_problem(V, 71)
    a, b = make_cl(), make_cl()
    a.set_weights(w0)
    b.set_weights(w0)
    grads = torch.empty(b.nparam, dtype=torch.float32, device="cuda")
    with V.Context(p) as ca, V.Context(p) as cb:
        assert ca.init_fields(Q0) == V.VLBM_OK and cb.init_fields(Q0) == V.VLBM_OK
        for _ in range(4):
            la = a.train_step_ctx(ca.ptr, Qtd.data_ptr())
            w_before = b.get_weights()
            lb = b.grad_step_ctx(cb.ptr, Qtd.data_ptr(), grads.data_ptr())
            assert np.array_equal(b.get_weights(), w_before)  # the gradient half changes no weight
            b.apply_grads(grads.data_ptr())
            # the loss is summed with FP64 atomics (order-dependent rounding); the gradient
            # is summed in a fixed order, so weights and states must agree bit for bit
            assert abs(la - lb) <= 1e-12 * abs(la)
        assert np.array_equal(a.get_weights(), b.get_weights())
        assert np.array_equal(ca.moments(), cb.moments())
    a.close()
    b.close()


def test_apply_grads_is_adam_on_the_given_gradient(V):
    # the update half against the reference's Adam (pinned by its closed form), over
    # three steps with gradients of widely different magnitudes (the bias corrections
    # of steps 2 and 3 matter); FP32 weights and moment estimates, so within FP32 rounding
    import torch
    _, _, _, _, make_cl, _ = _dp_problem(V, 72)
    cl = make_cl()
    rng = np.random.default_rng(72)
    w0 = (0.2 * rng.normal(size=cl.nparam)).astype(np.float32)
    cl.set_weights(w0)
    theta, m, v = w0.astype(np.float64), 0.0, 0.0
    for t in range(1, 4):
        g = (rng.normal(size=cl.nparam) * 10.0 ** rng.uniform(-4, 0, size=cl.nparam)).astype(np.float32)
        gd = torch.from_numpy(g).cuda()
        cl.apply_grads(gd.data_ptr())
        theta, m, v = C.adam_step(theta, m, v, g.astype(np.float64), t, 1e-3, 0.9, 0.999, 1e-8)
        got = cl.get_weights().astype(np.float64)
        assert np.abs(got - theta).max() < 2e-6, (t, np.abs(got - theta).max())
        # the step taken is the step of the reference (not merely small)
        assert np.abs((got - w0) - (theta - w0)).max() < 2e-3 * np.abs(theta - w0).max()
    cl.close()
