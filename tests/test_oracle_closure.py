"""Pins of the learned-closure reference (oracle/closure_ref.py).

The convolution is checked against scipy.ndimage.correlate (a library
routine for the single-channel case); both backward passes against the exact
adjoint identities of a linear map; the network gradient against central
finite differences; the flux correction against its closed-form effect on
one lattice Boltzmann step of the C oracle (zero change of every domain sum,
moment change equal to minus the centred divergence of dPhi).  Adam against
its closed form for a constant gradient and its invariance to the gradient's
scale.
"""
import numpy as np
from scipy import ndimage

from oracle import closure_ref as C


def test_conv_matches_scipy_correlate_single_channel():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 5, 6, 7))
    W = rng.normal(size=(1, 1, 27))
    kernel = np.zeros((3, 3, 3))
    for t, (dx, dy, dz) in enumerate(C.TAPS):
        kernel[dz + 1, dy + 1, dx + 1] = W[0, 0, t]
    ref = ndimage.correlate(x[0], kernel, mode="wrap")
    np.testing.assert_allclose(C.conv3d(x, W)[0], ref, rtol=1e-13, atol=1e-13)


def test_conv_of_delta_is_the_mirrored_kernel():
    W = np.arange(27, dtype=float).reshape(1, 1, 27) + 1.0
    x = np.zeros((1, 5, 5, 5))
    x[0, 2, 2, 2] = 1.0
    y = C.conv3d(x, W)[0]
    for t, (dx, dy, dz) in enumerate(C.TAPS):
        assert y[2 - dz, 2 - dy, 2 - dx] == W[0, 0, t]


def test_backward_passes_are_exact_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 4, 5, 6))
    W = rng.normal(size=(2, 3, 27))
    g = rng.normal(size=(2, 4, 5, 6))
    lhs = (C.conv3d(x, W) * g).sum()
    assert abs(lhs - (x * C.conv3d_bwd_data(g, W)).sum()) < 1e-12 * abs(lhs)
    gW, gb = C.conv3d_bwd_weight(g, x)
    assert abs(lhs - (W * gW).sum()) < 1e-12 * abs(lhs)
    np.testing.assert_allclose(gb, g.reshape(2, -1).sum(1))


def test_network_gradient_by_finite_differences():
    rng = np.random.default_rng(2)
    p = C.init_params(rng, hidden=4, last_scale=1.0)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(size=p[k].shape) * 0.1
    x = rng.normal(size=(8, 3, 4, 5))
    gy = rng.normal(size=(24, 3, 4, 5))
    y, cache = C.net_forward(p, x)
    grads = C.net_backward(p, cache, gy)
    h = 1e-6
    for name in ("W1", "b1", "W2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=4, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            fp = (C.net_forward(p, x)[0] * gy).sum()
            flat[idx] = old - h
            fm = (C.net_forward(p, x)[0] * gy).sum()
            flat[idx] = old
            fd = (fp - fm) / (2 * h)
            assert abs(fd - grads[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), name


def test_correction_is_conservative_and_acts_as_a_flux_divergence(orc):
    from paper_2606_00641_gb300 import fields
    shape = (6, 7, 8)
    f0 = fields.ideal_fields(shape, 31, mach=1.0, cfl=0.2)
    f = orc.ideal_init(f0.Q, f0.gamma)
    rng = np.random.default_rng(3)
    dphi = rng.normal(size=(8, 3) + shape) * 1e-4

    def plain(ff, gamma, tau):
        return orc.ideal_step(ff, gamma, tau)

    f_plain = plain(f, f0.gamma, 0.7)
    f_corr = C.corrected_step(f, f0.gamma, 0.7, dphi, plain)
    Qp, Qc = f_plain.sum(1), f_corr.sum(1)
    # every domain sum is unchanged by the correction
    np.testing.assert_allclose(Qc.reshape(8, -1).sum(1), Qp.reshape(8, -1).sum(1), atol=1e-13)
    # the moment change is minus the centred divergence of dPhi
    for k in range(8):
        np.testing.assert_allclose(Qc[k] - Qp[k], -C.centred_divergence3(dphi[k]), atol=1e-15)
    # zeroth and first moments of the correction populations: 0 and dPhi
    corr = C.correction_populations(dphi)
    assert np.abs(corr.sum(1)).max() == 0.0
    c = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)])
    first = np.einsum("kizyx,ia->kazyx", corr, c)
    np.testing.assert_allclose(first, dphi, atol=1e-18)


def test_loss_gradient_through_the_corrected_step(orc):
    from paper_2606_00641_gb300 import fields
    shape = (4, 5, 6)
    f0 = fields.ideal_fields(shape, 32, mach=1.0, cfl=0.2)
    f = orc.ideal_init(f0.Q, f0.gamma)
    rng = np.random.default_rng(4)
    dphi = rng.normal(size=(8, 3) + shape) * 1e-4
    Qt = f0.Q * (1 + 1e-3 * rng.normal(size=f0.Q.shape))
    sigma = np.abs(f0.Q).reshape(8, -1).max(1)

    def loss(dp):
        ff = C.corrected_step(f, f0.gamma, 0.7, dp, lambda a, g, t: orc.ideal_step(a, g, t))
        return C.loss_and_grad_q(ff.sum(1), Qt, sigma)

    L0, gQ = loss(dphi)
    g = C.grad_dphi_from_grad_q(gQ)
    h = 1e-7
    for _ in range(6):
        k, a = rng.integers(8), rng.integers(3)
        z, y, x = (rng.integers(n) for n in shape)
        d = np.zeros_like(dphi)
        d[k, a, z, y, x] = h
        fd = (loss(dphi + d)[0] - loss(dphi - d)[0]) / (2 * h)
        assert abs(fd - g[k, a, z, y, x]) < 1e-5 * max(abs(fd), 1e-8) + 1e-12


def test_storage_rounding_applies_where_the_hidden_values_are_kept():
    # store = identity is the exact network; a store that keeps nothing (zero)
    # leaves y = b3 and no gradient below the last layer, so the hook sits on a1,
    # a2 (forward) and on the hidden-layer gradients (backward); a rounding store
    # shows up in the cached activations exactly
    rng = np.random.default_rng(8)
    p = C.init_params(rng, hidden=4, last_scale=1.0)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(size=p[k].shape)
    x = rng.normal(size=(8, 3, 4, 5))
    gy = rng.normal(size=(24, 3, 4, 5))
    y0, c0 = C.net_forward(p, x)
    y1, c1 = C.net_forward(p, x, store=lambda a: a)
    assert np.array_equal(y0, y1)
    yz, cz = C.net_forward(p, x, store=np.zeros_like)
    assert np.allclose(yz, p["b3"][:, None, None, None] + 0 * yz)
    g = C.net_backward(p, cz, gy, store=np.zeros_like)
    for name in ("W1", "b1", "W2", "b2", "W3"):
        assert not np.any(g[name]), name
    assert np.allclose(g["b3"], gy.reshape(24, -1).sum(1))
    yr, cr = C.net_forward(p, x, store=lambda a: np.round(a, 2))
    assert np.array_equal(cr["a1"], np.round(np.tanh(C.conv3d(x, p["W1"], p["b1"])), 2))
    assert np.array_equal(cr["a2"], np.round(np.tanh(C.conv3d(cr["a1"], p["W2"], p["b2"])), 2))


def test_adam_under_a_constant_gradient_moves_by_lr_each_step():
    # with a constant gradient g from zero estimates, the bias corrections make the
    # corrected estimates exactly g and g^2 at every step t, so each step moves every
    # parameter by lr g / (|g| + eps), whatever the decay rates
    rng = np.random.default_rng(3)
    theta0 = rng.normal(size=50)
    g = rng.normal(size=50) * 10.0 ** rng.uniform(-3, 1, size=50)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    theta, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 8):
        theta, m, v = C.adam_step(theta, m, v, g, t, lr, b1, b2, eps)
        np.testing.assert_allclose(theta, theta0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)
    # other decay rates, the same path
    theta2, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 8):
        theta2, m, v = C.adam_step(theta2, m, v, g, t, lr, 0.5, 0.7, eps)
    np.testing.assert_allclose(theta2, theta, rtol=0, atol=1e-12)


def test_adam_step_is_invariant_to_the_gradient_scale_without_eps():
    # m_hat / sqrt(v_hat) is homogeneous of degree zero in g: scaling every gradient
    # of a sequence by c > 0 leaves the path unchanged (eps = 0)
    rng = np.random.default_rng(4)
    theta0 = rng.normal(size=40)
    gs = [rng.normal(size=40) for _ in range(5)]
    paths = []
    for c in (1.0, 37.0):
        theta, m, v = theta0.copy(), np.zeros(40), np.zeros(40)
        for t, g in enumerate(gs, start=1):
            theta, m, v = C.adam_step(theta, m, v, c * g, t, 1e-2, 0.9, 0.99, 0.0)
        paths.append(theta)
    np.testing.assert_allclose(paths[0], paths[1], rtol=0, atol=1e-13)
    # and the second step differs from the first: the estimates carry history
    t1, m, v = C.adam_step(theta0, 0.0, 0.0, gs[0], 1, 1e-2, 0.9, 0.99, 0.0)
    t2, _, _ = C.adam_step(t1, m, v, gs[1], 2, 1e-2, 0.9, 0.99, 0.0)
    assert np.abs((t2 - t1) - (-1e-2 * np.sign(gs[1]))).max() > 1e-4
