"""FP64 reference of the learned flux closure (TEST INFRASTRUCTURE).

Only ``tests/`` may import this module.  It states, in plain NumPy, what the
closure kernels compute; it shares no code with them.

Network (3 x 3 x 3 periodic convolutions, channels first):
    x  = (Q - mu) / sigma                      8 input channels per cell
    a1 = tanh(conv(x,  W1, b1))                8 -> 32
    a2 = tanh(conv(a1, W2, b2))                32 -> 32
    y  = conv(a2, W3, b3)                      32 -> 24
    dPhi[k, a] = out_scale[k] * y[3 k + a]     flux correction per field k, axis a
with conv(x, W, b)[o, p] = b[o] + sum_{c, t} W[o, c, t] x[c, p + e_t], the 27
taps e_t = (dx, dy, dz) in {-1, 0, 1}^3 ordered t = 9 (dz+1) + 3 (dy+1) + (dx+1).

Correction of the lattice Boltzmann step (Eq. 2): after the collision,
    f*_{k, 2a+1} += dPhi[k, a] w_moving / cs^2,   f*_{k, 2a+2} -= dPhi[k, a] w_moving / cs^2
(w_moving / cs^2 = 1/2 on D3Q7); the rest population is unchanged, so the
zeroth moment of the correction vanishes and its first moment is dPhi: it adds
dPhi to the flux carried by the populations.  After streaming, Q_k changes by
-sum_a delta_a dPhi[k, a] (delta the centred difference): a conservative flux
divergence.

Training loss for one coarse step from state Q0 to target Qt:
    L = sum_{k, x} ((Q1_k(x) - Qt_k(x)) / sigma_k)^2 / N
with Q1 the moments after the corrected step.

Optimiser: Adam (Kingma and Ba, 2015, "Adam: a method for stochastic
optimization", their Algorithm 1): first and second moment estimates of the
gradient, each divided by one minus its decay rate to the power of the step
count, and the parameter moved by the learning rate times the corrected first
estimate over (the square root of the corrected second estimate + eps).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, e, sign=1):
    """out[..., z, y, x] = x[..., z + s dz, y + s dy, x + s dx] (periodic)."""
    dx, dy, dz = e
    return np.roll(x, shift=(-sign * dz, -sign * dy, -sign * dx), axis=(-3, -2, -1))


def conv3d(x, W, b=None):
    """x [C, Z, Y, X], W [O, C, 27], b [O] -> [O, Z, Y, X]."""
    O = W.shape[0]
    y = np.zeros((O,) + x.shape[1:])
    for t, e in enumerate(TAPS):
        y += np.einsum("oc,czyx->ozyx", W[:, :, t], _shift(x, e))
    if b is not None:
        y += b[:, None, None, None]
    return y


def conv3d_bwd_data(gy, W):
    """Adjoint of conv3d in x: gx[c, p] = sum_{o, t} W[o, c, t] gy[o, p - e_t]."""
    C = W.shape[1]
    gx = np.zeros((C,) + gy.shape[1:])
    for t, e in enumerate(TAPS):
        gx += np.einsum("oc,ozyx->czyx", W[:, :, t], _shift(gy, e, sign=-1))
    return gx


def conv3d_bwd_weight(gy, x):
    """Gradient in W: gW[o, c, t] = sum_p gy[o, p] x[c, p + e_t]; gb[o] = sum_p gy[o, p]."""
    gW = np.zeros((gy.shape[0], x.shape[0], 27))
    for t, e in enumerate(TAPS):
        gW[:, :, t] = np.einsum("ozyx,czyx->oc", gy, _shift(x, e))
    return gW, gy.reshape(gy.shape[0], -1).sum(1)


def _exact(a):
    return a


def net_forward(p, x, store=_exact):
    """The network on features x.  `store` is applied to each hidden activation
    as it is kept for the next layer (default: exact FP64).  A network whose
    activations are held in a narrower type between layers is stated by passing
    that type's rounding; every sum stays FP64."""
    z1 = conv3d(x, p["W1"], p["b1"])
    a1 = store(np.tanh(z1))
    z2 = conv3d(a1, p["W2"], p["b2"])
    a2 = store(np.tanh(z2))
    y = conv3d(a2, p["W3"], p["b3"])
    return y, {"x": x, "a1": a1, "a2": a2}


def net_backward(p, cache, gy, store=_exact):
    """Gradients of sum(gy * y) with respect to every weight and bias; `store`
    is applied to each hidden-layer gradient as it is kept for the next layer
    down (as in net_forward)."""
    g = {}
    g["W3"], g["b3"] = conv3d_bwd_weight(gy, cache["a2"])
    gz2 = store(conv3d_bwd_data(gy, p["W3"]) * (1.0 - cache["a2"] ** 2))
    g["W2"], g["b2"] = conv3d_bwd_weight(gz2, cache["a1"])
    gz1 = store(conv3d_bwd_data(gz2, p["W2"]) * (1.0 - cache["a1"] ** 2))
    g["W1"], g["b1"] = conv3d_bwd_weight(gz1, cache["x"])
    return g


def features(Q, mu, sigma):
    return (Q - np.asarray(mu)[:, None, None, None]) / np.asarray(sigma)[:, None, None, None]


def dphi_from_output(y, out_scale):
    """[24, Z, Y, X] network output -> dPhi[8, 3, Z, Y, X]."""
    return y.reshape((8, 3) + y.shape[1:]) * np.asarray(out_scale)[:, None, None, None, None]


def correction_populations(dphi):
    """Post-collision correction [8, 7, Z, Y, X] on D3Q7 from dPhi[8, 3, ...]."""
    corr = np.zeros((8, 7) + dphi.shape[2:])
    for a in range(3):
        corr[:, 2 * a + 1] = 0.5 * dphi[:, a]
        corr[:, 2 * a + 2] = -0.5 * dphi[:, a]
    return corr


def stream_d3q7(g):
    """Move direction i of g[8, 7, Z, Y, X] to x + c_i (periodic)."""
    c = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    out = np.empty_like(g)
    for i, e in enumerate(c):
        out[:, i] = _shift(g[:, i], e, sign=-1)
    return out


def corrected_step(f, gamma, tau, dphi, plain_step):
    """One Eq. 2 step with the closure: plain_step(f) + streamed correction
    (streaming is linear, so the correction can be streamed on its own)."""
    return plain_step(f, gamma, tau) + stream_d3q7(correction_populations(dphi))


def centred_divergence3(dphi_k):
    """sum_a delta_a dPhi[a] for one field, dphi_k [3, Z, Y, X]."""
    out = np.zeros(dphi_k.shape[1:])
    for a, axis in ((0, -1), (1, -2), (2, -3)):
        out += 0.5 * (np.roll(dphi_k[a], -1, axis=axis) - np.roll(dphi_k[a], 1, axis=axis))
    return out


def loss_and_grad_q(Q1, Qt, sigma):
    """L and dL/dQ1 for the normalised squared error."""
    s = np.asarray(sigma)[:, None, None, None]
    N = Q1[0].size
    r = (Q1 - Qt) / s
    return float((r * r).sum() / N), 2.0 * r / s / N


def grad_dphi_from_grad_q(gQ):
    """dL/dPhi[k, a] given dL/dQ1, through Q1 = Q_plain - sum_a delta_a dPhi[k, a]:
    the adjoint of -delta_a is +delta_a."""
    g = np.zeros((8, 3) + gQ.shape[1:])
    for a, axis in ((0, -1), (1, -2), (2, -3)):
        g[:, a] = 0.5 * (np.roll(gQ, -1, axis=axis) - np.roll(gQ, 1, axis=axis))
    return g


def init_params(rng, hidden=32, last_scale=0.0):
    """He-style initial weights; the last layer starts at `last_scale` times that."""
    def w(o, c, s=1.0):
        return rng.normal(0.0, s * np.sqrt(2.0 / (27 * c)), size=(o, c, 27))
    return {"W1": w(hidden, 8), "b1": np.zeros(hidden),
            "W2": w(hidden, hidden), "b2": np.zeros(hidden),
            "W3": w(24, hidden, last_scale), "b3": np.zeros(24)}


def adam_step(theta, m, v, g, t, lr, beta1, beta2, eps):
    """Step t (1, 2, ...) of Adam from parameters theta, moment estimates m and v
    (zero before the first step) and gradient g; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
