"""FP64 reference of the learned warm start's network (test infrastructure only).

A 4-layer fully convolutional network on the periodic mesh: 3x3 convolutions
2 -> 32 -> 32 -> 32 -> 1 with bias, ReLU after the first three, periodic
padding (the mesh is a torus). Input channels: the delta assignment of a field
(Sec. 2.2, Eq. delta) divided by the field's max |A|, and the residual of that
start, 64 (b - M delta) / (h^2 max|A|) (b = int A psi_j, Eq. proj). Output: 64
(mass - delta) / max|A|, the scaled correction that turns the delta field into
the mass assignment (Sec. 2.4); it starts the conjugate-gradient solve.

Written plainly with numpy (np.roll for the periodic shifts) in float64; the
backward pass is the adjoint of each forward step, pinned by central finite
differences in the tests.

Parameter layout (flat vector, the GPU library uses the same order):
    for each layer l: W_l [Co][Ci][3][3] then b_l [Co]
with tap (dy, dx) at index [dy + 1][dx + 1], reading x[y + dy][x + dx].
"""
from __future__ import annotations

import numpy as np

CHANNELS = [2, 32, 32, 32, 1]


def param_shapes():
    out = []
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        out.append((co, ci, 3, 3))
        out.append((co,))
    return out


def n_params():
    return int(sum(np.prod(s) for s in param_shapes()))


def unflatten(theta):
    ps, o = [], 0
    for s in param_shapes():
        k = int(np.prod(s))
        ps.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return ps


def init_params(seed=0):
    """He-normal weights, zero biases; the last layer is scaled down so that the
    untrained network starts close to the delta warm start."""
    g = np.random.default_rng(seed)
    theta = []
    for li, (ci, co) in enumerate(zip(CHANNELS[:-1], CHANNELS[1:])):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if li == len(CHANNELS) - 2 else 1.0)
        theta.append(g.standard_normal((co, ci, 3, 3)).ravel() * std)
        theta.append(np.zeros(co))
    return np.concatenate(theta)


def shift(x, dy, dx):
    """x[..., y + dy, x + dx] with periodic wrap."""
    return np.roll(x, shift=(-dy, -dx), axis=(-2, -1))


def conv(x, W, b):
    """y[co] = b[co] + sum_ci sum_taps W[co, ci, tap] x[ci][y + dy, x + dx]."""
    co = W.shape[0]
    y = np.zeros((co,) + x.shape[1:])
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = shift(x, dy, dx)
            y += np.einsum("oc,chw->ohw", W[:, :, dy + 1, dx + 1], xs)
    return y + b[:, None, None]


def conv_backward(x, W, gy):
    """Adjoints of conv: (dx, dW, db) for upstream gradient gy."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = shift(x, dy, dx)
            gW[:, :, dy + 1, dx + 1] = np.einsum("ohw,chw->oc", gy, xs)
            gx += shift(np.einsum("oc,ohw->chw", W[:, :, dy + 1, dx + 1], gy), -dy, -dx)
    return gx, gW, gy.sum(axis=(1, 2))


def forward(theta, x, keep=False):
    """x [2][H][W] -> correction [H][W] (and the activations if keep)."""
    ps = unflatten(theta)
    acts = [x]
    h = x
    nl = len(CHANNELS) - 1
    for l in range(nl):
        h = conv(h, ps[2 * l], ps[2 * l + 1])
        if l < nl - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return (h[0], acts) if keep else h[0]


def loss_and_grad(theta, x, target):
    """Mean squared error 0.5 mean((out - target)^2) and its gradient."""
    ps = unflatten(theta)
    out, acts = forward(theta, x, keep=True)
    r = out - target
    loss = 0.5 * float(np.mean(r * r))
    g = (r / r.size)[None]
    grads = [None] * len(ps)
    nl = len(CHANNELS) - 1
    for l in range(nl - 1, -1, -1):
        if l < nl - 1:
            g = g * (acts[l + 1] > 0)
        gx, gW, gb = conv_backward(acts[l], ps[2 * l], g)
        grads[2 * l], grads[2 * l + 1] = gW, gb
        g = gx
    return loss, np.concatenate([q.ravel() for q in grads])


RSCALE = 64.0


def features(delta, residual, h, scale):
    """Network input from the delta field and its residual b - M delta."""
    return np.stack([np.asarray(delta, np.float64) / scale,
                     RSCALE * np.asarray(residual, np.float64) / (h * h * scale)])
