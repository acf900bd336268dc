"""Pins of the FP64 network reference: central finite differences of the loss
for every parameter block, the adjoint identity of the periodic convolution,
and translation equivariance on the torus."""
import numpy as np
import pytest

from oracle import net


def test_conv_adjoint_identity():
    g = np.random.default_rng(1)
    x = g.standard_normal((3, 7, 9))
    W = g.standard_normal((4, 3, 3, 3))
    gy = g.standard_normal((4, 7, 9))
    y = net.conv(x, W, np.zeros(4))
    gx, gW, _ = net.conv_backward(x, W, gy)
    # <conv(x), gy> = <x, conv^T(gy)> and = <W, dW>
    assert np.sum(y * gy) == pytest.approx(np.sum(x * gx), rel=1e-12)
    assert np.sum(y * gy) == pytest.approx(np.sum(W * gW), rel=1e-12)


def test_conv_brute_force():
    g = np.random.default_rng(2)
    x = g.standard_normal((2, 5, 6))
    W = g.standard_normal((3, 2, 3, 3))
    b = g.standard_normal(3)
    y = net.conv(x, W, b)
    H, Wd = 5, 6
    for co in range(3):
        for i in range(H):
            for j in range(Wd):
                s = b[co]
                for ci in range(2):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            s += W[co, ci, dy + 1, dx + 1] * x[ci, (i + dy) % H, (j + dx) % Wd]
                assert y[co, i, j] == pytest.approx(s, abs=1e-12)


def test_gradient_finite_differences():
    g = np.random.default_rng(3)
    theta = net.init_params(4)
    theta[-1] = 0.3  # make the output bias non-trivial
    x = g.standard_normal((2, 6, 6))
    tgt = g.standard_normal((6, 6))
    L, grad = net.loss_and_grad(theta, x, tgt)
    idx = list(range(0, net.n_params(), max(1, net.n_params() // 300))) + [net.n_params() - 1]
    eps = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (net.loss_and_grad(tp, x, tgt)[0] - net.loss_and_grad(tm, x, tgt)[0]) / (2 * eps)
        assert grad[k] == pytest.approx(fd, rel=1e-6, abs=1e-10), k


def test_translation_equivariance():
    g = np.random.default_rng(5)
    theta = net.init_params(6)
    x = g.standard_normal((2, 8, 8))
    y = net.forward(theta, x)
    ys = net.forward(theta, net.shift(x, 2, 3))
    np.testing.assert_allclose(ys, net.shift(y, 2, 3), atol=1e-12)
