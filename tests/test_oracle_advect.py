"""Pins of the oracle's advection steps (Sec. 3.1-3.3) against closed forms:
a shift by the box length and a rotation by 2 pi return the input, four
quarter turns compose to the identity, a quarter turn maps offsets (a, b) to
(-b, a), distances to the centre are kept, and the midpoint rule with the
mesh velocity is exact for a linear shear flow (its exact trajectory is
quadratic in time), which also reduces to a plain shift for a uniform flow."""
import math

import numpy as np

import oracle
from oracle import advect

ULP = 2.0 ** -23


def _torus_dist(a, b, L):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return np.minimum(d, L - d)


def test_shift_by_box_length_is_identity():
    g = np.random.default_rng(3)
    L = 1.0
    x = g.uniform(1e-3, L, 2000).astype(np.float32)
    y, _ = advect.shift(L, x, None, L)
    np.testing.assert_array_equal(y, x)
    y, _ = advect.shift(L, x, None, -3 * L)
    np.testing.assert_array_equal(y, x)


def test_shift_wraps_into_box_and_composes():
    g = np.random.default_rng(4)
    L = 2 * math.pi
    x = g.uniform(-3 * L, 4 * L, 3000).astype(np.float32)
    y = g.uniform(0, L, 3000).astype(np.float32)
    a, b = advect.shift(L, x, y, 0.3, -1.7)
    assert a.dtype == np.float32 and np.all((a >= 0) & (a < L)) and np.all((b >= 0) & (b < L))
    want = np.mod(x.astype(np.float64) + 0.3, L)
    assert np.max(_torus_dist(a, want, L)) <= L * ULP
    # n shifts of L/n return to the start within a few float ulps of L
    z = x
    for _ in range(16):
        z, _ = advect.shift(L, z, None, L / 16)
    assert np.max(_torus_dist(z, np.mod(x.astype(np.float64), L), L)) <= 16 * L * ULP


def test_rotation_closed_forms():
    g = np.random.default_rng(5)
    L, cx, cy = 1.0, 0.5, 0.5
    r = g.uniform(0.0, 0.45, 2000)
    th = g.uniform(0, 2 * math.pi, 2000)
    x = (cx + r * np.cos(th)).astype(np.float32)
    y = (cy + r * np.sin(th)).astype(np.float32)
    # a full turn
    a, b = advect.rotate(L, x, y, cx, cy, 2 * math.pi)
    assert np.max(np.abs(a - x)) <= ULP and np.max(np.abs(b - y)) <= ULP
    # a quarter turn: (cx + X, cy + Y) -> (cx - Y, cy + X)
    a, b = advect.rotate(L, x, y, cx, cy, math.pi / 2)
    X, Y = x.astype(np.float64) - cx, y.astype(np.float64) - cy
    assert np.max(np.abs(a - (cx - Y))) <= ULP and np.max(np.abs(b - (cy + X))) <= ULP
    # four quarter turns compose to the identity within a few ulps
    for _ in range(3):
        a, b = advect.rotate(L, a, b, cx, cy, math.pi / 2)
    assert np.max(np.abs(a - x)) <= 4 * ULP and np.max(np.abs(b - y)) <= 4 * ULP
    # 1000 steps of 2 pi / 1000 keep the distance to the centre
    a, b = x, y
    for _ in range(1000):
        a, b = advect.rotate(L, a, b, cx, cy, 2 * math.pi / 1000)
    r1 = np.hypot(a.astype(np.float64) - cx, b.astype(np.float64) - cy)
    r0 = np.hypot(x.astype(np.float64) - cx, y.astype(np.float64) - cy)
    assert np.max(np.abs(r1 - r0)) <= 1000 * ULP
    assert np.max(np.hypot(a - x, b - y)) <= 1000 * ULP  # back where they started


def test_rotation_wraps_periodically():
    L = 1.0
    x = np.array([0.95], np.float32)
    y = np.array([0.5], np.float32)
    a, b = advect.rotate(L, x, y, 0.5, 0.5, math.pi)  # to (0.05, 0.5)
    assert abs(a[0] - 0.05) <= ULP and abs(b[0] - 0.5) <= ULP
    a, b = advect.rotate(L, np.array([0.5], np.float32), np.array([0.5], np.float32), 0.0, 0.0, math.pi)
    assert abs(a[0] - 0.5) <= ULP and abs(b[0] - 0.5) <= ULP  # (-0.5, -0.5) wraps to (0.5, 0.5)


def _shear_case(n=32, L=1.0, a=0.7, b=-1.3, c=0.4, seed=6):
    g = np.random.default_rng(seed)
    h = L / n
    yn = (np.arange(n) * h)[:, None] * np.ones((1, n))
    u = (a + b * yn).ravel()
    v = np.full(n * n, c)
    npt = 3000
    # particles whose midpoints and end points stay clear of the periodic seam
    px = g.uniform(0, L, npt).astype(np.float32)
    py = g.uniform(3 * h, L - 4 * h, npt).astype(np.float32)
    return n, L, h, np.stack([u, v]), px, py


def test_midpoint_rule_exact_for_linear_shear():
    """u = a + b y, v = c (bilinear interpolation reproduces it away from the
    seam): the exact trajectory x(t) = x + a t + b (y t + c t^2 / 2),
    y(t) = y + c t, which the midpoint rule integrates exactly."""
    a, b, c = 0.7, -1.3, 0.4
    n, L, h, mv, px, py = _shear_case(a=a, b=b, c=c)
    dt = 0.5 * h
    vel = np.stack([a + b * py.astype(np.float64), np.full(px.shape[0], c)])
    x1, y1, _ = advect.rk2(2, n, L, mv, vel, px, py, dt)
    X = px.astype(np.float64) + a * dt + b * (py.astype(np.float64) * dt + c * dt * dt / 2)
    Y = py.astype(np.float64) + c * dt
    assert np.max(_torus_dist(x1, np.mod(X, L), L)) <= 4 * L * ULP
    assert np.max(_torus_dist(y1, np.mod(Y, L), L)) <= 4 * L * ULP


def test_midpoint_rule_uniform_flow_is_a_shift_and_scales_values():
    n, L = 24, 2 * math.pi
    g = np.random.default_rng(7)
    px = g.uniform(0, L, 500).astype(np.float32)
    py = g.uniform(0, L, 500).astype(np.float32)
    U, V, dt = 0.8, -0.35, 0.05
    mv = np.stack([np.full(n * n, U), np.full(n * n, V)])
    vel = np.stack([np.full(500, U), np.full(500, V)])
    vals = g.standard_normal((2, 500))
    x1, y1, v1 = advect.rk2(2, n, L, mv, vel, px, py, dt, vals=vals, factor=0.9)
    xs, ys = advect.shift(L, px, py, U * dt, V * dt)
    assert np.max(_torus_dist(x1, xs, L)) <= 2 * L * ULP and np.max(_torus_dist(y1, ys, L)) <= 2 * L * ULP
    np.testing.assert_allclose(v1, vals * 0.9, rtol=1e-15)
    # 1D: the same
    x1, _, _ = advect.rk2(1, n, L, np.full(n, U), np.full(500, U), px, None, dt)
    xs, _ = advect.shift(L, px, None, U * dt)
    assert np.max(_torus_dist(x1, xs, L)) <= 2 * L * ULP
