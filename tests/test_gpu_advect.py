"""Parity of the advection kernels (the driver steps of Sec. 3.1-3.3) with the
oracle, element by element: the shift and the rigid rotation bit for bit
(both sides evaluate the same FP64 expression and round to float32), the
midpoint rule with the mesh velocity within a few float ulps of the box
(the GPU computes it in FP32)."""
import math

import numpy as np
import pytest

import oracle
from oracle import advect as OA
from paper_1610_05258_gb300 import workloads as W
from gpu_util import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ULP = 2.0 ** -23


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


def _torus_dist(a, b, L):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return np.minimum(d, L - d)


@pytest.mark.parametrize("dim,L", [(1, 1.0), (2, 1.0), (2, 2 * math.pi), (2, 3.0)])
def test_shift_bit_exact(built, dim, L):
    from paper_1610_05258_gb300 import Context
    g = np.random.default_rng(40 + dim)
    npt = 100003  # several blocks and a ragged tail
    x = g.uniform(-2 * L, 3 * L, npt).astype(np.float32)
    x[:6] = np.array([0.0, -0.0, L, np.nextafter(np.float32(L), np.float32(0)), -1e-30, 1e-30], np.float32)
    y = g.uniform(0, L, npt).astype(np.float32) if dim == 2 else None
    c = Context(dim, 16, L, npt, 1)
    for dx, dy in ((1.0 / 256, 0.0), (-0.3 * L, 0.77 * L), (L, -L), (1e-9, 5.5 * L)):
        px, py = to_dev(torch, x, y)
        c.advect_shift(px, py, dx, dy)
        wx, wy = OA.shift(L, x, y, dx, dy)
        np.testing.assert_array_equal(px.cpu().numpy(), wx)
        if dim == 2:
            np.testing.assert_array_equal(py.cpu().numpy(), wy)


def test_rotate_bit_exact_and_zalesak_revolution(built):
    from paper_1610_05258_gb300 import Context
    inst = W.zalesak(64)
    c = Context(2, inst.n, inst.L, inst.np, 1)
    px, py = to_dev(torch, inst.px, inst.py)
    ox, oy = inst.px.copy(), inst.py.copy()
    for angle in (2 * math.pi / 1000, 0.5, -2.0, math.pi):
        c.advect_rotate(px, py, 0.5, 0.5, angle)
        ox, oy = OA.rotate(inst.L, ox, oy, 0.5, 0.5, angle)
        np.testing.assert_array_equal(px.cpu().numpy(), ox)
        np.testing.assert_array_equal(py.cpu().numpy(), oy)
    # one revolution of 1000 steps (the configuration's rotation): still bit
    # for bit, and back within 1000 float ulps of the start
    px, py = to_dev(torch, inst.px, inst.py)
    ox, oy = inst.px.copy(), inst.py.copy()
    for _ in range(1000):
        c.advect_rotate(px, py, 0.5, 0.5, 2 * math.pi / 1000)
        ox, oy = OA.rotate(inst.L, ox, oy, 0.5, 0.5, 2 * math.pi / 1000)
    gx, gy = px.cpu().numpy(), py.cpu().numpy()
    np.testing.assert_array_equal(gx, ox)
    np.testing.assert_array_equal(gy, oy)
    inside = np.hypot(inst.px - 0.5, inst.py - 0.5) < 0.45
    assert np.max(np.hypot(gx - inst.px, gy - inst.py)[inside]) <= 1000 * ULP


@pytest.mark.parametrize("dim,kind", [(1, "q1"), (2, "q1"), (2, "p1")])
def test_rk2_matches_oracle(built, dim, kind):
    """Midpoint step r += dt u(r + dt/2 v) on the Taylor-Green velocity (2D) or
    a sine (1D): positions within 4 float ulps of L, decayed values to one
    float rounding."""
    from paper_1610_05258_gb300 import Context
    n, L = 64, 2 * math.pi
    h = L / n
    g = np.random.default_rng(50 + dim)
    if dim == 2:
        npt = 4 * n * n + 77
        x = g.uniform(0, L, npt).astype(np.float32)
        y = g.uniform(0, L, npt).astype(np.float32)
        xn = np.arange(n) * h
        XN, YN = np.meshgrid(xn, xn, indexing="xy")
        mv = np.stack([(np.sin(XN) * np.cos(YN)).ravel(), (-np.cos(XN) * np.sin(YN)).ravel()])
    else:
        npt = 4 * n + 5
        x = g.uniform(0, L, npt).astype(np.float32)
        y = None
        mv = np.sin(np.arange(n) * h)[None, :] + 0.5
    vals = g.standard_normal((2, npt)).astype(np.float32)
    dt, factor = 0.5 * h, math.exp(-2 * 0.01 * 0.5 * h)
    c = Context(dim, n, L, npt, 2, mesh=kind)
    px, py, dv, dm = to_dev(torch, x, y, vals, mv)
    vel = c.interpolate(dm, px, py)
    vel_h = vel.cpu().numpy()
    c.advect_rk2(dm, vel, px, py, dt, vals=dv, factor=factor)
    c.sync()
    wx, wy, wv = OA.rk2(dim, n, L, mv.astype(np.float32), vel_h, x, y, dt, vals=vals, factor=factor, kind=kind)
    assert np.max(_torus_dist(px.cpu().numpy(), wx, L)) <= 4 * L * ULP
    if dim == 2:
        assert np.max(_torus_dist(py.cpu().numpy(), wy, L)) <= 4 * L * ULP
    np.testing.assert_allclose(dv.cpu().numpy(), wv, rtol=2 * ULP, atol=0)
