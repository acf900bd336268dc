"""FP64 oracle of the particle advection driver steps (Sec. 3.1-3.3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the product library
never imports or calls it.

The particle state is a float32 position per coordinate (the library's
convention, see include/pmt.h). Each step restates the paper's motion:

* ``shift``   Sec. 3.1: dx/dt = u with u constant, so r <- r + u dt.
* ``rotate``  Sec. 3.2: rigid rotation about a centre by a fixed angle per
              step (the slotted disk turns once in a number of steps).
* ``rk2``     Sec. 3.3: particles move with the interpolated mesh velocity;
              explicit midpoint rule r <- r + dt u(r + dt/2 v), v the
              particle's velocity at r and u the mesh velocity interpolated
              at the midpoint (Eq. delta2); particle fields optionally scaled
              by a known decay factor (Taylor-Green exp(-2 nu dt)).

The update is computed in FP64 from the float32 positions, wrapped into the
periodic box [0, L) and rounded to float32; a value that rounds to L or above
becomes 0 (the same torus point). For ``shift`` and ``rotate`` the FP64
expression order is fixed below (numpy evaluates every operation with one
IEEE rounding and never fuses), so the float32 result is a plain function of
the inputs; cos and sin of the angle come from the host's libm (Python's
``math``).
"""
from __future__ import annotations

import math

import numpy as np

from . import interpolate as _interpolate


def wrap_round(r, L):
    """r (FP64 array) into [0, L), then rounded to float32 (L -> 0)."""
    r = np.asarray(r, dtype=np.float64)
    k = np.floor(r / L)
    r = r - L * k
    r = np.where(r < 0.0, r + L, r)
    r = np.where(r >= L, r - L, r)
    f = r.astype(np.float32)
    return np.where(f.astype(np.float64) >= L, np.float32(0.0), f).astype(np.float32)


def shift(L, px, py, dx, dy=0.0):
    """r <- r + (dx, dy) (Sec. 3.1), FP64, wrapped, rounded to float32."""
    x = wrap_round(np.asarray(px, np.float32).astype(np.float64) + float(dx), L)
    if py is None:
        return x, None
    y = wrap_round(np.asarray(py, np.float32).astype(np.float64) + float(dy), L)
    return x, y


def rotate(L, px, py, cx, cy, angle):
    """Rigid rotation about (cx, cy) by `angle` (Sec. 3.2):
    x' = cx + (c X - s Y), y' = cy + (s X + c Y), X = x - cx, Y = y - cy,
    c = cos(angle), s = sin(angle); FP64, wrapped, rounded to float32."""
    c, s = math.cos(angle), math.sin(angle)
    X = np.asarray(px, np.float32).astype(np.float64) - float(cx)
    Y = np.asarray(py, np.float32).astype(np.float64) - float(cy)
    x = float(cx) + (c * X - s * Y)
    y = float(cy) + (s * X + c * Y)
    return wrap_round(x, L), wrap_round(y, L)


def rk2(dim, n, L, mesh_vel, vel, px, py, dt, vals=None, factor=1.0, kind="q1"):
    """Explicit midpoint step with the mesh velocity (Sec. 3.3).

    mesh_vel [dim][n^dim] nodal velocity, vel [dim][np] the particles'
    velocity at their current positions. Midpoint r_m = r + dt/2 vel (wrapped,
    float32 like every particle position), mesh velocity interpolated there
    (Eq. delta2), r' = r + dt u(r_m). vals [F][np] (or None) are multiplied by
    `factor`. Returns (px', py', vals')."""
    px = np.asarray(px, np.float32)
    vel = np.asarray(vel, np.float64).reshape(dim, -1)
    mv = np.asarray(mesh_vel, np.float64).reshape(dim, -1)
    xm = wrap_round(px.astype(np.float64) + 0.5 * dt * vel[0], L)
    ym = None
    if dim == 2:
        py = np.asarray(py, np.float32)
        ym = wrap_round(py.astype(np.float64) + 0.5 * dt * vel[1], L)
    um = _interpolate(dim, n, L, mv, xm, ym, kind=kind)
    x = wrap_round(px.astype(np.float64) + dt * um[0], L)
    y = wrap_round(py.astype(np.float64) + dt * um[1], L) if dim == 2 else None
    out = None
    if vals is not None:
        out = np.asarray(vals, np.float64) * float(factor)
    return x, y, out
