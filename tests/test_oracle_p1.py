"""Pins of the oracle's P1 mesh functions (2D cells split by the diagonal
from (0,0) to (1,1), linear hats on the triangles), against definitions that
do not share its per-cell formulas. The hat of node i is the hexagonal
pyramid psi_i(r) = max(0, 1 - max(|u|, |v|, |u - v|)), (u, v) = (r - r_i)/h
(periodic): 1 at the node, 0 at its six neighbours (+-1, 0), (0, +-1),
+-(1, 1), linear on each of the six triangles around it."""
import math

import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W

TWO32 = 2 ** 32


def pyramid(X, Y, ix, iy, n, L):
    h = L / n
    u = (np.mod(X - ix * h + L / 2, L) - L / 2) / h
    v = (np.mod(Y - iy * h + L / 2, L) - L / 2) / h
    return np.maximum(0.0, 1.0 - np.maximum(np.maximum(np.abs(u), np.abs(v)), np.abs(u - v)))


def exact_xy(px, py, L):
    X = oracle.fixed_coords(px, L).astype(np.float64) * (L / TWO32)
    Y = oracle.fixed_coords(py, L).astype(np.float64) * (L / TWO32)
    return X, Y


# --------------------------------------------------------------------------
# mass matrix
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [8, 12])
def test_p1_mass_fourier_eigenvalues(n):
    """The P1 mass stencil is (h^2/12) [6 at the node, 1 at its six
    neighbours], so a periodic mode cos(th i + ph j + c) is an eigenvector with
    lambda = (h^2/12)(6 + 2 cos th + 2 cos ph + 2 cos(th + ph)). A stencil
    along the other diagonal would give cos(th - ph) instead."""
    L = 1.7
    h = L / n
    i = np.arange(n)
    for k in range(n):
        th = 2 * math.pi * k / n
        l = (k * 3 + 1) % n
        ph = 2 * math.pi * l / n
        x = np.cos(th * i[None, :] + ph * i[:, None] + 0.3).ravel()
        lam = h * h / 12 * (6 + 2 * math.cos(th) + 2 * math.cos(ph) + 2 * math.cos(th + ph))
        y = oracle.mass_apply(2, n, L, x, kind="p1")[0]
        np.testing.assert_allclose(y, lam * x, rtol=0, atol=1e-14)


def test_p1_mass_brute_force_pyramids():
    """m_ij = int psi_i psi_j by a fine midpoint rule on the pyramids."""
    n, L, K = 4, 1.0, 96
    h = L / n
    q = (np.arange(n * K) + 0.5) * (L / (n * K))
    QX, QY = np.meshgrid(q, q, indexing="xy")
    psi = [pyramid(QX, QY, j % n, j // n, n, L) for j in range(n * n)]
    for j in (0, 5, 15):
        e = np.zeros(n * n)
        e[j] = 1.0
        got = oracle.mass_apply(2, n, L, e, kind="p1")[0]
        want = np.array([(psi[i] * psi[j]).sum() for i in range(n * n)]) * (L / (n * K)) ** 2
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-4 * h * h)
        # exactly seven non-zero entries
        assert np.count_nonzero(np.abs(got) > 1e-15) == 7


def test_p1_solve_inverts_and_matches_cg():
    n, L = 10, 2.0
    b = W.mesh_field(2, n, L, F=2, seed=3, kind="noise")
    x = oracle.mass_solve(2, n, L, b, kind="p1")
    np.testing.assert_allclose(oracle.mass_apply(2, n, L, x, kind="p1"), b, rtol=0, atol=1e-12 * np.abs(b).max())
    xc, it, res = oracle.mass_solve_cg(2, n, L, b, rtol=1e-13, kind="p1")
    np.testing.assert_allclose(x, xc, rtol=0, atol=1e-9 * np.abs(x).max())
    np.testing.assert_allclose(oracle.mass_apply(2, n, L, np.ones(n * n), kind="p1"), (L / n) ** 2, rtol=1e-14)


# --------------------------------------------------------------------------
# G2P and FLIP
# --------------------------------------------------------------------------
def test_p1_interpolate_brute_force():
    """sum over ALL nodes of Ab_i psi_i(r_mu), psi_i the pyramids."""
    n, L = 6, 1.3
    g = np.random.default_rng(4)
    px = g.uniform(-L, 2 * L, 60).astype(np.float32)
    py = g.uniform(-L, 2 * L, 60).astype(np.float32)
    mesh = g.standard_normal((2, n * n))
    got = oracle.interpolate(2, n, L, mesh, px, py, kind="p1")
    X, Y = exact_xy(px, py, L)
    want = sum(mesh[:, i : i + 1] * pyramid(X, Y, i % n, i // n, n, L)[None, :] for i in range(n * n))
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_p1_interpolate_affine_exact_bilinear_not():
    n, L = 16, 1.0
    g = np.random.default_rng(5)
    px = g.uniform(0.2, 0.7, 300).astype(np.float32)
    py = g.uniform(0.2, 0.7, 300).astype(np.float32)
    X, Y = exact_xy(px, py, L)
    i = np.arange(n) * (L / n)
    xx, yy = np.meshgrid(i, i, indexing="xy")
    aff = (0.3 + 1.1 * xx - 0.7 * yy).ravel()
    np.testing.assert_allclose(oracle.interpolate(2, n, L, aff, px, py, kind="p1")[0], 0.3 + 1.1 * X - 0.7 * Y,
                               atol=1e-12)
    bil = (xx * yy).ravel()
    err = np.abs(oracle.interpolate(2, n, L, bil, px, py, kind="p1")[0] - X * Y)
    assert err.max() > 1e-4 and err.max() <= (L / n) ** 2 / 4 + 1e-12


def test_p1_flip_brute_force_and_conservation():
    inst = W.uniform_instance(10, 3, F=2, seed=21)
    v = oracle.particle_volumes(2, inst.L, inst.px, inst.py)
    mesh, vol, empty = oracle.flip(2, inst.n, inst.L, inst.px, inst.py, inst.vals, v=v, kind="p1")
    X, Y = exact_xy(inst.px, inst.py, inst.L)
    for i in (0, 13, 77):
        w = v * pyramid(X, Y, i % inst.n, i // inst.n, inst.n, inst.L)
        assert vol[i] == pytest.approx(w.sum(), rel=1e-12, abs=1e-15)
        if w.sum() > 0:
            assert mesh[0, i] == pytest.approx((w * inst.vals[0]).sum() / w.sum(), rel=1e-11)
    # conservation with the FLIP node volumes, and their total
    assert vol.sum() == pytest.approx(v.sum(), rel=1e-12)
    np.testing.assert_allclose((vol[None, :] * mesh).sum(1), (v[None, :] * inst.vals).sum(1), rtol=1e-11)


# --------------------------------------------------------------------------
# right-hand side, mesh -> particle integral, mass assignment
# --------------------------------------------------------------------------
def test_p1_rhs_constant_affine_and_sum():
    """A = 1: b_j = int psi_j = h^2 (pyramid over a hexagon of area 3 h^2).
    Affine A: the hexagon is symmetric about the node, so b_j = h^2 A(x_j) at
    nodes away from the seam. sum_j b_j = sum_mu v_mu A_mu."""
    n, L = 16, 1.0
    h = L / n
    px, py = W.jittered_lattice(n, sub=2, jitter=0.4, seed=31)
    X, Y = exact_xy(px, py, L)
    tri = oracle.triangulate(L, px, py)
    a = np.stack([np.ones_like(X), 0.3 + 1.7 * X - 0.9 * Y])
    b = oracle.rhs(2, n, L, px, py, a, tri=tri, kind="p1")
    np.testing.assert_allclose(b[0], h * h, rtol=1e-12)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    inner = ((ii >= 3) & (ii <= n - 3) & (jj >= 3) & (jj <= n - 3)).ravel()
    want = h * h * (0.3 + 1.7 * ii * h - 0.9 * jj * h).ravel()
    np.testing.assert_allclose(b[1][inner], want[inner], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(b.sum(1), (tri[2][None, :] * a).sum(1), rtol=1e-12)


def test_p1_rhs_brute_force_fine_grid():
    """b_j = int A psi_j against a fine-grid product rule with A on a refined
    grid (delta: P1 on the particle triangulation) and psi_j the pyramid:
    second-order convergence to the oracle's exact value."""
    inst = W.uniform_instance(6, 4, F=1, seed=51)
    tri = oracle.triangulate(inst.L, inst.px, inst.py)
    b = oracle.rhs(2, inst.n, inst.L, inst.px, inst.py, inst.vals, tri=tri, kind="p1")[0]
    h = inst.L / inst.n
    errs = []
    for r in (8, 16, 32):
        m = inst.n * r
        A = oracle.delta(2, m, inst.L, inst.px, inst.py, inst.vals, tri=tri)[0].reshape(m, m)
        q = np.arange(m) * (inst.L / m)
        QX, QY = np.meshgrid(q, q, indexing="xy")
        est = np.array([(A * pyramid(QX, QY, j % inst.n, j // inst.n, inst.n, inst.L)).sum()
                        for j in range(inst.n * inst.n)]) * (inst.L / m) ** 2
        errs.append(np.abs(est - b).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5 and errs[2] < 1e-3 * h * h
    # not the bilinear right-hand side
    bq = oracle.rhs(2, inst.n, inst.L, inst.px, inst.py, inst.vals, tri=tri)[0]
    assert np.abs(b - bq).max() > 1e-6 * np.abs(b).max()


def test_p1_g2p_integral_is_the_transpose_of_the_rhs():
    inst = W.uniform_instance(10, 3, F=1, seed=31)
    n, L = inst.n, inst.L
    g = np.random.default_rng(5)
    A = g.standard_normal((3, inst.np))
    Ab = g.standard_normal((3, n * n))
    tri = oracle.triangulate(L, inst.px, inst.py)
    c = oracle.g2p_integral(2, n, L, Ab, inst.px, inst.py, tri=tri, kind="p1")
    b = oracle.rhs(2, n, L, inst.px, inst.py, A, tri=tri, kind="p1")
    for f in range(3):
        assert np.dot(c[f], A[f]) == pytest.approx(np.dot(Ab[f], b[f]), rel=1e-12, abs=1e-14)
    assert c.sum(axis=1) == pytest.approx((L / n) ** 2 * Ab.sum(axis=1), rel=1e-12, abs=1e-14)


def test_p1_mass_conservation_and_stability():
    inst = W.uniform_instance(12, 4, F=1, seed=61)
    tri, off, v = oracle.triangulate(inst.L, inst.px, inst.py)
    a = inst.vals[0].astype(np.float64)
    m = oracle.assign_mass(2, inst.n, inst.L, inst.px, inst.py, a, tri=(tri, off, v), kind="p1")[0]
    h = inst.L / inst.n
    assert (h * h * m).sum() == pytest.approx((v * a).sum(), rel=1e-11, abs=1e-14)
    e_mesh = m @ oracle.mass_apply(2, inst.n, inst.L, m, kind="p1")[0]
    e_part = oracle.particle_mass_apply(2, inst.L, inst.px, inst.py, a, tri=(tri, off, v))[0] @ a
    assert e_mesh <= e_part * (1 + 1e-12)


def test_p1_rejects_appendix_b_mode():
    inst = W.uniform_instance(8, 2, F=1, seed=3)
    with pytest.raises(Exception):
        oracle.rhs(2, inst.n, inst.L, inst.px, inst.py, inst.vals, mode=1, kind="p1")
