"""Pins of the oracle's PIC assignment (Eq. PIC with mesh volumes) and of its
stability integrals (Eq. stab, integral form) against brute force and closed
forms: PIC equals the direct sum over hat functions on tiny inputs and is
conservative with the mesh volumes; int Ab^2 of a Fourier mode is its
eigenvalue times its squared norm; int A^2 of a constant field is c^2 L^dim;
the 1D particle integral equals a fine quadrature of the explicit
piecewise-linear interpolant; the mass assignment never increases it."""
import math

import numpy as np
import pytest

import oracle

TWO32 = 2 ** 32


def _hat(d, h):
    return np.maximum(0.0, 1.0 - np.abs(d) / h)


def _wrapd(d, L):
    return np.mod(d + L / 2, L) - L / 2


@pytest.mark.parametrize("dim", [1, 2])
def test_pic_brute_force_and_conservation(dim):
    g = np.random.default_rng(80 + dim)
    n, L = 6, 1.7
    h = L / n
    npt = 40 if dim == 1 else 400
    px = g.uniform(0, L, npt).astype(np.float32)
    py = g.uniform(0, L, npt).astype(np.float32) if dim == 2 else None
    a = g.standard_normal((2, npt))
    v = oracle.particle_volumes(dim, L, px, py)
    got = oracle.pic(dim, n, L, px, py, a, v=v)
    X = oracle.fixed_coords(px, L).astype(np.float64) * (L / TWO32)
    Y = oracle.fixed_coords(py, L).astype(np.float64) * (L / TWO32) if dim == 2 else None
    want = np.zeros((2, n ** dim))
    for node in range(n ** dim):
        ix, iy = node % n, node // n
        w = _hat(_wrapd(X - ix * h, L), h)
        if dim == 2:
            w = w * _hat(_wrapd(Y - iy * h, L), h)
        want[:, node] = (a * v * w).sum(axis=1) / h ** dim
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    # conservation with the mesh volumes (Eq. cons): sum h^dim Ab = sum v A
    np.testing.assert_allclose(got.sum(axis=1) * h ** dim, (a * v).sum(axis=1), rtol=1e-12)


def test_pic_lattice_at_nodes_is_exact():
    """One particle on every node, v_mu = h^dim: PIC returns the values."""
    n, L = 8, 2.0
    h = L / n
    ix, iy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    px = (ix.ravel() * h).astype(np.float32)
    py = (iy.ravel() * h).astype(np.float32)
    a = np.random.default_rng(3).standard_normal((1, n * n))
    got = oracle.pic(2, n, L, px, py, a, v=np.full(n * n, h * h))
    np.testing.assert_allclose(got, a, rtol=1e-12)


@pytest.mark.parametrize("dim,kind", [(1, "q1"), (2, "q1"), (2, "p1")])
def test_energy_mesh_fourier_mode(dim, kind):
    n, L = 16, 3.0
    h = L / n
    k1, k2 = 3, 5
    i = np.arange(n)
    if dim == 1:
        x = np.cos(2 * np.pi * k1 * i / n)
        lam = h * (2 + math.cos(2 * np.pi * k1 / n)) / 3
    else:
        I, J = np.meshgrid(i, i, indexing="xy")
        th, ph = 2 * np.pi * k1 / n, 2 * np.pi * k2 / n
        x = np.cos(th * I + ph * J).ravel()
        if kind == "q1":
            lam = h * h * (2 + math.cos(th)) * (2 + math.cos(ph)) / 9
        else:  # 6 at the node, 1 at (+-1, 0), (0, +-1), (1, 1), (-1, -1), times h^2 / 12
            lam = h * h * (6 + 2 * math.cos(th) + 2 * math.cos(ph) + 2 * math.cos(th + ph)) / 12
    got = oracle.energy_mesh(dim, n, L, x, kind)[0]
    assert got == pytest.approx(lam * (x * x).sum(), rel=1e-12)


def test_energy_particles_constant_and_1d_quadrature():
    g = np.random.default_rng(9)
    L = 1.3
    px = g.uniform(0, L, 300).astype(np.float32)
    py = g.uniform(0, L, 300).astype(np.float32)
    assert oracle.energy_particles(2, L, px, py, np.full((1, 300), 2.5))[0] == pytest.approx(2.5 ** 2 * L * L,
                                                                                          rel=1e-12)
    # 1D: int A^2 of the explicit periodic piecewise-linear interpolant
    x1 = px[:40]
    a = g.standard_normal(40)
    X = oracle.fixed_coords(x1, L).astype(np.float64) * (L / TWO32)
    o = np.argsort(X, kind="stable")
    xs = np.concatenate([X[o] - L, X[o], X[o] + L])
    av = np.concatenate([a[o]] * 3)
    m = 400000
    q = (np.arange(m) + 0.5) * (L / m)
    want = (np.interp(q, xs, av) ** 2).sum() * (L / m)
    assert oracle.energy_particles(1, L, x1, None, a)[0] == pytest.approx(want, rel=1e-6)


@pytest.mark.parametrize("dim", [1, 2])
def test_mass_assignment_does_not_increase_energy(dim):
    g = np.random.default_rng(20 + dim)
    n, L = 12, 1.0
    npt = 50 if dim == 1 else 500
    px = g.uniform(0, L, npt).astype(np.float32)
    py = g.uniform(0, L, npt).astype(np.float32) if dim == 2 else None
    a = g.standard_normal((2, npt))
    tri = oracle.triangulate(L, px, py) if dim == 2 else None
    mesh = oracle.assign_mass(dim, n, L, px, py, a, tri=tri)
    em = oracle.energy_mesh(dim, n, L, mesh)
    ep = oracle.energy_particles(dim, L, px, py, a, tri=tri)
    assert np.all(em <= ep * (1 + 1e-12))
    # and the projection is a contraction strictly for rough particle data
    assert np.all(em < 0.99 * ep)
