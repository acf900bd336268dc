"""Seeded synthetic inputs (positions and particle/mesh fields).

This module holds input generation only: random positions, lattices and
analytic fields. It contains none of the transfer method's arithmetic and is
shared by the tests, the benchmark and the smoke check, so that the CUDA path
and the oracle always see the very same arrays.

Workloads (sizes follow the experiments of arXiv 1610.05258, Sec. 3, scaled up):

* ``tophat_1d``      1D periodic convection of a top-hat (Sec. 3.1)
* ``zalesak``        2D slotted disk on a jittered lattice (Sec. 3.2)
* ``taylor_green``   2D Taylor-Green vortex, uniform random particles (Sec. 3.3)
* ``batched``        many uneven 2D instances with smooth random fields
* ``mixture``        2D Gaussian-mixture particle density, 10x contrast
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    dim: int
    n: int
    L: float
    px: np.ndarray            # float32 [Np]
    py: np.ndarray | None     # float32 [Np] (2D) or None
    vals: np.ndarray          # float32 [F, Np]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def np(self) -> int:
        return int(self.px.shape[0])

    @property
    def F(self) -> int:
        return int(self.vals.shape[0])


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def torus_keys(x, y, L):
    """The library's position convention (x -> floor(frac(fl32(x fl32(1/L))) 2^32),
    see include/pmt.h) as one 64-bit key per particle; used only to keep the
    generated particles distinct, which the particle functions require."""
    invL = np.float32(1.0 / L)
    def q(v):
        t = (np.asarray(v, np.float32) * invL).astype(np.float32)
        f = (t - np.floor(t)).astype(np.float32)
        f = np.where(f >= np.float32(1.0), np.float32(0.0), f)
        return (f.astype(np.float64) * 4294967296.0).astype(np.uint64)
    return (q(x) << np.uint64(32)) | q(y)


def redraw_coincident(x, y, L, g, draw):
    """Redraw particles whose torus coordinates coincide with an earlier one's."""
    for _ in range(16):
        k = torus_keys(x, y, L)
        _, first = np.unique(k, return_index=True)
        dup = np.ones(k.shape[0], bool)
        dup[first] = False
        nd = int(dup.sum())
        if nd == 0:
            return x, y
        nx, ny = draw(nd)
        x[dup], y[dup] = nx, ny
    return x, y


def tophat_1d(n=128, npart=128, seed=16101, lo=0.25, hi=0.5, L=1.0, regular=False, jitter=0.0):
    g = rng(seed)
    if regular:
        x = (np.arange(npart) + 0.5) * (L / npart)
        if jitter:
            x = x + g.uniform(-jitter, jitter, npart) * (L / npart)
    else:
        x = g.uniform(0.0, L, npart)
    x = np.mod(x, L).astype(np.float32)
    a = ((x >= lo) & (x < hi)).astype(np.float32)[None, :]
    return Instance(1, n, L, x, None, a, name=f"tophat_1d_n{n}_np{npart}")


def jittered_lattice(n, sub=2, jitter=0.4, seed=16102, L=1.0):
    """sub x sub particles per cell on a lattice of spacing h/sub, each
    coordinate jittered uniformly by +-jitter * (h/sub) / 2."""
    g = rng(seed)
    m = n * sub
    d = L / m
    ix, iy = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    x = (ix.ravel() + 0.5) * d + g.uniform(-0.5, 0.5, m * m) * jitter * d
    y = (iy.ravel() + 0.5) * d + g.uniform(-0.5, 0.5, m * m) * jitter * d
    return np.mod(x, L).astype(np.float32), np.mod(y, L).astype(np.float32)


def zalesak_indicator(x, y, cx=0.5, cy=0.75, R=0.15, slot_w=0.05, slot_top=0.85):
    inside = (x - cx) ** 2 + (y - cy) ** 2 < R * R
    slot = (np.abs(x - cx) < 0.5 * slot_w) & (y < slot_top)
    return (inside & ~slot).astype(np.float32)


def zalesak(n=256, seed=16102, jitter=0.4):
    x, y = jittered_lattice(n, 2, jitter, seed)
    a = zalesak_indicator(x.astype(np.float64), y.astype(np.float64))[None, :]
    return Instance(2, n, 1.0, x, y, a, name=f"zalesak_n{n}")


def taylor_green_fields(x, y, t=0.0, nu=0.01):
    f = math.exp(-2.0 * nu * t)
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    u = f * np.sin(x) * np.cos(y)
    v = -f * np.cos(x) * np.sin(y)
    return np.stack([u, v]).astype(np.float32)


def taylor_green(n=1024, ppc=4, seed=16103):
    L = 2.0 * math.pi
    g = rng(seed)
    npart = ppc * n * n
    x = g.uniform(0.0, L, npart).astype(np.float32)
    y = g.uniform(0.0, L, npart).astype(np.float32)
    x = np.where(x >= np.float32(L), np.float32(0), x)
    y = np.where(y >= np.float32(L), np.float32(0), y)
    x, y = redraw_coincident(x, y, L, g, lambda k: (g.uniform(0.0, L, k).astype(np.float32),
                                                    g.uniform(0.0, L, k).astype(np.float32)))
    return Instance(2, n, L, x, y, taylor_green_fields(x, y), name=f"taylor_green_n{n}")


def random_phase_field(n, slope=-3.0, seed=0, L=1.0):
    """Periodic Gaussian random field on an n x n grid with power spectrum
    P(k) ~ |k|^slope, zero mean and unit RMS (host FFT)."""
    g = rng(seed)
    kx = np.fft.fftfreq(n) * n
    k = np.sqrt(kx[None, :] ** 2 + kx[:, None] ** 2)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (slope / 2.0)
    c = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) * amp
    f = np.fft.ifft2(c).real
    f -= f.mean()
    f /= max(f.std(), 1e-30)
    return f


def sample_grid_field(f, L, x, y):
    """Bilinear sample of a periodic grid field (input generation only)."""
    n = f.shape[0]
    gx = x.astype(np.float64) / L * n
    gy = y.astype(np.float64) / L * n
    i0 = np.floor(gx).astype(np.int64)
    j0 = np.floor(gy).astype(np.int64)
    s = gx - i0
    t = gy - j0
    i0 %= n
    j0 %= n
    i1 = (i0 + 1) % n
    j1 = (j0 + 1) % n
    return (f[j0, i0] * (1 - s) * (1 - t) + f[j0, i1] * s * (1 - t) + f[j1, i0] * (1 - s) * t + f[j1, i1] * s * t)


def uniform_instance(n, ppc, F=3, seed=16104, L=1.0, slope=-3.0, field_grid=128):
    """Uniform random particles, F smooth Gaussian random fields (spectral
    slope `slope`) generated on a min(n, field_grid)^2 grid and sampled at
    the particles."""
    g = rng(seed)
    npart = max(16, int(round(ppc * n * n)))
    x = g.uniform(0.0, L, npart).astype(np.float32)
    y = g.uniform(0.0, L, npart).astype(np.float32)
    x, y = redraw_coincident(x, y, L, g, lambda k: (g.uniform(0.0, L, k).astype(np.float32),
                                                    g.uniform(0.0, L, k).astype(np.float32)))
    m = min(n, field_grid)
    vals = np.stack([sample_grid_field(random_phase_field(m, slope, seed * 7 + f, L), L, x, y) for f in range(F)])
    return Instance(2, n, L, x, y, vals.astype(np.float32), name=f"uniform_n{n}_ppc{ppc}")


def batched(count=256, nmin=64, nmax=512, ppc_min=1, ppc_max=8, F=3, seed=16104, take=None):
    """`count` instances with sides and particles per cell drawn uniformly;
    take=k builds only the first k of the same draw."""
    g = rng(seed)
    sides = g.integers(nmin, nmax + 1, count)
    ppcs = g.integers(ppc_min, ppc_max + 1, count)
    m = count if take is None else min(take, count)
    return [uniform_instance(int(sides[k]), int(ppcs[k]), F, seed * 1000 + k) for k in range(m)]


def mixture(n=2048, ppc=4, F=4, seed=16105, contrast=10.0, ncomp=8):
    """Particles drawn by rejection from rho ~ 1 + (contrast-1) g / max g, g a
    sum of periodic Gaussians of width 0.05 L; fields: Taylor-Green u, v plus
    random-phase Fourier fields."""
    L = 2.0 * math.pi
    g = rng(seed)
    cen = g.uniform(0.0, L, (ncomp, 2))
    sig = 0.05 * L
    m = 256
    gx = (np.arange(m) + 0.5) * (L / m)
    X, Y = np.meshgrid(gx, gx, indexing="xy")
    dens = np.zeros((m, m))
    for cx, cy in cen:
        dx = np.mod(X - cx + L / 2, L) - L / 2
        dy = np.mod(Y - cy + L / 2, L) - L / 2
        dens += np.exp(-(dx * dx + dy * dy) / (2 * sig * sig))
    rho = 1.0 + (contrast - 1.0) * dens / dens.max()
    rho /= rho.max()
    npart = ppc * n * n
    xs, ys = [], []
    have = 0
    while have < npart:
        k = int((npart - have) * 3.5) + 1024
        x = g.uniform(0.0, L, k)
        y = g.uniform(0.0, L, k)
        acc = g.uniform(0.0, 1.0, k) < sample_grid_field(rho, L, x, y)
        xs.append(x[acc])
        ys.append(y[acc])
        have += int(acc.sum())
    x = np.concatenate(xs)[:npart].astype(np.float32)
    y = np.concatenate(ys)[:npart].astype(np.float32)
    x = np.where(x >= np.float32(L), np.float32(0), x)
    y = np.where(y >= np.float32(L), np.float32(0), y)

    def draw(k):  # a fresh draw from the same density
        ox, oy = [], []
        while sum(len(a) for a in ox) < k:
            cx = g.uniform(0.0, L, 4 * k + 16)
            cy = g.uniform(0.0, L, 4 * k + 16)
            acc = g.uniform(0.0, 1.0, cx.shape[0]) < sample_grid_field(rho, L, cx, cy)
            ox.append(cx[acc])
            oy.append(cy[acc])
        return (np.concatenate(ox)[:k].astype(np.float32) % np.float32(L),
                np.concatenate(oy)[:k].astype(np.float32) % np.float32(L))
    x, y = redraw_coincident(x, y, L, g, draw)
    vals = [*taylor_green_fields(x, y)]
    for f in range(F - 2):
        grid = random_phase_field(256, -3.0, seed * 11 + f, L)
        vals.append(sample_grid_field(grid, L, x, y).astype(np.float32))
    return Instance(2, n, L, x, y, np.stack(vals[:F]).astype(np.float32), name=f"mixture_n{n}")


def mesh_field(dim, n, L, F=1, seed=7, kind="smooth"):
    """Nodal mesh values [F, n^dim] for G2P and solver tests."""
    g = rng(seed)
    if dim == 1:
        x = np.arange(n) * (L / n)
        out = [np.sin(2 * math.pi * x / L * (f + 1)) + 0.3 * g.standard_normal(n) * (kind == "noise") for f in range(F)]
        return np.stack(out)
    out = []
    for f in range(F):
        if kind == "noise":
            out.append(g.standard_normal((n, n)).ravel())
        else:
            out.append(random_phase_field(n, -3.0, seed + f, L).ravel())
    return np.stack(out)
