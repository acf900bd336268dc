"""Positions outside [0, L) and reuse of one context across calls of
different sizes.

* Positions are taken modulo L (the periodic domain): shifting every
  particle by whole periods, up or down, must give the same bits. The
  positions sit on a 2^-16 grid with L = 1, so the shifted values are exact in
  float32 and the wrapped torus coordinates are the same numbers.
* A context sized for N particles serves calls of N (its maximum), then
  fewer, then N again; each result equals that of a fresh context."""
import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W
from gpu_util import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


def _grid_instance(n, npart, F, seed, dim=2):
    g = np.random.default_rng(seed)
    q = 2.0 ** -16
    span = 2 ** 32 if dim == 2 else 2 ** 16
    k = np.unique(g.integers(0, span, size=2 * npart))  # distinct grid points
    k = g.permutation(k)[:npart]
    assert k.size == npart
    if dim == 2:
        px = ((k % 2 ** 16) * q).astype(np.float32)
        py = ((k // 2 ** 16) * q).astype(np.float32)
    else:
        px = (k * q).astype(np.float32)
        py = None
    # smooth fields (the parity tolerance is set for those; white noise puts
    # the cancelling right-hand side at the FP32 floor)
    y = py if dim == 2 else np.zeros_like(px)
    w = 2.0 * np.pi
    vals = np.stack([np.sin(w * px) * np.cos(w * y) + 0.3, np.cos(w * (px + 2.0 * y)) - 0.2][:F])
    return px, py, vals.astype(np.float32)


@pytest.mark.parametrize("dim", [1, 2])
def test_positions_wrap_by_whole_periods(built, dim):
    from paper_1610_05258_gb300 import Context
    n, F = (37, 2) if dim == 2 else (101, 2)
    px, py, vals = _grid_instance(n, 3000 if dim == 2 else 700, F, seed=71 + dim, dim=dim)
    shift = np.where(np.arange(px.size) % 3 == 0, 3.0, np.where(np.arange(px.size) % 3 == 1, -2.0, 0.0))
    sx = (px + shift).astype(np.float32)
    sy = (py - shift).astype(np.float32) if dim == 2 else None
    assert np.array_equal(np.mod(sx, 1.0).astype(np.float32), px)
    c = Context(dim, n, 1.0, px.size, F)
    a = to_dev(torch, px, py, vals)
    b = to_dev(torch, sx, sy, vals)
    for name, call in (("mass", lambda d: c.assign_mass(*d, info=False)),
                       ("delta", lambda d: c.assign_delta(*d)),
                       ("flip", lambda d: c.assign_flip(*d)),
                       ("pic", lambda d: c.assign_pic(*d))):
        ra = call(a).clone()
        rb = call(b).clone()
        assert torch.equal(ra, rb), name
    mesh = W.mesh_field(dim, n, 1.0, F=F, seed=5, kind="noise").astype(np.float32)
    dm = to_dev(torch, mesh)[0]
    assert torch.equal(c.interpolate(dm, a[0], a[1]), c.interpolate(dm, b[0], b[1]))
    want = oracle.assign_mass(dim, n, 1.0, px, py, vals)
    assert rel_l2(c.assign_mass(*b, info=False).double().cpu().numpy(), want) <= 1e-5


def test_context_reuse_across_sizes(built):
    from paper_1610_05258_gb300 import Context
    n, F, N = 48, 3, 9000
    insts = [W.uniform_instance(n, 4, F=F, seed=80 + k) for k in range(3)]
    sizes = [N, 2500, N]
    big = Context(2, n, 1.0, N, F)
    for inst, m in zip(insts, sizes):
        px, py, vals = inst.px[:m], inst.py[:m], inst.vals[:, :m]
        d = to_dev(torch, px, py, vals)
        fresh = Context(2, n, 1.0, m, F)
        got, ginfo = big.assign_mass(*d)
        want, winfo = fresh.assign_mass(*d)
        assert torch.equal(got, want), m
        assert [x.iters for x in ginfo] == [x.iters for x in winfo]
        mesh = got.clone()
        assert torch.equal(big.interpolate_mass(mesh, d[0], d[1], info=False),
                           fresh.interpolate_mass(mesh, d[0], d[1], info=False)), m
        assert torch.equal(big.assign_delta(*d), fresh.assign_delta(*d)), m
    with pytest.raises(Exception):
        more = to_dev(torch, np.zeros(N + 1, np.float32), np.zeros(N + 1, np.float32), np.zeros((F, N + 1), np.float32))
        big.assign_mass(*more)
