"""Parity at the benchmark configurations' full sizes, in the launch
configuration the benchmark times.

* Zalesak slotted disk, 256^2 mesh, 262,144 jittered particles: element by
  element against the oracle (triangulation bit-exact; delta, FLIP, right-hand
  side and mass assignment to relative L2 <= 1e-5).
* Learned-warm-start workload, 2048^2 mesh, 16,777,216 mixture particles,
  F = 4, and Taylor-Green 1024^2 with 4.2M particles, F = 2: too large for
  the oracle as a whole, so
  - stars of sampled particles against the oracle's stars on the full set;
  - volumes of sampled particles against their stars' areas (FP64);
  - the right-hand side at sampled nodes against the oracle's exact
    integral over the triangles of the particles around them, with the
    coverage of each node's support checked on the constant field;
  - properties at every node: Euler count 2N, sum of volumes L^2, the solve's
    residual recomputed in FP64 from the GPU's right-hand side, conservation.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W
from gpu_util import canon_tris, rel_l2, to_dev
from sampled import full_properties, sampled_checks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


# ---------------------------------------------------------------------------
def test_zalesak_full_size_elementwise(built):
    from paper_1610_05258_gb300 import Context
    inst = W.zalesak(256)
    assert inst.np == 262144
    c = Context(2, inst.n, inst.L, inst.np, inst.F)
    px, py, vals = to_dev(torch, inst.px, inst.py, inst.vals)
    tri, off = c.triangulate(px, py)
    t, o, v = oracle.triangulate(inst.L, inst.px, inst.py)
    assert canon_tris(tri.cpu().numpy(), off.cpu().numpy()) == canon_tris(t, o)
    T = (t, o, v)
    assert rel_l2(c.particle_volumes(px, py).cpu().numpy(), v) <= TOL
    assert rel_l2(c.assign_delta(px, py, vals).cpu().numpy(),
                  oracle.delta(2, inst.n, inst.L, inst.px, inst.py, inst.vals, tri=T)) <= TOL
    got = c.assign_flip(px, py, vals)
    want, _, _ = oracle.flip(2, inst.n, inst.L, inst.px, inst.py, inst.vals, v=v)
    assert rel_l2(got.cpu().numpy(), want) <= TOL
    b_or = oracle.rhs(2, inst.n, inst.L, inst.px, inst.py, inst.vals, tri=T)
    assert rel_l2(c.mass_rhs(px, py, vals).cpu().numpy(), b_or) <= TOL
    got, info = c.assign_mass(px, py, vals)
    assert rel_l2(got.cpu().numpy(), oracle.mass_solve(2, inst.n, inst.L, b_or)) <= TOL
    assert info[0].rel_resid <= 1e-6 and info[0].cons_err <= 1e-6


@pytest.mark.slow
def test_mixture_2048_sampled(built):
    """The learned-warm-start workload at full size (the benchmark's default)."""
    from paper_1610_05258_gb300 import Context, warmstart
    n, F = 2048, 4
    L = 2.0 * math.pi
    px, py, vals = warmstart.mixture_gpu(torch, n, 4, F, seed=16105, device="cuda")
    N = px.numel()
    c = Context(2, n, L, N, F)
    hx, hy, hv = px.cpu().numpy(), py.cpu().numpy(), vals.cpu().numpy()
    b = sampled_checks(c, hx, hy, hv, n, L, F, seed=1)
    full_properties(c, px, py, vals, b, n, L, F)


@pytest.mark.slow
def test_taylor_green_1024_sampled(built):
    from paper_1610_05258_gb300 import Context
    inst = W.taylor_green(1024, 4, seed=16103)
    c = Context(2, inst.n, inst.L, inst.np, inst.F)
    b = sampled_checks(c, inst.px, inst.py, inst.vals, inst.n, inst.L, inst.F, seed=2)
    px, py, vals = to_dev(torch, inst.px, inst.py, inst.vals)
    full_properties(c, px, py, vals, b, inst.n, inst.L, inst.F)
