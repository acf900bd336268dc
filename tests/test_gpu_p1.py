"""P1 mesh functions (2D cells split by the (0,0)-(1,1) diagonal) on the GPU
through the C ABI (pm_ctx_create_mesh with PM_MESH_P1) against the FP64
oracle's P1 mode, element by element: G2P, FLIP, mass apply, right-hand side,
mass assignment and solve, mesh -> particle integrals (lumped and full mass).
Tolerance: relative L2 <= 1e-5; solves to the 1e-6 residual; conservation to
1e-6."""
import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W
from gpu_util import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


def refined_lattice(n, L=1.0, F=2):
    """A particle at every node, edge midpoint and cell centre: triangle edges
    lie on cell lines and on cell diagonals (exact ties of the clipping)."""
    m = 2 * n
    iy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    px = (ix.ravel() * (L / m)).astype(np.float32)
    py = (iy.ravel() * (L / m)).astype(np.float32)
    vals = np.random.default_rng(n).standard_normal((F, px.size)).astype(np.float32)
    return W.Instance(2, n, L, px, py, vals, name="refined_lattice")


CASES = [
    ("uniform_n40_ppc4", lambda: W.uniform_instance(40, 4, F=2, seed=101)),
    ("uniform_n37_ppc1", lambda: W.uniform_instance(37, 1, F=1, seed=102)),
    ("uniform_n64_ppc7_F3", lambda: W.uniform_instance(64, 7, F=3, seed=103)),
    ("zalesak_n48", lambda: W.zalesak(48, seed=104)),
    ("mixture_n32_F4", lambda: W.mixture(32, 4, 4)),
    ("uniform_n24_ppc3_F8", lambda: W.uniform_instance(24, 3, F=8, seed=108)),
]


def unpack(inst):
    return inst.n, inst.L, inst.px, inst.py, inst.vals


def ctx(n, L, N, F):
    from paper_1610_05258_gb300 import Context
    return Context(2, n, L, N, F, mesh="p1")


@pytest.mark.parametrize("name,mk", CASES + [("refined_lattice_n24", lambda: refined_lattice(24))])
def test_p1_rhs_and_mass_assignment(built, name, mk):
    n, L, px, py, vals = unpack(mk())
    F, N = vals.shape[0], px.size
    c = ctx(n, L, N, F)
    dpx, dpy, dv = to_dev(torch, px, py, vals)
    tri = oracle.triangulate(L, px, py)
    b_or = oracle.rhs(2, n, L, px, py, vals, tri=tri, kind="p1")
    b = c.mass_rhs(dpx, dpy, dv).cpu().numpy().reshape(F, -1)
    assert rel_l2(b, b_or) <= TOL
    out, info = c.assign_mass(dpx, dpy, dv)
    want = oracle.mass_solve(2, n, L, b_or, kind="p1")
    assert rel_l2(out.cpu().numpy().reshape(F, -1), want) <= TOL
    for f in range(F):
        assert info[f].rel_resid <= 1e-6 and info[f].cons_err <= 1e-6


@pytest.mark.parametrize("name,mk", CASES[:3])
def test_p1_g2p_flip_and_apply(built, name, mk):
    n, L, px, py, vals = unpack(mk())
    F, N = vals.shape[0], px.size
    c = ctx(n, L, N, F)
    dpx, dpy, dv = to_dev(torch, px, py, vals)
    mesh = W.mesh_field(2, n, L, F=F, seed=9, kind="noise").astype(np.float32)
    (dm,) = to_dev(torch, mesh)
    got = c.interpolate(dm, dpx, dpy).cpu().numpy().reshape(F, -1)
    assert rel_l2(got, oracle.interpolate(2, n, L, mesh, px, py, kind="p1")) <= TOL
    v = oracle.particle_volumes(2, L, px, py)
    fl, _, _ = oracle.flip(2, n, L, px, py, vals, v=v, kind="p1")
    assert rel_l2(c.assign_flip(dpx, dpy, dv).cpu().numpy().reshape(F, -1), fl) <= TOL
    ap = c.mass_apply(dm).cpu().numpy().reshape(F, -1)
    assert rel_l2(ap, oracle.mass_apply(2, n, L, mesh, kind="p1")) <= TOL
    x, info = c.mass_solve(dm)
    assert rel_l2(x.cpu().numpy().reshape(F, -1), oracle.mass_solve(2, n, L, mesh, kind="p1")) <= TOL


@pytest.mark.parametrize("name,mk", [CASES[0], CASES[4]])
def test_p1_mesh_to_particle(built, name, mk):
    n, L, px, py, vals = unpack(mk())
    F, N = vals.shape[0], px.size
    c = ctx(n, L, N, F)
    dpx, dpy = to_dev(torch, px, py)
    mesh = W.mesh_field(2, n, L, F=F, seed=11, kind="smooth").astype(np.float32)
    (dm,) = to_dev(torch, mesh)
    tri = oracle.triangulate(L, px, py)
    lum = c.interpolate_lumped(dm, dpx, dpy).cpu().numpy().reshape(F, -1)
    assert rel_l2(lum, oracle.interpolate_lumped(2, n, L, mesh, px, py, tri=tri, kind="p1")) <= TOL
    full, info = c.interpolate_mass(dm, dpx, dpy)
    want = oracle.interpolate_mass(2, n, L, mesh, px, py, tri=tri, kind="p1")
    assert rel_l2(full.cpu().numpy().reshape(F, -1), want) <= 2e-5
    for f in range(F):
        assert info[f].rel_resid <= 1e-6


def test_p1_differs_from_q1_and_rejects_q1_only_options(built):
    from paper_1610_05258_gb300 import Context, PMError
    inst = W.uniform_instance(32, 3, F=1, seed=7)
    dpx, dpy, dv = to_dev(torch, inst.px, inst.py, inst.vals)
    q1 = Context(2, inst.n, inst.L, inst.np, 1).mass_rhs(dpx, dpy, dv).cpu().numpy()
    c = ctx(inst.n, inst.L, inst.np, 1)
    p1 = c.mass_rhs(dpx, dpy, dv).cpu().numpy()
    assert rel_l2(p1, q1) > 1e-4
    for kw in ({"rhs": "appb"}, {"warm_start": "direct"}):
        with pytest.raises(PMError) as e:
            c.assign_mass(dpx, dpy, dv, **kw)
        assert e.value.status == 1
    with pytest.raises(PMError):
        c.mass_rhs(dpx, dpy, dv, rhs="appb")
    # the context stays usable
    out, info = c.assign_mass(dpx, dpy, dv)
    assert info[0].rel_resid <= 1e-6


def test_p1_is_the_linear_mesh_in_1d(built):
    """In 1D both mesh kinds are the linear hats: identical results."""
    from paper_1610_05258_gb300 import Context
    inst = W.tophat_1d(203, 517, seed=7)
    px, vals = to_dev(torch, inst.px, inst.vals)
    outs = []
    for kind in ("q1", "p1"):
        c = Context(1, inst.n, inst.L, inst.np, 1, mesh=kind)
        m, _ = c.assign_mass(px, None, vals)
        outs.append(m.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
