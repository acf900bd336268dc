"""GPU path (through the C ABI) against the FP64 oracle, element by element,
on the same seeded inputs. Tolerance: relative L2 <= 1e-5 for floating point
results; bit-exact for the sort, the cell table and the triangulation."""
import math

import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W
from gpu_util import canon_tris, rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def ctx_for(inst, F=None, extra=0):
    from paper_1610_05258_gb300 import Context
    return Context(inst.dim, inst.n, inst.L, inst.np + extra, F or inst.F)


def dev(inst):
    px, py, vals = to_dev(torch, inst.px, inst.py, inst.vals)
    return px, py, vals


CASES_2D = [
    ("uniform_n40_ppc4", lambda: W.uniform_instance(40, 4, F=2, seed=101)),
    ("uniform_n37_ppc1", lambda: W.uniform_instance(37, 1, F=1, seed=102)),
    ("uniform_n64_ppc7", lambda: W.uniform_instance(64, 7, F=3, seed=103)),
    ("zalesak_n48", lambda: W.zalesak(48, seed=104)),
    ("taylor_green_n33", lambda: W.taylor_green(33, 4, seed=105)),
    # small, sparse boxes: Voronoi cells reaching far rings (regression: a
    # star must never keep a virtual bounding point)
    ("uniform_n24_ppc1", lambda: W.uniform_instance(24, 1, F=2, seed=500)),
    ("uniform_n17_ppc5", lambda: W.uniform_instance(17, 5, F=2, seed=505)),
]
CASES_1D = [
    ("tophat_128", lambda: W.tophat_1d(128, 128, seed=16101)),
    ("tophat_ragged", lambda: W.tophat_1d(203, 517, seed=7)),
    ("tophat_sparse", lambda: W.tophat_1d(300, 40, seed=8)),
]


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,mk", CASES_2D + CASES_1D)
def test_sort_exact(built, name, mk):
    inst = mk()
    c = ctx_for(inst)
    px, py, _ = dev(inst)
    perm, cs = c.sort(px, py)
    perm, cs = perm.cpu().numpy(), cs.cpu().numpy()
    if inst.dim == 2:
        want_perm, want_cs = oracle.sort_by_cell(2, inst.n, inst.L, inst.px, inst.py)
    else:
        X = oracle.fixed_coords(inst.px, inst.L).astype(np.int64)
        cell = (X * inst.n) >> 32
        want_perm = np.lexsort((np.arange(inst.np), X, cell))
        want_cs = np.concatenate([[0], np.cumsum(np.bincount(cell, minlength=inst.n))])
    np.testing.assert_array_equal(perm, want_perm)
    np.testing.assert_array_equal(cs, want_cs)


@pytest.mark.parametrize("dim,n,npart,F", [(2, 50, 20011, 3), (2, 7, 333, 1), (1, 129, 5003, 2), (2, 256, 70000, 2)])
def test_interpolate(built, dim, n, npart, F):
    from paper_1610_05258_gb300 import Context
    g = np.random.default_rng(dim * 1000 + n)
    L = 2.0 * math.pi
    px = g.uniform(-L, 2 * L, npart).astype(np.float32)
    py = g.uniform(-L, 2 * L, npart).astype(np.float32)
    mesh = g.standard_normal((F, n ** dim))
    c = Context(dim, n, L, npart, F)
    dpx, dpy, dmesh = to_dev(torch, px, py if dim == 2 else None, mesh)
    got = c.interpolate(dmesh, dpx, dpy).cpu().numpy()
    want = oracle.interpolate(dim, n, L, mesh, px, py)
    assert rel_l2(got, want) <= TOL
    assert np.abs(got - want).max() <= 1e-5 * np.abs(mesh).max()


def test_interpolate_empty(built):
    from paper_1610_05258_gb300 import Context
    c = Context(2, 16, 1.0, 10, 1)
    z = torch.zeros(0, dtype=torch.float32, device="cuda")
    out = c.interpolate(torch.ones(256, device="cuda"), z, z)
    assert out.shape == (1, 0)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,mk", CASES_2D)
def test_triangulation_exact(built, name, mk):
    inst = mk()
    c = ctx_for(inst)
    px, py, _ = dev(inst)
    tri, off = c.triangulate(px, py)
    got = canon_tris(tri.cpu().numpy(), off.cpu().numpy())
    t, o, _ = oracle.triangulate(inst.L, inst.px, inst.py)
    assert len(got) == 2 * inst.np
    assert got == canon_tris(t, o)


def test_triangulation_degenerate_lattice(built):
    """Perfect lattice (every cell's corners cocircular): the symbolic
    perturbation must pick the same diagonals as the oracle."""
    from paper_1610_05258_gb300 import Context
    m = 64
    i = (np.arange(m) + 0.5) / m
    xx, yy = np.meshgrid(i, i, indexing="xy")
    px, py = xx.ravel().astype(np.float32), yy.ravel().astype(np.float32)
    c = Context(2, 32, 1.0, px.size, 1)
    dpx, dpy = to_dev(torch, px, py)
    tri, off = c.triangulate(dpx, dpy)
    t, o, _ = oracle.triangulate(1.0, px, py)
    assert canon_tris(tri.cpu().numpy(), off.cpu().numpy()) == canon_tris(t, o)


@pytest.mark.parametrize("name,mk", CASES_2D[:3] + CASES_1D)
def test_particle_volumes(built, name, mk):
    inst = mk()
    c = ctx_for(inst)
    px, py, _ = dev(inst)
    got = c.particle_volumes(px, py).cpu().numpy()
    want = oracle.particle_volumes(inst.dim, inst.L, inst.px, inst.py)
    assert rel_l2(got, want) <= TOL
    assert got.astype(np.float64).sum() == pytest.approx(inst.L ** inst.dim, rel=1e-5)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,mk", CASES_2D + CASES_1D)
def test_delta(built, name, mk):
    inst = mk()
    c = ctx_for(inst)
    px, py, vals = dev(inst)
    got = c.assign_delta(px, py, vals).cpu().numpy()
    want = oracle.delta(inst.dim, inst.n, inst.L, inst.px, inst.py, inst.vals)
    assert rel_l2(got, want) <= TOL


@pytest.mark.parametrize("name,mk", CASES_2D + CASES_1D)
def test_flip(built, name, mk):
    inst = mk()
    c = ctx_for(inst)
    px, py, vals = dev(inst)
    vol = torch.empty(inst.n ** inst.dim, device="cuda")
    got, empty = c.assign_flip(px, py, vals, node_volume=vol, count_empty=True)
    want, wvol, wempty = oracle.flip(inst.dim, inst.n, inst.L, inst.px, inst.py, inst.vals)
    assert rel_l2(got.cpu().numpy(), want) <= TOL
    assert rel_l2(vol.cpu().numpy(), wvol) <= TOL
    assert empty == wempty


@pytest.mark.parametrize("name,mk", CASES_2D + CASES_1D)
def test_mass_rhs(built, name, mk):
    inst = mk()
    c = ctx_for(inst)
    px, py, vals = dev(inst)
    got = c.mass_rhs(px, py, vals).cpu().numpy()
    want = oracle.rhs(inst.dim, inst.n, inst.L, inst.px, inst.py, inst.vals)
    for f in range(inst.F):
        assert rel_l2(got[f], want[f]) <= TOL


@pytest.mark.parametrize("dim,n,F", [(1, 64, 2), (1, 1001, 1), (2, 48, 3), (2, 301, 1)])
def test_mass_apply_and_solve(built, dim, n, F):
    from paper_1610_05258_gb300 import Context
    L = 1.3
    b = W.mesh_field(dim, n, L, F=F, seed=n, kind="noise")
    c = Context(dim, n, L, 16, F)
    (db,) = to_dev(torch, b)
    y = c.mass_apply(db).cpu().numpy()
    assert rel_l2(y, oracle.mass_apply(dim, n, L, b)) <= 1e-6
    x, info = c.mass_solve(db, rtol=1e-6)
    want = oracle.mass_solve(dim, n, L, b)
    for f in range(F):
        assert rel_l2(x.cpu().numpy()[f], want[f]) <= TOL
        assert info[f].rel_resid <= 1e-6
        kappa = 3.0 if dim == 1 else 9.0
        rate = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
        assert info[f].iters <= math.ceil(math.log(2 * math.sqrt(kappa) / 1e-6) / math.log(1 / rate)) + 3
    # the exact inverse as start: the solution to rounding, no iteration needed
    xd, dinfo = c.mass_solve(db, rtol=1e-6, warm_start="direct")
    for f in range(F):
        assert rel_l2(xd.cpu().numpy()[f], want[f]) <= TOL
        assert dinfo[f].init_rel_resid <= 1e-6 and dinfo[f].iters == 0


@pytest.mark.parametrize("name,mk", CASES_2D + CASES_1D)
@pytest.mark.parametrize("warm", ["delta", "zero", "direct"])
def test_assign_mass(built, name, mk, warm):
    inst = mk()
    c = ctx_for(inst)
    px, py, vals = dev(inst)
    got, info = c.assign_mass(px, py, vals, warm_start=warm, rtol=1e-6)
    want = oracle.assign_mass(inst.dim, inst.n, inst.L, inst.px, inst.py, inst.vals)
    got = got.cpu().numpy()
    for f in range(inst.F):
        assert rel_l2(got[f], want[f]) <= TOL, (f, rel_l2(got[f], want[f]))
        assert info[f].rel_resid <= 1e-6
        assert info[f].cons_err <= 1e-6
    v = oracle.particle_volumes(inst.dim, inst.L, inst.px, inst.py)
    for f in range(inst.F):
        assert info[f].sum_particles == pytest.approx(float((v * inst.vals[f]).sum()), rel=1e-5, abs=1e-9)


# ---------------------------------------------------------------------------
# errors are reported, never faults
# ---------------------------------------------------------------------------
def test_invalid_arguments(built):
    from paper_1610_05258_gb300 import Context, PMError
    with pytest.raises(PMError):
        Context(3, 16, 1.0, 10, 1)
    c = Context(2, 16, 1.0, 100, 1)
    px, py, vals = to_dev(torch, np.zeros(200), np.zeros(200), np.zeros(200))
    with pytest.raises(PMError) as e:
        c.assign_delta(px, py, vals)
    assert e.value.status == 1


def test_nonfinite_and_coincident_positions(built):
    from paper_1610_05258_gb300 import Context, PMError
    inst = W.uniform_instance(16, 4, F=1, seed=3)
    c = ctx_for(inst)
    x = inst.px.copy()
    x[5] = np.nan
    px, py, vals = to_dev(torch, x, inst.py, inst.vals)
    with pytest.raises(PMError) as e:
        c.assign_mass(px, py, vals)
    assert e.value.status == 5
    x = inst.px.copy()
    y = inst.py.copy()
    x[7], y[7] = x[3], y[3]
    px, py, vals = to_dev(torch, x, y, inst.vals)
    with pytest.raises(PMError) as e:
        c.assign_mass(px, py, vals)
    assert e.value.status == 5
    # the context stays usable afterwards
    px, py, vals = dev(inst)
    out, info = c.assign_mass(px, py, vals)
    assert info[0].rel_resid <= 1e-6


# ---------------------------------------------------------------------------
# high-degree particles: the working Voronoi cell outgrows the main pass's
# capacity and the particle goes through the retry pass
# ---------------------------------------------------------------------------
def flowers(petals, n=32, ppc=2, seed=77):
    """Uniform background with "flowers": a centre particle ringed by k
    particles at 0.3 cell widths (angles jittered), so that the centre's
    Delaunay degree is k."""
    g = np.random.default_rng(seed)
    h = 1.0 / n
    rho = 0.3 * h
    cen = [((i + 0.5) / len(petals) * 0.9 + 0.05, 0.5 + 0.3 * ((-1) ** i)) for i in range(len(petals))]
    pts = []
    for (cx, cy), k in zip(cen, petals):
        pts.append((cx, cy))
        ang = 2 * np.pi * (np.arange(k) + 0.2 * g.uniform(-1, 1, k)) / k
        pts += list(zip(cx + rho * np.cos(ang), cy + rho * np.sin(ang)))
    bg = g.uniform(0.0, 1.0, (ppc * n * n, 2))
    keep = np.ones(len(bg), bool)
    for cx, cy in cen:
        d = np.hypot((bg[:, 0] - cx + 0.5) % 1.0 - 0.5, (bg[:, 1] - cy + 0.5) % 1.0 - 0.5)
        keep &= d > 2.5 * rho
    pts = np.concatenate([np.array(pts), bg[keep]])
    return pts[:, 0].astype(np.float32), pts[:, 1].astype(np.float32)


def test_triangulation_high_degree_retry(built):
    from paper_1610_05258_gb300 import Context
    px, py = flowers([11, 12, 14, 16, 20, 23])
    c = Context(2, 32, 1.0, px.size, 1)
    dpx, dpy = to_dev(torch, px, py)
    tri, off = c.triangulate(dpx, dpy)
    got = canon_tris(tri.cpu().numpy(), off.cpu().numpy())
    t, o, _ = oracle.triangulate(1.0, px, py)
    assert got == canon_tris(t, o)
    # the centres have the planted degrees
    deg = np.bincount(np.asarray(t).ravel(), minlength=px.size)
    assert sorted(deg[[0, 12, 25, 40, 57, 78]].tolist()) == [11, 12, 14, 16, 20, 23]
    vals = np.ones((1, px.size), np.float32)
    (dv,) = to_dev(torch, vals)
    out, info = c.assign_mass(dpx, dpy, dv)
    assert np.abs(out.cpu().numpy() - 1.0).max() <= 1e-5
    # the counting build: every centre outgrows the main pass's 9 slots, the
    # four of degree > 12 also the first retry pass's 12; the counting build
    # gives the same stars
    c.profile(True, count_work=True)
    tri2, off2 = c.triangulate(dpx, dpy)
    w = c.work_read()
    c.profile(False)
    assert canon_tris(tri2.cpu().numpy(), off2.cpu().numpy()) == got
    assert w["retried"] >= 6 and 4 <= w["retried_last"] <= w["retried"]
    assert w["clips"] > 0 and w["cell_size_sum"] >= 3 * w["clips"]


def test_triangulation_degree_above_capacity(built):
    """A particle with more than 24 Delaunay neighbours is reported, never a fault."""
    from paper_1610_05258_gb300 import Context, PMError
    px, py = flowers([30])
    c = Context(2, 32, 1.0, px.size, 1)
    dpx, dpy = to_dev(torch, px, py)
    vals = torch.ones(1, px.size, device="cuda")
    with pytest.raises(PMError) as e:
        c.assign_mass(dpx, dpy, vals)
    assert e.value.status == 5
    # the context stays usable
    qx, qy = flowers([16])
    c2 = Context(2, 32, 1.0, qx.size, 1)
    a, b = to_dev(torch, qx, qy)
    out, info = c2.assign_mass(a, b, torch.ones(1, qx.size, device="cuda"))
    assert info[0].rel_resid <= 1e-6


def test_delta_degenerate_lattice(built):
    """Perfect lattice whose mesh nodes fall exactly on triangle edges and
    vertices: the orientation tests reach their exact ties, which the
    (eps, eps^2) node perturbation must resolve as in the oracle."""
    from paper_1610_05258_gb300 import Context
    m = 64
    i = (np.arange(m) + 0.5) / m
    xx, yy = np.meshgrid(i, i, indexing="xy")
    px, py = xx.ravel().astype(np.float32), yy.ravel().astype(np.float32)
    g = np.random.default_rng(11)
    vals = g.standard_normal((2, px.size)).astype(np.float32)
    for n in (32, 64, 128):
        c = Context(2, n, 1.0, px.size, 2)
        dpx, dpy, dv = to_dev(torch, px, py, vals)
        got = c.assign_delta(dpx, dpy, dv).cpu().numpy()
        want = oracle.delta(2, n, 1.0, px, py, vals)
        assert rel_l2(got, want) <= TOL, n


def test_tiny_amplitude_fields_scale_exactly(built):
    """A field of amplitude 1e-25 (max|A| near 2^-83, where the fixed-point
    exponent is capped) is assigned as 1e-25 times the unit field: the
    right-hand side and the solve read the fixed point at the same scale."""
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(40, 4, F=1, seed=111)
    c = Context(2, inst.n, inst.L, inst.np, 2)
    px, py = to_dev(torch, inst.px, inst.py)
    v = torch.from_numpy(np.concatenate([inst.vals, inst.vals * np.float32(1e-25)])).cuda()
    out, info = c.assign_mass(px, py, v)
    o = out.cpu().numpy().reshape(2, -1).astype(np.float64)
    assert rel_l2(o[1] * 1e25, o[0]) <= 1e-5
    assert info[1].rel_resid <= 1e-6 and info[1].cons_err <= 1e-6
    b = c.mass_rhs(px, py, v).cpu().numpy().reshape(2, -1).astype(np.float64)
    assert rel_l2(b[1] * 1e25, b[0]) <= 1e-5
