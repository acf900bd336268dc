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

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


def mass_apply64(n, L, x):
    """M x in FP64 for the periodic bilinear mesh (h^2/36 [1 4 1]x[1 4 1])."""
    h = L / n
    X = x.reshape(-1, n, n)
    r = 4.0 * X + np.roll(X, 1, axis=2) + np.roll(X, -1, axis=2)
    r = 4.0 * r + np.roll(r, 1, axis=1) + np.roll(r, -1, axis=1)
    return (h * h / 36.0 * r).reshape(x.shape)


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


# ---------------------------------------------------------------------------
def stars_from_triangles(tri, off, which):
    """Neighbour sets {(q, ox, oy)} of the particles in `which` from a
    triangle list (p, a, b) with image offsets of a and b relative to p."""
    want = {int(w): set() for w in which}
    sel = np.isin(tri, np.asarray(which)).any(axis=1)
    for (p, a, b), (oax, oay, obx, oby) in zip(tri[sel], off[sel]):
        verts = [(int(p), 0, 0), (int(a), int(oax), int(oay)), (int(b), int(obx), int(oby))]
        for k, (s, sx, sy) in enumerate(verts):
            if s in want:
                for j, (q, qx, qy) in enumerate(verts):
                    if j != k:
                        want[s].add((q, qx - sx, qy - sy))
    return want


def sampled_checks(c, inst_px, inst_py, vals_h, n, L, F, seed, k_stars=600, k_nodes=12):
    """Sampled stars, volumes and right-hand side entries against the oracle."""
    N = inst_px.size
    g = np.random.default_rng(seed)
    px, py, vals = to_dev(torch, inst_px, inst_py, vals_h)
    # --- stars of sampled particles
    tri, off = c.triangulate(px, py)
    tri, off = tri.cpu().numpy(), off.cpu().numpy()
    assert tri.shape[0] == 2 * N  # Euler on the torus
    which = g.choice(N, k_stars, replace=False)
    got = stars_from_triangles(tri, off, which)
    st = oracle.stars(L, inst_px, inst_py, which)
    for w, (nb, nof) in zip(which, st):
        assert got[int(w)] == {(int(q), int(a), int(b)) for q, (a, b) in zip(nb, nof)}, int(w)
    # --- volumes: a third of the areas of the incident triangles (FP64)
    vol = c.particle_volumes(px, py).cpu().numpy()
    assert vol.astype(np.float64).sum() == pytest.approx(L * L, rel=1e-5)
    X = oracle.fixed_coords(inst_px, L).astype(np.float64) * (L / 2 ** 32)
    Y = oracle.fixed_coords(inst_py, L).astype(np.float64) * (L / 2 ** 32)
    for w, (nb, nof) in zip(which[:100], st[:100]):
        qx = X[nb] + nof[:, 0] * L - X[w]
        qy = Y[nb] + nof[:, 1] * L - Y[w]
        area = 0.5 * np.sum(qx * np.roll(qy, -1) - np.roll(qx, -1) * qy)
        assert vol[w] == pytest.approx(area / 3.0, rel=2e-5)
    # --- right-hand side at sampled nodes: the oracle's exact integral over
    # the triangles of the particles within 3.5 h of each node
    b_gpu = c.mass_rhs(px, py, vals).cpu().numpy().reshape(F, n * n)
    h = L / n
    nodes = g.choice(n * n, k_nodes, replace=False)
    near_of = []
    for node in nodes:
        ix, iy = node % n, node // n
        dx = (X - ix * h + L / 2) % L - L / 2
        dy = (Y - iy * h + L / 2) % L - L / 2
        near_of.append(np.nonzero((np.abs(dx) < 3.5 * h) & (np.abs(dy) < 3.5 * h))[0])
    allnear = np.unique(np.concatenate(near_of))
    star_of = dict(zip(allnear.tolist(), oracle.stars(L, inst_px, inst_py, allnear)))
    ones = np.ones((1, N))
    scale = np.abs(b_gpu).max(axis=1)
    for node, near in zip(nodes, near_of):
        tris = set()
        for p in near.tolist():
            nb, nof = star_of[p]
            m = len(nb)
            for k in range(m):
                a, b = int(nb[k]), int(nb[(k + 1) % m])
                oa, ob = nof[k], nof[(k + 1) % m]
                # canonical: lowest index first, offsets relative to it
                verts = [(p, 0, 0), (a, int(oa[0]), int(oa[1])), (b, int(ob[0]), int(ob[1]))]
                r = min(range(3), key=lambda i: verts[i][0])
                v0 = verts[r]
                rot = [verts[(r + i) % 3] for i in range(3)]
                tris.add(tuple((q, qx - v0[1], qy - v0[2]) for q, qx, qy in rot))
        t = np.array([[v[0] for v in tr] for tr in tris], dtype=np.int64)
        o = np.array([[tr[1][1], tr[1][2], tr[2][1], tr[2][2]] for tr in tris], dtype=np.int32)
        cover = oracle.rhs(2, n, L, inst_px, inst_py, ones, tri=(t, o, None))[0, node]
        assert cover == pytest.approx(h * h, rel=1e-9)  # the support is fully covered
        b_or = oracle.rhs(2, n, L, inst_px, inst_py, vals_h, tri=(t, o, None))[:, node]
        assert np.all(np.abs(b_gpu[:, node] - b_or) <= 1e-5 * scale), (node, b_gpu[:, node], b_or)
    return b_gpu


def full_properties(c, px, py, vals, b_gpu, n, L, F):
    out, info = c.assign_mass(px, py, vals)
    x = out.cpu().numpy().astype(np.float64).reshape(F, n * n)
    r = b_gpu.astype(np.float64) - mass_apply64(n, L, x)
    for f in range(F):
        assert np.linalg.norm(r[f]) <= 2e-6 * np.linalg.norm(b_gpu[f].astype(np.float64))
        assert info[f].rel_resid <= 1e-6
        assert info[f].cons_err <= 1e-6


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
