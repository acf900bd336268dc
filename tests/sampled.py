"""Parity checks at sizes too large for the oracle as a whole (test side,
shared by the full-size tests): sampled stars, volumes and right-hand-side
entries against the oracle's own integrals over the local triangles, and
properties that hold at every node (Euler count, sum of volumes, the solve's
FP64 residual, conservation)."""
import numpy as np
import pytest

import oracle
from gpu_util import to_dev

torch = pytest.importorskip("torch")


def mass_apply64(n, L, x):
    """M x in FP64 for the periodic bilinear mesh (h^2/36 [1 4 1]x[1 4 1])."""
    h = L / n
    X = x.reshape(-1, n, n)
    r = 4.0 * X + np.roll(X, 1, axis=2) + np.roll(X, -1, axis=2)
    r = 4.0 * r + np.roll(r, 1, axis=1) + np.roll(r, -1, axis=1)
    return (h * h / 36.0 * r).reshape(x.shape)


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


def _star_area(X, Y, L, w, nb, nof):
    qx = X[nb] + nof[:, 0] * L - X[w]
    qy = Y[nb] + nof[:, 1] * L - Y[w]
    return 0.5 * np.sum(qx * np.roll(qy, -1) - np.roll(qx, -1) * qy)


def sampled_checks(c, inst_px, inst_py, vals_h, n, L, F, seed, k_stars=600, k_nodes=12, delta_flip=True):
    """Sampled stars, volumes and right-hand side entries against the oracle;
    with delta_flip also the delta and FLIP assignments at the sampled nodes."""
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
        assert vol[w] == pytest.approx(_star_area(X, Y, L, w, nb, nof) / 3.0, rel=2e-5)
    # --- right-hand side at sampled nodes: the oracle's exact integral over
    # the triangles of the particles within 3.5 h of each node
    b_gpu = c.mass_rhs(px, py, vals).cpu().numpy().reshape(F, n * n)
    if delta_flip:
        d_gpu = c.assign_delta(px, py, vals).cpu().numpy().reshape(F, n * n)
        f_gpu = c.assign_flip(px, py, vals).cpu().numpy().reshape(F, n * n)
        amax = np.abs(vals_h).max(axis=1)
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
        if delta_flip:
            # delta: the node's value in the local triangle that contains it
            d_or = oracle.delta(2, n, L, inst_px, inst_py, vals_h, tri=(t, o, None), partial=True)[:, node]
            assert np.all(np.isfinite(d_or))
            assert np.all(np.abs(d_gpu[:, node] - d_or) <= 1e-5 * amax), (node, d_gpu[:, node], d_or)
            # FLIP: sums over the particles of the node's support (all within
            # 3.5 h), volumes = a third of their star areas (FP64)
            v_near = np.array([_star_area(X, Y, L, p, *star_of[p]) / 3.0 for p in near.tolist()])
            f_or, _, _ = oracle.flip(2, n, L, inst_px[near], inst_py[near], vals_h[:, near], v=v_near)
            assert np.all(np.abs(f_gpu[:, node] - f_or[:, node]) <= 1e-5 * amax), (node, f_gpu[:, node], f_or[:, node])
    return b_gpu


def full_properties(c, px, py, vals, b_gpu, n, L, F):
    out, info = c.assign_mass(px, py, vals)
    x = out.cpu().numpy().astype(np.float64).reshape(F, n * n)
    r = b_gpu.astype(np.float64) - mass_apply64(n, L, x)
    for f in range(F):
        assert np.linalg.norm(r[f]) <= 2e-6 * np.linalg.norm(b_gpu[f].astype(np.float64))
        assert info[f].rel_resid <= 1e-6
        assert info[f].cons_err <= 1e-6


