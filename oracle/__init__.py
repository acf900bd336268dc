"""FP64 CPU oracle for particle<->mesh transfer (arXiv 1610.05258).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product library never imports,
links or calls it, and it shares no code with the CUDA path.

Every function restates a definition of the paper in plain double precision
(see ``pmt_oracle.c`` for the per-routine citations):

* ``interpolate``      G2P, Sec. 2.2 Eq. delta2
* ``delta``            delta assignment, Sec. 2.2 Eq. delta
* ``flip``             FLIP assignment, Sec. 2.3 Eqs. PIC and FLIP_vol
* ``pic``              PIC assignment, Sec. 2.3 Eq. PIC with mesh volumes
* ``energy_mesh``, ``energy_particles``  int Ab^2 = Ab^T M Ab and
                       int A^2 = A^T M_p A (stability, Eq. stab)
* ``rhs``              mass right-hand side, Sec. 2.4 Eqs. proj and phi_def
                       (mode 0 exact overlay integral, mode 1 App. B quadrature)
* ``mass_apply``       m_ij = int psi_i psi_j, Sec. 2.4
* ``mass_solve``       direct tensor-product periodic tridiagonal solve
* ``triangulate``      periodic Delaunay triangulation of the particles by the
                       empty-circumcircle definition (Sec. 3.2, App. A)
* ``g2p_integral``     c_mu = int Ab psi_mu (mesh interpolant against the
                       particle functions), Table 1 right column
* ``particle_mass_apply``  m_{mu nu} = int psi_mu psi_nu on the particles
* ``interpolate_lumped``   Abb_mu = c_mu / v_mu, Eq. lumped
* ``interpolate_mass``     full mass: m_p Abb = c, Eq. proj2 (phi_mu of
                       Eq. phi_def on the particles), solved by FP64 CG
* ``advect``           the driver steps of Sec. 3.1-3.3 (shift, rigid
                       rotation, midpoint rule with the mesh velocity)

The App. B quadrature in 2D (mode 1) follows a reading of a garbled passage
(the paper's text describes six-point quadratic fits on triangles; this
build's mesh is bilinear). Its implementation is pinned by closed forms
(exact for fields affine over a node's support; with particles at all 3 x 3
sample points, exact for quadratic fields, which fixes the point weights);
the reading itself has no value printed in the paper to compare with.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmt_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

MAXSTAR = 64


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain gcc, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_tri_monomial.restype = ctypes.c_double
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise OracleError(f"oracle {what} failed with status {st}")


def _fields(vals, np_):
    v = _f64(vals)
    if v.ndim == 1:
        v = v.reshape(1, -1)
    assert v.shape[1] == np_
    return v


def fixed_coords(x, L):
    x = _f32(x)
    out = np.empty(x.shape[0], dtype=np.uint32)
    _check(lib().or_fixed_coords(_p(x), ctypes.c_longlong(x.shape[0]), ctypes.c_double(L), _p(out)), "fixed_coords")
    return out


def sort_by_cell(dim, n, L, px, py=None):
    px = _f32(px)
    py = _f32(py) if py is not None else px
    npt = px.shape[0]
    perm = np.empty(npt, dtype=np.int64)
    cs = np.empty(n ** dim + 1, dtype=np.int64)
    _check(lib().or_sort_by_cell(dim, n, ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(npt), _p(perm), _p(cs)),
           "sort_by_cell")
    return perm, cs


def _p1(dim, kind):
    """Mesh functions: "q1" (linear in 1D, bilinear in 2D) or "p1" (2D: cells
    split by the diagonal from (0,0) to (1,1), linear hats on the triangles;
    in 1D the same as q1)."""
    if kind not in ("q1", "p1"):
        raise ValueError(f"unknown mesh functions {kind!r}")
    return 1 if (kind == "p1" and dim == 2) else 0


def interpolate(dim, n, L, mesh, px, py=None, kind="q1"):
    px = _f32(px)
    py = _f32(py) if py is not None else px
    m = _f64(mesh).reshape(-1, n ** dim)
    F = m.shape[0]
    out = np.empty((F, px.shape[0]))
    _check(lib().or_interpolate(dim, n, ctypes.c_double(L), _p(m), F, _p(px), _p(py),
                                ctypes.c_longlong(px.shape[0]), _p(out), _p1(dim, kind)), "interpolate")
    return out


def mass_apply(dim, n, L, x, kind="q1"):
    x = _f64(x).reshape(-1, n ** dim)
    y = np.empty_like(x)
    lib().or_mass_apply(dim, n, ctypes.c_double(L), _p(x), x.shape[0], _p(y), _p1(dim, kind))
    return y


def mass_solve(dim, n, L, b, kind="q1"):
    """M x = b. Q1: direct tensor-product periodic tridiagonal solve. P1 (2D):
    M is circulant on the periodic grid, so it is diagonalised by the 2D FFT;
    its eigenvalues are the FFT of M applied to a unit impulse."""
    b = _f64(b).reshape(-1, n ** dim)
    if _p1(dim, kind):
        e0 = np.zeros(n * n)
        e0[0] = 1.0
        lam = np.fft.fft2(mass_apply(2, n, L, e0, "p1").reshape(n, n))
        x = np.fft.ifft2(np.fft.fft2(b.reshape(-1, n, n)) / lam).real
        return x.reshape(b.shape)
    x = np.empty_like(b)
    _check(lib().or_mass_solve_direct(dim, n, ctypes.c_double(L), _p(b), b.shape[0], _p(x)), "mass_solve")
    return x


def mass_solve_cg(dim, n, L, b, x0=None, rtol=1e-12, max_iter=10000, kind="q1"):
    b = _f64(b).reshape(-1, n ** dim)
    x = np.empty_like(b)
    F = b.shape[0]
    it = np.zeros(F, dtype=np.int32)
    res = np.zeros(F)
    x0p = _p(_f64(x0).reshape(b.shape)) if x0 is not None else None
    _check(lib().or_mass_solve_cg(dim, n, ctypes.c_double(L), _p(b), F, _p(x), x0p, ctypes.c_double(rtol), max_iter,
                                  _p(it), _p(res), _p1(dim, kind)), "mass_solve_cg")
    return x, it, res


def particle_volumes(dim, L, px, py=None):
    """v_mu = int psi_mu (Eq. part_v)."""
    px = _f32(px)
    if dim == 1:
        v = np.empty(px.shape[0])
        _check(lib().or1_particle_volumes(ctypes.c_double(L), _p(px), ctypes.c_longlong(px.shape[0]), _p(v)), "volumes")
        return v
    return triangulate(L, px, py)[2]


def triangulate(L, px, py):
    """Periodic Delaunay triangulation; every triangle once as (p, a, b), p the
    smallest index, counter-clockwise; off = image offsets of a and b relative
    to p (in box lengths); v = particle volumes."""
    px, py = _f32(px), _f32(py)
    npt = px.shape[0]
    cap = 2 * npt + 16
    tri = np.empty((cap, 3), dtype=np.int64)
    off = np.empty((cap, 4), dtype=np.int32)
    v = np.empty(npt)
    nt = ctypes.c_longlong(0)
    _check(lib().or2_triangulate(ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(npt), _p(tri), _p(off),
                                 ctypes.c_longlong(cap), ctypes.byref(nt), _p(v)), "triangulate")
    return tri[: nt.value].copy(), off[: nt.value].copy(), v


def stars(L, px, py, which):
    """Delaunay star (counter-clockwise neighbour cycle) of each particle in which."""
    px, py = _f32(px), _f32(py)
    w = np.ascontiguousarray(which, dtype=np.int64)
    deg = np.empty(w.shape[0], dtype=np.int32)
    nbr = np.empty((w.shape[0], MAXSTAR), dtype=np.int64)
    nof = np.empty((w.shape[0], MAXSTAR, 2), dtype=np.int32)
    _check(lib().or2_stars(ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(px.shape[0]), _p(w),
                           ctypes.c_longlong(w.shape[0]), _p(deg), _p(nbr), _p(nof)), "stars")
    return [(nbr[k, : deg[k]].copy(), nof[k, : deg[k]].copy()) for k in range(w.shape[0])]


def delta(dim, n, L, px, py, vals, tri=None, partial=False):
    """delta assignment (Eq. delta). partial=True (2D, a subset of the
    triangles given in `tri`): nodes that no given triangle covers are NaN
    instead of an error."""
    px = _f32(px)
    v = _fields(vals, px.shape[0])
    F = v.shape[0]
    out = np.empty((F, n ** dim))
    if dim == 1:
        _check(lib().or1_delta(n, ctypes.c_double(L), _p(px), ctypes.c_longlong(px.shape[0]), _p(v), F, _p(out)), "delta")
        return out
    py = _f32(py)
    t, o, _ = tri if tri is not None else triangulate(L, px, py)
    t = np.ascontiguousarray(t, dtype=np.int64)
    o = np.ascontiguousarray(o, dtype=np.int32)
    if partial:
        out.fill(np.nan)
    st = lib().or2_delta(n, ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(px.shape[0]), _p(v), F, _p(t),
                         _p(o), ctypes.c_longlong(t.shape[0]), _p(out))
    if not (partial and st == 5):  # 5: some node not covered
        _check(st, "delta")
    return out


def flip(dim, n, L, px, py, vals, v=None, kind="q1"):
    """FLIP assignment; returns (mesh values, FLIP node volumes, #empty nodes)."""
    px = _f32(px)
    py = _f32(py) if py is not None else px
    a = _fields(vals, px.shape[0])
    F = a.shape[0]
    if v is None:
        v = particle_volumes(dim, L, px, py)
    v = _f64(v)
    out = np.empty((F, n ** dim))
    vol = np.empty(n ** dim)
    e = ctypes.c_longlong(0)
    _check(lib().or_flip(dim, n, ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(px.shape[0]), _p(a), F, _p(v),
                         _p(out), _p(vol), ctypes.byref(e), _p1(dim, kind)), "flip")
    return out, vol, e.value


def pic(dim, n, L, px, py, vals, v=None, kind="q1"):
    """PIC assignment (Sec. 2.3, Eq. PIC with the mesh volumes of Eq. mesh_v,
    v_i = int psi_i = h^dim): Ab_i = sum_mu A_mu v_mu psi_i(r_mu) / h^dim.
    The sum is FLIP's numerator: the FLIP value times the FLIP node volume."""
    out, vol, _ = flip(dim, n, L, px, py, vals, v=v, kind=kind)
    return out * vol[None, :] / (L / n) ** dim


def energy_mesh(dim, n, L, x, kind="q1"):
    """int Ab^2 = Ab^T M Ab per field (Eq. stab in integral form)."""
    x = _f64(x).reshape(-1, n ** dim)
    return (x * mass_apply(dim, n, L, x, kind)).sum(axis=1)


def energy_particles(dim, L, px, py, vals, tri=None):
    """int A^2 = A^T M_p A per field, M_p the particle mass matrix."""
    a = _fields(vals, _f32(px).shape[0])
    return (a * particle_mass_apply(dim, L, px, py, a, tri)).sum(axis=1)


def rhs(dim, n, L, px, py, vals, mode=0, tri=None, kind="q1"):
    """b_j = int A psi_j (mode 0 exact, mode 1 App. B quadrature; the P1 mesh
    has mode 0 only)."""
    px = _f32(px)
    a = _fields(vals, px.shape[0])
    F = a.shape[0]
    b = np.empty((F, n ** dim))
    if dim == 1:
        _check(lib().or1_rhs(n, ctypes.c_double(L), _p(px), ctypes.c_longlong(px.shape[0]), _p(a), F, mode, _p(b)), "rhs")
        return b
    py = _f32(py)
    t, o, _ = tri if tri is not None else triangulate(L, px, py)
    _check(lib().or2_rhs(n, ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(px.shape[0]), _p(a), F, _p(t), _p(o),
                         ctypes.c_longlong(t.shape[0]), mode, _p(b), _p1(dim, kind)), "rhs")
    return b


def assign_mass(dim, n, L, px, py, vals, mode=0, tri=None, kind="q1"):
    """Mass assignment (Sec. 2.4): Ab = M^-1 b."""
    return mass_solve(dim, n, L, rhs(dim, n, L, px, py, vals, mode, tri, kind), kind)


def tri_monomial(x, y, a, b):
    x, y = _f64(x), _f64(y)
    return lib().or_tri_monomial(_p(x), _p(y), a, b)


def _tri_or_none(dim, L, px, py, tri):
    if dim == 1:
        return np.zeros((0, 3), np.int64), np.zeros((0, 4), np.int32), 0
    t, o, _ = tri if tri is not None else triangulate(L, px, py)
    t = np.ascontiguousarray(t, dtype=np.int64)
    o = np.ascontiguousarray(o, dtype=np.int32)
    return t, o, t.shape[0]


def g2p_integral(dim, n, L, mesh, px, py=None, tri=None, kind="q1"):
    """c_mu = int Ab(r) psi_mu(r) dr with Ab the mesh interpolant of `mesh`
    ([F][n^dim]); exact (Simpson on merged breakpoints in 1D, clipped
    polygons with a degree-3 rule in 2D)."""
    px = _f32(px)
    npt = px.shape[0]
    m = _f64(mesh)
    if m.ndim == 1:
        m = m.reshape(1, -1)
    F = m.shape[0]
    c = np.empty((F, npt))
    if dim == 1:
        _check(lib().or1_g2p_int(n, ctypes.c_double(L), _p(px), ctypes.c_longlong(npt), _p(m), F, _p(c)), "g2p_int")
        return c
    py = _f32(py)
    t, o, nt = _tri_or_none(2, L, px, py, tri)
    _check(lib().or2_g2p_int(n, ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(npt), _p(m), F, _p(t), _p(o),
                             ctypes.c_longlong(nt), _p(c), _p1(2, kind)), "g2p_int")
    return c


def particle_mass_apply(dim, L, px, py, x, tri=None):
    """y = M_p x, M_p the particle mass matrix (1D hats, 2D P1 triangles)."""
    px = _f32(px)
    npt = px.shape[0]
    xv = _fields(x, npt)
    F = xv.shape[0]
    py = _f32(py) if py is not None else px
    t, o, nt = _tri_or_none(dim, L, px, py, tri)
    y = np.empty((F, npt))
    _check(lib().or_particle_mass_apply(dim, ctypes.c_double(L), _p(px), _p(py), ctypes.c_longlong(npt), _p(t), _p(o),
                                        ctypes.c_longlong(nt), _p(xv), F, _p(y)), "particle_mass_apply")
    return y


def interpolate_lumped(dim, n, L, mesh, px, py=None, tri=None, kind="q1"):
    """Lumped mesh -> particle projection, Abb_mu = c_mu / v_mu (Eq. lumped)."""
    c = g2p_integral(dim, n, L, mesh, px, py, tri, kind)
    if dim == 1:
        v = particle_volumes(1, L, px)
    else:
        v = (tri[2] if tri is not None and tri[2] is not None else triangulate(L, px, py)[2])
    return c / v


def interpolate_mass(dim, n, L, mesh, px, py=None, tri=None, rtol=1e-13, max_iter=20000, kind="q1"):
    """Full mass mesh -> particle projection (Eq. proj2): M_p Abb = c."""
    px = _f32(px)
    py_ = _f32(py) if py is not None else px
    if dim == 2 and tri is None:
        tri = triangulate(L, px, py_)
    c = g2p_integral(dim, n, L, mesh, px, py_, tri, kind)
    F, npt = c.shape
    t, o, nt = _tri_or_none(dim, L, px, py_, tri)
    x = np.empty_like(c)
    it = lib().or_particle_mass_solve(dim, ctypes.c_double(L), _p(px), _p(py_), ctypes.c_longlong(npt), _p(t), _p(o),
                                      ctypes.c_longlong(nt), _p(c), F, ctypes.c_double(rtol), max_iter, _p(x))
    if it < 0:
        raise OracleError(f"oracle particle mass solve failed with status {-it}")
    return x


from . import advect  # noqa: E402  (driver steps of Sec. 3.1-3.3; uses interpolate above)
