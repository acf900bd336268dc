"""GPU parity of the PIC assignment (Eq. PIC with mesh volumes) and of the
stability diagnostics reported by the solves (Eq. stab in integral form:
int Ab^2 = Ab^T M Ab, int A^2 = A^T M_p A), against the oracle, plus the
stability inequalities of the two L2 projections."""
import math

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


def _case(dim, seed):
    if dim == 1:
        inst = W.tophat_1d(n=97, npart=301, seed=seed)
        vals = np.stack([inst.vals[0], np.sin(7 * inst.px)]).astype(np.float32)
        return inst.n, inst.L, inst.px, None, vals
    inst = W.uniform_instance(45, 3, F=2, seed=seed, L=1.3)
    return inst.n, inst.L, inst.px, inst.py, inst.vals


@pytest.mark.parametrize("dim,kind", [(1, "q1"), (2, "q1"), (2, "p1")])
def test_pic_parity_and_conservation(built, dim, kind):
    from paper_1610_05258_gb300 import Context
    n, L, px_h, py_h, vals = _case(dim, 90)
    c = Context(dim, n, L, px_h.size, 2, mesh=kind)
    px, py, dv = to_dev(torch, px_h, py_h, vals)
    got = c.assign_pic(px, py, dv).double().cpu().numpy()
    want = oracle.pic(dim, n, L, px_h, py_h, vals, kind=kind)
    assert rel_l2(got, want) <= TOL
    v = oracle.particle_volumes(dim, L, px_h, py_h)
    h = L / n
    for f in range(2):
        lhs = got[f].sum() * h ** dim
        rhs = float((v * vals[f]).sum())
        assert abs(lhs - rhs) <= 1e-6 * float((v * np.abs(vals[f])).sum())


@pytest.mark.parametrize("dim,kind", [(1, "q1"), (2, "q1"), (2, "p1")])
def test_mass_assignment_energies(built, dim, kind):
    from paper_1610_05258_gb300 import Context
    n, L, px_h, py_h, vals = _case(dim, 91)
    c = Context(dim, n, L, px_h.size, 2, mesh=kind)
    px, py, dv = to_dev(torch, px_h, py_h, vals)
    out, info = c.assign_mass(px, py, dv)
    x = out.double().cpu().numpy()
    tri = oracle.triangulate(L, px_h, py_h) if dim == 2 else None
    em = oracle.energy_mesh(dim, n, L, x, kind)
    ep = oracle.energy_particles(dim, L, px_h, py_h, vals, tri=tri)
    for f in range(2):
        assert info[f].energy_mesh == pytest.approx(em[f], rel=TOL)
        assert info[f].energy_particles == pytest.approx(ep[f], rel=TOL)
        # the mass assignment is an L2 projection: it never adds to int A^2
        assert info[f].energy_mesh <= info[f].energy_particles * (1 + 1e-6)
    # against the oracle's own assignment as well
    want = oracle.assign_mass(dim, n, L, px_h, py_h, vals, tri=tri, kind=kind)
    em_or = oracle.energy_mesh(dim, n, L, want, kind)
    for f in range(2):
        assert info[f].energy_mesh == pytest.approx(em_or[f], rel=TOL)


@pytest.mark.parametrize("dim,fmax", [(1, 2), (2, 2), (2, 5)])
def test_full_mass_interpolation_energies(built, dim, fmax):
    """fmax = 5: a context sized for more fields than the call projects (the
    solve's interleaved width follows the call's field count, 2, not 8)."""
    from paper_1610_05258_gb300 import Context
    n, L, px_h, py_h, _ = _case(dim, 92)
    mesh = W.mesh_field(dim, n, L, F=2, seed=5).astype(np.float32)
    c = Context(dim, n, L, px_h.size, fmax)
    px, py, dm = to_dev(torch, px_h, py_h, mesh)
    out, info = c.interpolate_mass(dm, px, py)
    got = out.double().cpu().numpy()
    tri = oracle.triangulate(L, px_h, py_h) if dim == 2 else None
    em = oracle.energy_mesh(dim, n, L, mesh)
    ep = oracle.energy_particles(dim, L, px_h, py_h, got, tri=tri)
    for f in range(2):
        assert info[f].energy_mesh == pytest.approx(em[f], rel=TOL)
        assert info[f].energy_particles == pytest.approx(ep[f], rel=TOL)
        # the full-mass projection onto the particles is a contraction too
        assert info[f].energy_particles <= info[f].energy_mesh * (1 + 1e-6)


def test_mass_solve_reports_mesh_energy(built):
    from paper_1610_05258_gb300 import Context
    n, L = 64, 2 * math.pi
    b = W.mesh_field(2, n, L, F=1, seed=3, kind="noise").astype(np.float32)
    c = Context(2, n, L, 16, 1)
    x, info = c.mass_solve(to_dev(torch, b)[0])
    em = oracle.energy_mesh(2, n, L, x.double().cpu().numpy())
    assert info[0].energy_mesh == pytest.approx(em[0], rel=TOL)
    assert info[0].energy_particles == 0.0
