"""Mesh -> particle projections other than delta (lumped and full mass,
Table 1 right column; Eq. lumped, Eq. proj2) and the lumped assignment,
through the C ABI against the FP64 oracle on the same seeded inputs.
Tolerance: relative L2 <= 1e-5; the full-mass solve to 1e-6 relative
residual, conservation error <= 1e-6."""
import math

import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W
from gpu_util import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    ("uniform_n40_ppc4", lambda: W.uniform_instance(40, 4, F=2, seed=201)),
    ("uniform_n37_ppc1", lambda: W.uniform_instance(37, 1, F=1, seed=202)),
    ("zalesak_n48", lambda: W.zalesak(48, seed=203)),
    ("taylor_green_n33", lambda: W.taylor_green(33, 4, seed=204)),
    ("uniform_n17_ppc5", lambda: W.uniform_instance(17, 5, F=2, seed=205)),
    ("tophat_128", lambda: W.tophat_1d(128, 128, seed=16101)),
    ("tophat_ragged", lambda: W.tophat_1d(203, 517, seed=7)),
    ("tophat_sparse", lambda: W.tophat_1d(300, 40, seed=8)),
]


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


def setup(inst, F=2, seed=0):
    from paper_1610_05258_gb300 import Context
    mesh = W.mesh_field(inst.dim, inst.n, inst.L, F=F, seed=seed, kind="noise")
    c = Context(inst.dim, inst.n, inst.L, inst.np, F)
    dm, px = to_dev(torch, mesh, inst.px)
    py = to_dev(torch, inst.py)[0] if inst.dim == 2 else None
    return c, mesh, dm, px, py


@pytest.mark.parametrize("name,mk", CASES)
def test_interpolate_lumped(built, name, mk):
    inst = mk()
    c, mesh, dm, px, py = setup(inst, seed=11)
    got = c.interpolate_lumped(dm, px, py).cpu().numpy()
    want = oracle.interpolate_lumped(inst.dim, inst.n, inst.L, mesh, inst.px, inst.py)
    for f in range(mesh.shape[0]):
        assert rel_l2(got[f], want[f]) <= TOL, (f, rel_l2(got[f], want[f]))


@pytest.mark.parametrize("name,mk", CASES)
def test_interpolate_mass(built, name, mk):
    inst = mk()
    c, mesh, dm, px, py = setup(inst, seed=12)
    got, info = c.interpolate_mass(dm, px, py, rtol=1e-6)
    got = got.cpu().numpy()
    want = oracle.interpolate_mass(inst.dim, inst.n, inst.L, mesh, inst.px, inst.py)
    h = inst.L / inst.n
    for f in range(mesh.shape[0]):
        assert rel_l2(got[f], want[f]) <= TOL, (f, rel_l2(got[f], want[f]))
        assert info[f].rel_resid <= 1e-6
        assert info[f].cons_err <= 1e-6
        # sum_mesh is int Ab
        assert info[f].sum_mesh == pytest.approx(h ** inst.dim * mesh[f].sum(), rel=1e-5, abs=1e-7)


@pytest.mark.parametrize("name,mk", CASES)
def test_assign_lumped(built, name, mk):
    from paper_1610_05258_gb300 import Context
    inst = mk()
    c = Context(inst.dim, inst.n, inst.L, inst.np, inst.F)
    px, py, vals = to_dev(torch, inst.px, inst.py, inst.vals)
    got = c.assign_lumped(px, py, vals).cpu().numpy()
    want = oracle.rhs(inst.dim, inst.n, inst.L, inst.px, inst.py, inst.vals) / (inst.L / inst.n) ** inst.dim
    for f in range(inst.F):
        assert rel_l2(got[f], want[f]) <= TOL


def test_full_mass_keeps_constants_and_interpolants(built):
    """A constant mesh field projects to the same constant on the particles
    (both projections); the full mass projection of the mass assignment of
    particle values returns close to them (the two L2 projections)."""
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(32, 4, F=1, seed=206)
    c = Context(2, inst.n, inst.L, inst.np, 1)
    px, py = to_dev(torch, inst.px, inst.py)
    k = torch.full((1, inst.n ** 2), 1.75, device="cuda")
    a, _ = c.interpolate_mass(k, px, py)
    assert torch.allclose(a, torch.full_like(a, 1.75), rtol=1e-5)
    b = c.interpolate_lumped(k, px, py)
    assert torch.allclose(b, torch.full_like(b, 1.75), rtol=1e-5)


def test_projection_errors(built):
    from paper_1610_05258_gb300 import Context, PMError
    inst = W.uniform_instance(16, 2, F=1, seed=207)
    c = Context(2, 16, inst.L, inst.np, 1)
    px, py = to_dev(torch, inst.px, inst.py)
    k = torch.zeros(2, 256, device="cuda")
    with pytest.raises(PMError) as e:  # more fields than the context holds
        c.interpolate_mass(k, px, py)
    assert e.value.status == 1
    # max_iter = 0 on a non-trivial field: not converged, reported
    m = torch.from_numpy(W.mesh_field(2, 16, inst.L, F=1, seed=3, kind="noise")).float().cuda()
    with pytest.raises(PMError) as e:
        c.interpolate_mass(m, px, py, max_iter=0)
    assert e.value.status == 3
    out, info = c.interpolate_mass(m, px, py)  # usable afterwards
    assert info[0].rel_resid <= 1e-6


@pytest.mark.parametrize("dim,F", [(2, 1), (2, 3), (2, 4), (2, 6), (2, 8), (1, 4), (1, 7)])
def test_interpolate_mass_field_counts(built, dim, F):
    """Every interleave width of the particle solve (2, 4 and 8 fields per
    particle record, fields past F padded), in a context sized for 8 fields:
    parity, residual and conservation per field; a field of zeros stays
    zero."""
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(29, 4, F=1, seed=300 + F) if dim == 2 else W.tophat_1d(157, 389, seed=300 + F)
    mesh = W.mesh_field(dim, inst.n, inst.L, F=F, seed=40 + F, kind="noise").astype(np.float32)
    if F > 2:
        mesh[1] = 0.0
    c = Context(dim, inst.n, inst.L, inst.np, 8)
    dm, px = to_dev(torch, mesh, inst.px)
    py = to_dev(torch, inst.py)[0] if dim == 2 else None
    got, info = c.interpolate_mass(dm, px, py, rtol=1e-6)
    got = got.cpu().numpy()
    want = oracle.interpolate_mass(dim, inst.n, inst.L, mesh, inst.px, inst.py)
    for f in range(F):
        if not mesh[f].any():
            assert not got[f].any(), f
            continue
        assert rel_l2(got[f], want[f]) <= TOL, (f, rel_l2(got[f], want[f]))
        assert info[f].rel_resid <= 1e-6 and info[f].cons_err <= 1e-6
    back = c.interpolate(dm, px, py).cpu().numpy()
    want_d = oracle.interpolate(dim, inst.n, inst.L, mesh, inst.px, inst.py)
    for f in range(F):
        if mesh[f].any():
            assert rel_l2(back[f], want_d[f]) <= TOL, f
