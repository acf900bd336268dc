"""Delta interpolation at the particles of the context's last sort, in sorted
order (pm_interpolate_sorted): slot s equals, bit for bit, pm_interpolate at
caller particle perm[s], for every field width, in 1D and 2D, on bilinear and
P1 meshes; with particles so sparse that a block's cells overrun the staged
mesh windows (the corners beyond them read from the mesh directly); and it is
refused before any sort or with a different count."""
import numpy as np
import pytest

from paper_1610_05258_gb300 import workloads as W
from gpu_util import to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()
    return True


@pytest.mark.parametrize("dim,F,mesh_kind", [(2, 1, "q1"), (2, 2, "q1"), (2, 4, "q1"), (2, 6, "q1"), (2, 3, "p1"),
                                             (1, 1, "q1"), (1, 4, "q1")])
def test_sorted_interpolation_matches_caller_order(built, dim, F, mesh_kind):
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(45, 3, F=F, seed=700 + F) if dim == 2 else W.tophat_1d(157, 611, seed=700 + F)
    vals = inst.vals if inst.vals.shape[0] == F else np.repeat(inst.vals[:1], F, axis=0)
    c = Context(dim, inst.n, inst.L, inst.np, 8, mesh=mesh_kind)
    px, py, dv = to_dev(torch, inst.px, inst.py, vals)
    mesh = to_dev(torch, W.mesh_field(dim, inst.n, inst.L, F=F, seed=9, kind="noise").astype(np.float32))[0]
    c.assign_mass(px, py, dv, info=False)  # sorts the particles
    got = c.interpolate_sorted(mesh, inst.np).clone()
    perm, _ = c.sort(px, py)
    want = c.interpolate(mesh, px, py)
    assert torch.equal(got, want[:, perm.long()])


@pytest.mark.parametrize("n,ppc,F", [(200, 0.05, 4), (300, 0.02, 2), (64, 0.5, 6), (4, 30, 3), (5, 0.4, 4)])
def test_sorted_interpolation_sparse_and_tiny(built, n, ppc, F):
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(n, ppc, F=F, seed=720 + n)
    c = Context(2, n, inst.L, inst.np, F)
    px, py, dv = to_dev(torch, inst.px, inst.py, inst.vals)
    mesh = to_dev(torch, W.mesh_field(2, n, inst.L, F=F, seed=11, kind="noise").astype(np.float32))[0]
    perm, _ = c.sort(px, py)
    got = c.interpolate_sorted(mesh, inst.np).clone()
    want = c.interpolate(mesh, px, py)
    assert torch.equal(got, want[:, perm.long()])


def test_sorted_interpolation_refusals(built):
    from paper_1610_05258_gb300 import Context, PMError
    inst = W.uniform_instance(20, 2, F=1, seed=711)
    c = Context(2, inst.n, inst.L, inst.np, 1)
    mesh = torch.zeros(1, inst.n * inst.n, device="cuda")
    with pytest.raises(PMError):
        c.interpolate_sorted(mesh, inst.np)  # nothing sorted yet
    px, py = to_dev(torch, inst.px, inst.py)
    c.sort(px, py)
    with pytest.raises(PMError):
        c.interpolate_sorted(mesh, inst.np - 1)
    assert c.interpolate_sorted(mesh, inst.np).shape == (1, inst.np)
