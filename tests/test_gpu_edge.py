"""Edge cases through the C ABI: zero fields, too few particles, too many
fields, a particle set too sparse for the triangulation's search rings (an
error status, never a fault, and the context stays usable), and the largest
field count through the mass assignment."""
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


def test_zero_fields_give_zero_without_iterations(built):
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(32, 3, F=2, seed=41)
    c = Context(2, inst.n, inst.L, inst.np, 2)
    px, py = to_dev(torch, inst.px, inst.py)
    z = torch.zeros(2, inst.np, device="cuda")
    for solver in ("cg", "chebyshev"):
        out, info = c.assign_mass(px, py, z, solver=solver)
        assert torch.count_nonzero(out).item() == 0
        assert all(i.iters == 0 and i.rel_resid == 0.0 for i in info)


def test_argument_errors(built):
    from paper_1610_05258_gb300 import Context, PMError
    c = Context(2, 16, 1.0, 64, 2)
    two = torch.tensor([0.1, 0.6], device="cuda")
    with pytest.raises(PMError) as e:
        c.assign_mass(two, two, torch.ones(1, 2, device="cuda"))
    assert e.value.status == 1
    px = torch.rand(32, device="cuda")
    with pytest.raises(PMError) as e:
        c.assign_mass(px, px.flip(0), torch.ones(3, 32, device="cuda"))  # 3 fields > max 2
    assert e.value.status == 1


def test_sparse_set_is_reported_and_context_survives(built):
    """Four particles on a 32^2 mesh: their Voronoi cells reach past the
    search rings (n/4 - 1 = 7 cells), which the triangulation reports."""
    from paper_1610_05258_gb300 import Context, PMError
    c = Context(2, 32, 1.0, 4096, 1)
    g = np.random.default_rng(3)
    few = g.uniform(0, 1, (2, 4)).astype(np.float32)
    px, py = to_dev(torch, few[0], few[1])
    with pytest.raises(PMError) as e:
        c.assign_mass(px, py, torch.ones(1, 4, device="cuda"))
    assert e.value.status == 5  # PM_EDEGENERATE
    inst = W.uniform_instance(32, 4, F=1, seed=9)
    qx, qy, v = to_dev(torch, inst.px, inst.py, inst.vals)
    out, info = c.assign_mass(qx, qy, v)
    assert info[0].rel_resid <= 1e-6
    want = oracle.assign_mass(2, inst.n, inst.L, inst.px, inst.py, inst.vals)
    assert rel_l2(out.cpu().numpy().reshape(1, -1), want) <= 1e-5


def test_max_fields(built):
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(24, 3, F=8, seed=108)
    c = Context(2, inst.n, inst.L, inst.np, 8)
    px, py, v = to_dev(torch, inst.px, inst.py, inst.vals)
    out, info = c.assign_mass(px, py, v)
    want = oracle.assign_mass(2, inst.n, inst.L, inst.px, inst.py, inst.vals)
    assert rel_l2(out.cpu().numpy().reshape(8, -1), want) <= 1e-5
    assert all(i.rel_resid <= 1e-6 and i.cons_err <= 1e-6 for i in info)
