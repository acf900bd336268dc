"""Chebyshev solve of the mesh system (PM_SOLVER_CHEBYSHEV) through the C ABI
against the FP64 oracle's direct solve: bilinear and P1 meshes in 2D (quad
and ragged sides), 1D; the mass assignment built on it; the number of steps
against the Chebyshev bound. Tolerance: relative L2 <= 1e-5, residual 1e-6,
conservation 1e-6."""
import math

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


# (dim, n, mesh kind, smallest eigenvalue of M / h^dim)
CASES = [(2, 40, "q1", 1 / 9), (2, 37, "q1", 1 / 9), (2, 40, "p1", 1 / 4), (2, 33, "p1", 1 / 4), (1, 203, "q1", 1 / 3)]


@pytest.mark.parametrize("dim,n,kind,lmin", CASES)
def test_chebyshev_solve_matches_direct(built, dim, n, kind, lmin):
    from paper_1610_05258_gb300 import Context
    L = 1.3
    b = W.mesh_field(dim, n, L, F=3, seed=5, kind="noise").astype(np.float32)
    c = Context(dim, n, L, 16, 3, mesh=kind)
    (db,) = to_dev(torch, b)
    x, info = c.mass_solve(db, solver="chebyshev")
    want = oracle.mass_solve(dim, n, L, b.astype(np.float64), kind=kind)
    got = x.cpu().numpy().reshape(3, -1)
    q = (math.sqrt(1 / lmin) - 1) / (math.sqrt(1 / lmin) + 1)
    for f in range(3):
        assert rel_l2(got[f], want[f]) <= 1e-5
        assert info[f].rel_resid <= 1e-6
        # steps within the bound 2 q^k ||r0|| <= 1e-6 ||b|| (plus one restart's worth)
        k = math.ceil(math.log(1e-6 / (2 * info[f].init_rel_resid)) / math.log(q))
        assert info[f].iters <= 2 * k + 2
    # conservation: the mean mode is exact
    h = L / n
    np.testing.assert_allclose(got.astype(np.float64).sum(1) * h ** dim, b.astype(np.float64).sum(1),
                               rtol=1e-6, atol=1e-7 * np.abs(b).sum())


@pytest.mark.parametrize("name,mk", [("mixture_n32_F4", lambda: W.mixture(32, 4, 4)),
                                     ("zalesak_n48", lambda: W.zalesak(48, seed=104))])
def test_chebyshev_mass_assignment(built, name, mk):
    from paper_1610_05258_gb300 import Context
    inst = mk()
    c = Context(2, inst.n, inst.L, inst.np, inst.F)
    px, py, vals = to_dev(torch, inst.px, inst.py, inst.vals)
    out, info = c.assign_mass(px, py, vals, solver="chebyshev")
    want = oracle.assign_mass(2, inst.n, inst.L, inst.px, inst.py, inst.vals)
    assert rel_l2(out.cpu().numpy().reshape(inst.F, -1), want) <= 1e-5
    for f in range(inst.F):
        assert info[f].rel_resid <= 1e-6 and info[f].cons_err <= 1e-6


def test_unknown_solver_is_rejected(built):
    from paper_1610_05258_gb300 import Context
    import ctypes
    import paper_1610_05258_gb300 as pm
    c = Context(2, 16, 1.0, 16, 1)
    b = torch.ones(16 * 16, device="cuda")
    x = torch.empty_like(b)
    o = c._opts("zero", 1e-6, 200, None)
    o.solver = 7
    assert c.lib.pm_mass_solve(c.h, b.data_ptr(), 1, x.data_ptr(), ctypes.byref(o), None) == 1
