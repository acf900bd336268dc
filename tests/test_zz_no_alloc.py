"""The allocation-free mass solve (pm_mass_solve_noalloc), called through the
C ABI, gives the same result as the context-based pm_mass_solve on two calls
in a row (the shared scratch keeps the previous call's contents, which must not
leak into the next result). This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1610_05258_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _lib():
    import paper_1610_05258_gb300 as pm
    from paper_1610_05258_gb300 import build
    build.build()
    lib = pm.load_library()
    f = lib.pm_mass_solve_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_matches_context_solve_twice():
    from paper_1610_05258_gb300 import Context
    solve = _lib()
    dim, n, L, F = 2, 96, 1.7, 2
    ctx = Context(dim, n, L, 16, F)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((11, 12)):
        b = torch.from_numpy(W.mesh_field(dim, n, L, F=F, seed=seed, kind="noise").astype(np.float32)).cuda()
        ref, info = ctx.mass_solve(b, rtol=1e-6)
        x = torch.full_like(b, float("nan"))
        iters = (ctypes.c_int * F)()
        res = (ctypes.c_double * F)()
        s = solve(dim, n, ctypes.c_double(L), ctypes.c_void_p(b.data_ptr()), F, ctypes.c_void_p(x.data_ptr()),
                  ctypes.c_double(1e-6), 200, 0, st, iters, res)
        assert s == 0, (call, s)
        for f in range(F):
            assert _rel(x[f], ref[f]) <= TOL, (call, f)
            assert res[f] <= 1e-6
            assert iters[f] == info[f].iters


def test_noalloc_1d_and_rejects_oversize():
    from paper_1610_05258_gb300 import Context
    solve = _lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, L = 1000, 1.0
    ctx = Context(1, n, L, 16, 1)
    b = torch.from_numpy(W.mesh_field(1, n, L, F=1, seed=5, kind="noise").astype(np.float32)).cuda()
    ref, _ = ctx.mass_solve(b, rtol=1e-6)
    x = torch.zeros_like(b)
    s = solve(1, n, ctypes.c_double(L), ctypes.c_void_p(b.data_ptr()), 1, ctypes.c_void_p(x.data_ptr()),
              ctypes.c_double(1e-6), 200, 0, st, None, None)
    assert s == 0
    torch.cuda.synchronize()
    assert _rel(x[0], ref[0]) <= TOL
    big = torch.zeros(2, 1024 * 1024, device="cuda")
    s = solve(2, 1024, ctypes.c_double(1.0), ctypes.c_void_p(big.data_ptr()), 2, ctypes.c_void_p(big.data_ptr()),
              ctypes.c_double(1e-6), 200, 0, st, None, None)
    assert s == 1  # PM_EINVAL: F * n^2 above the 2^20 limit
