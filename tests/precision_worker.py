"""Runs one precision-study case on the GPU with a given build of the
library (loaded from its path) and saves the result; started as a separate
process by tests/test_gpu_precision.py, one per build, because a process
loads one build. Inputs are the seeded workload recipes; no oracle here.

    python tests/precision_worker.py <libpmt.so> <case> <out.npz>
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

NU = 0.01


def initial_mesh(case, inst):
    from paper_1610_05258_gb300 import workloads as W
    n, L = inst.n, inst.L
    x = np.arange(n) * (L / n)
    if case.startswith("tophat"):
        return ((x >= 0.25) & (x < 0.5)).astype(np.float64)[None, :]
    X, Y = np.meshgrid(x, x, indexing="xy")
    if case == "zalesak":
        return W.zalesak_indicator(X.ravel(), Y.ravel()).astype(np.float64)[None, :]
    return np.stack([(np.sin(X) * np.cos(Y)).ravel(), (-np.cos(X) * np.sin(Y)).ravel()])


def instance(case):
    from paper_1610_05258_gb300 import workloads as W
    if case.startswith("tophat"):
        return W.tophat_1d()
    if case == "zalesak":
        return W.zalesak(128)
    if case == "taylor_green":
        return W.taylor_green(128, 4, seed=16103)
    if case == "batched":
        return W.uniform_instance(96, 4, F=3, seed=16104 * 1000 + 7)
    return W.mixture(128, 4, F=4, seed=16105)


def main():
    libpath, case, out = sys.argv[1:4]
    import torch
    import paper_1610_05258_gb300 as pm
    pm.load_library(libpath)
    inst = instance(case)
    dim, n, L = inst.dim, inst.n, inst.L
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    px, py = t(inst.px), t(inst.py)
    cons = []
    if case in ("batched", "mixture"):
        c = pm.Context(dim, n, L, inst.np, inst.F)
        m, info = c.assign_mass(px, py, t(inst.vals))
        cons = [i.cons_err for i in info]
    elif case.startswith("tophat"):
        c = pm.Context(1, n, L, inst.np, 1)
        m = t(initial_mesh(case, inst))
        start = "direct" if case == "tophat_direct" else "delta"
        for _ in range(256):
            vals = c.interpolate(m, px)
            c.advect_shift(px, None, 1.0 / 256)
            m, info = c.assign_mass(px, None, vals, warm_start=start)
            cons.append(info[0].cons_err)
    else:
        mesh0 = initial_mesh(case, inst)
        c = pm.Context(dim, n, L, inst.np, mesh0.shape[0])
        m0 = t(mesh0)
        vals = c.interpolate(m0, px, py)
        if case == "zalesak":
            c.advect_rotate(px, py, 0.5, 0.5, 2 * math.pi / 1000)
        else:
            h = L / n
            c.advect_rk2(m0, vals, px, py, 0.5 * h, vals=vals, factor=math.exp(-2 * NU * 0.5 * h))
        m, info = c.assign_mass(px, py, vals)
        cons = [i.cons_err for i in info]
    torch.cuda.synchronize()
    np.savez(out, mesh=m.double().cpu().numpy(), px=px.cpu().numpy(), py=(py.cpu().numpy() if py is not None else 0),
             cons=np.array(cons))


if __name__ == "__main__":
    main()
