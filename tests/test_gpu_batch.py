"""Batched instances (pm_batch_*): every instance equals its single-context
result bit for bit (same kernels, deterministic), matches the oracle, and a
replayed CUDA graph gives the same bits again."""
import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W
from gpu_util import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_batch_matches_single_and_oracle():
    from paper_1610_05258_gb300 import Batch, Context, build
    build.build()
    specs = [(24, 1), (40, 4), (64, 7), (33, 2), (48, 3), (17, 5)]
    insts = [W.uniform_instance(n, ppc, F=2, seed=500 + k) for k, (n, ppc) in enumerate(specs)]
    b = Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=2, streams=0)
    dev = [to_dev(torch, i.px, i.py, i.vals) for i in insts]
    outs = [torch.empty(2, i.n * i.n, device="cuda") for i in insts]
    info = b.assign_mass([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev], outs)
    first = [o.clone() for o in outs]
    for k, inst in enumerate(insts):
        c = Context(2, inst.n, inst.L, inst.np, 2)
        single, sinfo = c.assign_mass(*dev[k], warm_start="direct")
        assert torch.equal(single, outs[k]), k
        want = oracle.assign_mass(2, inst.n, inst.L, inst.px, inst.py, inst.vals)
        for f in range(2):
            assert rel_l2(outs[k][f].cpu().numpy(), want[f]) <= 1e-5
            assert info[k][f].rel_resid <= 1e-6 and info[k][f].cons_err <= 1e-6
            assert info[k][f].iters == sinfo[f].iters
    S, ms = b.tuning()
    assert S in (1, 2, 4, 8, 16) and ms > 0
    # graph replay
    for o in outs:
        o.fill_(float("nan"))
    b.assign_mass([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev], outs, info=False)
    torch.cuda.synchronize()
    for k in range(len(insts)):
        assert torch.equal(first[k], outs[k])
