"""Batched instances in one packed workspace (pm_batch_*): every instance's
mass assignment matches the oracle and the single-context result, the step
is a handful of launches whatever the number of instances, a replayed CUDA
graph gives the same bits again, and the delta and zero starts (which run
the per-instance conjugate gradients) reach the same fields."""
import numpy as np
import pytest

import oracle
from paper_1610_05258_gb300 import workloads as W
from gpu_util import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [(24, 1), (40, 4), (64, 7), (33, 2), (48, 3), (17, 5)]


@pytest.fixture(scope="module")
def case():
    from paper_1610_05258_gb300 import build
    build.build()
    insts = [W.uniform_instance(n, ppc, F=2, seed=500 + k) for k, (n, ppc) in enumerate(SPECS)]
    want = [oracle.assign_mass(2, i.n, i.L, i.px, i.py, i.vals) for i in insts]
    return insts, want


def _run(b, insts, info=True, **kw):
    dev = [to_dev(torch, i.px, i.py, i.vals) for i in insts]
    outs = [torch.full((2, i.n * i.n), float("nan"), device="cuda") for i in insts]
    inf = b.assign_mass([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev], outs, info=info, **kw)
    torch.cuda.synchronize()
    return outs, inf, dev


@pytest.mark.parametrize("tune", [0, 256, 1024])
def test_batch_matches_oracle_and_single_context(case, tune):
    from paper_1610_05258_gb300 import Batch, Context
    insts, want = case
    b = Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=2, tune=tune)
    outs, info, dev = _run(b, insts)
    for k, inst in enumerate(insts):
        got = outs[k].double().cpu().numpy()
        assert rel_l2(got, want[k]) <= 1e-5, k
        c = Context(2, inst.n, inst.L, inst.np, 2)
        single, sinfo = c.assign_mass(*dev[k], warm_start="direct")
        assert rel_l2(got, single.double().cpu().numpy()) <= 1e-6, k
        for f in range(2):
            assert info[k][f].rel_resid <= 1e-6 and info[k][f].cons_err <= 1e-6
            assert info[k][f].energy_mesh <= info[k][f].energy_particles * (1 + 1e-6)  # Eq. stab
            assert info[k][f].energy_mesh == pytest.approx(sinfo[f].energy_mesh, rel=1e-5)
            assert info[k][f].energy_particles == pytest.approx(sinfo[f].energy_particles, rel=1e-5)
            assert info[k][f].sum_particles == pytest.approx(sinfo[f].sum_particles, rel=1e-6, abs=1e-12)
    threads, cluster, largest_first, ms = b.tuning()
    assert threads in (256, 512, 1024) and cluster in (1, 4, 8)
    if tune:
        assert threads == tune and cluster == 1 and not largest_first and ms == 0.0
    else:
        assert ms > 0.0


@pytest.mark.parametrize("threads,cluster,largest_first", [(1024, 8, True), (512, 4, False), (256, 8, False)])
def test_batch_solve_on_clusters(case, threads, cluster, largest_first):
    """The per-instance solve on a thread-block cluster (reductions through
    distributed shared memory) gives the same fields, from the exact-inverse
    start and from the zero start (CG iterations across the cluster)."""
    from paper_1610_05258_gb300 import Batch
    insts, want = case
    b = Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=2)
    b.set_tuning(threads, cluster, largest_first)
    assert b.tuning()[:3] == (threads, cluster, largest_first)
    for start in ("direct", "zero"):
        b.set_start(start)
        outs, info, _ = _run(b, insts)
        for k in range(len(insts)):
            assert rel_l2(outs[k].double().cpu().numpy(), want[k]) <= 1e-5, (start, k)
            for f in range(2):
                assert info[k][f].rel_resid <= 1e-6 and info[k][f].cons_err <= 1e-6
                assert info[k][f].energy_mesh <= info[k][f].energy_particles * (1 + 1e-6)
        if start == "zero":
            assert min(x.iters for row in info for x in row) > 0


def test_batch_graph_replay_and_launch_count(case):
    import paper_1610_05258_gb300 as pm
    from paper_1610_05258_gb300 import Batch
    insts, _ = case
    b = Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=2, tune=512)
    dev = [to_dev(torch, i.px, i.py, i.vals) for i in insts]
    outs = [torch.empty(2, i.n * i.n, device="cuda") for i in insts]
    args = ([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev], outs)
    b.assign_mass(*args, info=False)  # captures the step
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    l0 = pm.kernel_launches()
    b.assign_mass(*args, info=False)  # replays it
    torch.cuda.synchronize()
    launches = pm.kernel_launches() - l0
    assert 0 < launches <= 30, launches  # one launch per phase, independent of the instance count
    for k in range(len(insts)):
        assert torch.equal(first[k], outs[k])


@pytest.mark.parametrize("start", ["delta", "zero"])
def test_batch_other_starts_run_conjugate_gradients(case, start):
    from paper_1610_05258_gb300 import Batch
    insts, want = case
    b = Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=2, tune=256)
    b.set_start(start)
    outs, info, _ = _run(b, insts)
    iters = [x.iters for row in info for x in row]
    assert max(iters) > 0
    if start == "zero":
        assert min(iters) > 0
    for k in range(len(insts)):
        assert rel_l2(outs[k].double().cpu().numpy(), want[k]) <= 1e-5, k
        for f in range(2):
            assert info[k][f].rel_resid <= 1e-6 and info[k][f].cons_err <= 1e-6


def test_batch_rejects_bad_arguments(case):
    from paper_1610_05258_gb300 import Batch, PMError
    insts, _ = case
    with pytest.raises(PMError):
        Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=2, tune=300)
    b = Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=2, tune=256)
    with pytest.raises(PMError):
        b.set_start("user")  # not a batch start
    dev = [to_dev(torch, i.px, i.py, i.vals) for i in insts]
    big = [torch.zeros(i.np + 1, device="cuda") for i in insts]  # more particles than the batch holds
    outs = [torch.empty(2, i.n * i.n, device="cuda") for i in insts]
    with pytest.raises(PMError):
        b.assign_mass(big, big, [d[2] for d in dev], outs)
