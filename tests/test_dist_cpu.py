"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
the reduction of the step time over ranks, and the reference arm's rank
handling. One process per rank, rendezvous on 127.0.0.1."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(torch, dist, 10.0 + 3.5 * rank, torch.device("cpu"))
        q.put((rank, got))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_step_time_is_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: 13.5, 1: 13.5}


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 4.25, torch.device("cpu")) == 4.25


def test_reference_arm_rank_handling(monkeypatch):
    """Under torchrun only rank 0 runs the oracle and prints; other ranks exit
    quietly."""
    sys.path.insert(0, ROOT)
    import bench

    class A:
        world, rank, gpus, steps, warmup = 2, 1, 2, 1, 0
        workload, ref_procs = "mixture", 1

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A)
    assert buf.getvalue() == ""

    calls = []
    monkeypatch.setattr(bench, "_sample", lambda w, seed: calls.append(1) or {"inst": _tiny(), "what": "tiny"})
    monkeypatch.setattr(bench, "_CACHE", {})

    class B(A):
        rank = 0

    with redirect_stdout(buf):
        bench.run_reference(B)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and calls
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def _tiny():
    from paper_1610_05258_gb300 import workloads as W
    return W.mixture(16, 2, F=1, seed=3)


def test_alu_roofline_arithmetic():
    """The triangulation's roofline: weighted work counts over the phase time,
    the lane peak at the given clock, DRAM traffic in proportion to particles."""
    import bench
    counts = {k: 0 for k in bench.DELAUNAY_OP_WEIGHTS}
    counts["clips"] = 10 ** 9
    r = bench.alu_roofline("k", counts, 10.0, 2000.0, 4194304)
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["achieved"] == pytest.approx(80e9 / 1e-2 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == pytest.approx(100.109568e6 + 106.889216e6)  # the 1024^2 capture's DRAM bytes
    assert bench.alu_roofline("k", counts, 10.0, 2000.0, 2 * 4194304)["traffic"] == pytest.approx(2 * r["traffic"])
