"""Benchmark of the particle <-> mesh transfer hot path on GB300.

One JSON line per run. Workloads (--workload), after the benchmark
configurations of the learned-warm-start study of arXiv 1610.05258's method:

* mixture (default)  2048^2 periodic bilinear mesh on [0, 2 pi)^2 and
                     16,777,216 particles drawn from a Gaussian mixture with
                     10x density contrast; F = 4 (Taylor-Green u, v and two
                     random-phase fields). Step = one mass assignment (sort,
                     Delaunay stars, exact right-hand side, CG to 1e-6). The
                     headline `value` is the plain solve (delta warm start);
                     the same step with the learned warm start is reported
                     under "learned".
* tophat             1D periodic convection of a top-hat: 128 nodes, 128
                     particles, step = G2P -> shift by u dt -> mass P2G
                     (delta and FLIP variants reported beside it).
* zalesak            2D slotted disk: 256^2 mesh, 262,144 jittered particles,
                     step = G2P -> rotation by 2 pi / 1000 -> mass P2G
                     (delta and FLIP beside it).
* taylor_green       1024^2 mesh, 4.2M particles, F = 2, step = G2P ->
                     midpoint move with the mesh velocity and viscous decay
                     -> mass P2G.
* batched            256 instances of sides 64..512 and 1..8 particles per
                     cell, F = 3, every instance assigned once per step.

Metric: particles * fields / s of the mass assignment step. Inputs are
device-resident; the L2 cache (129 MB) is flushed by writing a 512 MB buffer
before every timed step; every step is timed with CUDA events on the
launching stream. "e2e" repeats the step through the public API with pinned
host buffers (host -> device inputs and device -> host results inside the
timed region).

cpu_baseline: the FP64 C oracle as it stands, run on a bounded sample of the
workload in one process per host core (spawned), each process on its own
seeded sample; the line records the core count and the CPU model, the
throughput of all cores and of one core, and the relative L2 difference
between the GPU path and the oracle on the same sample. --impl reference
times the same oracle sample as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time
from concurrent.futures import ProcessPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mass-assignment particles*fields/s at 1e-6 residual (plain CG, delta warm start); % HBM peak"
UNIT = "particle-fields/s"
NU = 0.01
WORKLOADS = ("mixture", "tophat", "zalesak", "taylor_green", "batched")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


def host_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        self.path = os.path.join("/tmp", f"pm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# The oracle on a bounded sample of each workload (cpu_baseline and the
# reference arm). Each unit of work is one step of the workload on the sample.
# ---------------------------------------------------------------------------
def _sample(workload, seed):
    from paper_1610_05258_gb300 import workloads as W
    if workload == "mixture":
        inst = W.mixture(32, 4, F=4, seed=16105 + seed)
        return {"inst": inst, "what": "mixture recipe on a 32^2 mesh (4096 particles, F=4), one mass assignment"}
    if workload == "tophat":
        inst = W.tophat_1d(seed=16101 + seed)
        return {"inst": inst, "what": "the full configuration (128 nodes, 128 particles, F=1), one "
                                      "G2P -> shift -> mass P2G step"}
    if workload == "zalesak":
        inst = W.zalesak(64, seed=16102 + seed)
        return {"inst": inst, "what": "Zalesak recipe on a 64^2 mesh (16,384 particles, F=1), one "
                                      "G2P -> rotation -> mass P2G step"}
    if workload == "taylor_green":
        inst = W.taylor_green(32, 4, seed=16103 + seed)
        return {"inst": inst, "what": "Taylor-Green recipe on a 32^2 mesh (4096 particles, F=2), one "
                                      "G2P -> midpoint move -> mass P2G step"}
    if workload == "batched":
        inst = W.uniform_instance(48, 4, F=3, seed=16104 * 1000 + seed)
        return {"inst": inst, "what": "one batched-recipe instance of side 48 (4 particles/cell, F=3), "
                                      "one mass assignment"}
    raise ValueError(workload)


def _initial_mesh(workload, inst):
    import numpy as np
    from paper_1610_05258_gb300 import workloads as W
    n, L = inst.n, inst.L
    x = np.arange(n) * (L / n)
    if workload == "tophat":
        return ((x >= 0.25) & (x < 0.5)).astype(np.float64)[None, :]
    X, Y = np.meshgrid(x, x, indexing="xy")
    if workload == "zalesak":
        return W.zalesak_indicator(X.ravel(), Y.ravel()).astype(np.float64)[None, :]
    return np.stack([(np.sin(X) * np.cos(Y)).ravel(), (-np.cos(X) * np.sin(Y)).ravel()])


def _oracle_step(workload, s):
    """One unit of the workload on the oracle; returns (particle-fields, result)."""
    import oracle
    from oracle import advect as OA
    inst = s["inst"]
    dim, n, L = inst.dim, inst.n, inst.L
    if workload in ("mixture", "batched"):
        return inst.np * inst.F, oracle.assign_mass(dim, n, L, inst.px, inst.py, inst.vals)
    mesh = s.setdefault("mesh", _initial_mesh(workload, inst))
    vals = oracle.interpolate(dim, n, L, mesh, inst.px, inst.py)
    if workload == "tophat":
        px, py = OA.shift(L, inst.px, None, 1.0 / 256)
    elif workload == "zalesak":
        px, py = OA.rotate(L, inst.px, inst.py, 0.5, 0.5, 2 * math.pi / 1000)
    else:
        h = L / n
        dt = 0.5 * h
        px, py, vals = OA.rk2(dim, n, L, mesh, vals, inst.px, inst.py, dt, vals=vals,
                              factor=math.exp(-2 * NU * dt))
    return inst.np * mesh.shape[0], (px, py, oracle.assign_mass(dim, n, L, px, py, vals))


def _oracle_worker(workload, seed, seconds):
    s = _sample(workload, seed)
    _oracle_step(workload, s)
    t0 = time.perf_counter()
    units = reps = 0
    while True:
        u, _ = _oracle_step(workload, s)
        units += u
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return units, time.perf_counter() - t0, reps


_CACHE = {}


def _oracle_once(workload, seed):
    """One unit of the workload on this process's cached sample."""
    key = (workload, seed)
    if key not in _CACHE:
        _CACHE[key] = _sample(workload, seed)
    u, _ = _oracle_step(workload, _CACHE[key])
    return u


def _gpu_sample_result(workload, pm, torch, dev, s):
    """The GPU path on the oracle's sample (same inputs, same step)."""
    import numpy as np
    inst = s["inst"]
    dim, n, L = inst.dim, inst.n, inst.L
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    F = inst.F if workload in ("mixture", "batched") else _initial_mesh(workload, inst).shape[0]
    ctx = pm.Context(dim, n, L, inst.np, F, device=dev)
    px, py = t(inst.px), t(inst.py)
    if workload in ("mixture", "batched"):
        out, _ = ctx.assign_mass(px, py, t(inst.vals))
        return out.double().cpu().numpy()
    mesh = t(_initial_mesh(workload, inst))
    vals = ctx.interpolate(mesh, px, py)
    if workload == "tophat":
        ctx.advect_shift(px, None, 1.0 / 256)
    elif workload == "zalesak":
        ctx.advect_rotate(px, py, 0.5, 0.5, 2 * math.pi / 1000)
    else:
        h = L / n
        ctx.advect_rk2(mesh, vals, px, py, 0.5 * h, vals=vals, factor=math.exp(-2 * NU * 0.5 * h))
    out, _ = ctx.assign_mass(px, py, vals)
    return out.double().cpu().numpy()


def cpu_baseline(workload, seconds, pm=None, torch=None, dev=None):
    """The oracle timed on all host cores (one spawned process per core, each
    on its own seeded sample), and the GPU path's relative L2 difference from
    the oracle on sample 0."""
    import numpy as np
    hi = host_info()
    P = hi["nproc"] or 1
    with ProcessPoolExecutor(max_workers=P, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, [workload] * P, range(P), [seconds] * P))
    rates = [u / t for u, t, _ in res]
    s = _sample(workload, 0)
    out = {"value": float(sum(rates)), "unit": UNIT, "cores": P, "kind": "oracle",
           "single_core_value": float(statistics.median(rates)), "cpu_model": hi["cpu_model"],
           "sample": f"{s['what']}; FP64 C oracle, {P} processes for {seconds:.0f} s each "
                     f"({sum(r for _, _, r in res)} steps)"}
    if pm is not None:
        _, want = _oracle_step(workload, s)
        if workload not in ("mixture", "batched"):
            want = want[2]
        got = _gpu_sample_result(workload, pm, torch, dev, _sample(workload, 0))
        out["gpu_rel_l2_vs_oracle"] = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    return out


def run_reference(args):
    """The oracle as the reference arm: each step runs one unit of the
    workload's sample on every host core at once (spawned processes)."""
    if args.world > 1 and args.rank != 0:
        return
    hi = host_info()
    P = getattr(args, "ref_procs", 0) or hi["nproc"] or 1
    times = []
    units = 0

    def one_step(run):
        t0 = time.perf_counter()
        res = run()
        return time.perf_counter() - t0, sum(res)

    if P == 1:
        steps = [one_step(lambda: [_oracle_once(args.workload, 0)]) for _ in range(args.warmup + args.steps)]
    else:
        with ProcessPoolExecutor(max_workers=P, mp_context=mp.get_context("spawn")) as ex:
            steps = [one_step(lambda: list(ex.map(_oracle_once, [args.workload] * P, range(P))))
                     for _ in range(args.warmup + args.steps)]
    for dt, u in steps[args.warmup:]:
        times.append(dt)
        units = u
    t = sum(times) / len(times)
    v = units / t
    s0 = _sample(args.workload, 0)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: bounded CPU sample ({s0['what']}) in each of {P} processes",
                   "host": hi},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": P, "kind": "oracle", "cpu_model": hi["cpu_model"],
                         "sample": f"{s0['what']}; one step per process per timed step, FP64 C oracle"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# Rooflines
# ---------------------------------------------------------------------------
# Roofline of the triangulation (the dominant kernel of the 2D steps): it is
# bound by ALU issue, not by memory. Its algorithmic operation count per
# launch is the arithmetic of the clipping algorithm on the actual particle
# set: the kernel's counting build (pm_profile mode 2) counts, over all
# particles, the candidates examined, the candidates passing the distance
# bound, the in-circle vertex tests, the clips and the cell sizes after each
# clip; each is weighted by the FP32/INT32 arithmetic instructions of that
# step as written (an FMA counts as one): distance test 10, margin set-up 5,
# vertex test 5, clip with two circumcentres and error bounds 80, radius bound
# 9 per vertex. Divergence, address arithmetic, loads and stores are not
# counted.
DELAUNAY_OP_WEIGHTS = {"candidates": 10, "tested": 5, "vertex_tests": 5, "clips": 80, "cell_size_sum": 9}
# ALU peak: 152 SMs x 128 FP32 lanes x one instruction per lane per clock.
ALU_LANES = 152 * 128
# DRAM traffic of one k_delaunay launch per particle: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture on the 1024^2 mixture (4,194,304
# particles: 100.11 MB read + 106.89 MB written), scaled to a launch by its
# particle count (the kernel's traffic grows in proportion to it).
DELAUNAY_DRAM_BYTES_PER_PARTICLE = (100.109568e6 + 106.889216e6) / 4194304


def alu_roofline(kernel, counts, ms, sm_mhz, n_particles):
    ops = float(sum(DELAUNAY_OP_WEIGHTS[k] * counts[k] for k in DELAUNAY_OP_WEIGHTS))
    achieved = ops / (ms * 1e-3) / 1e12
    peak = ALU_LANES * sm_mhz * 1e6 / 1e12
    return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": DELAUNAY_DRAM_BYTES_PER_PARTICLE * n_particles,
            "traffic_source": "ncu dram bytes of k_delaunay on the 1024^2 mixture, scaled by particles",
            "ops_per_launch": ops, "work_counts": counts,
            "peak_source": f"derived: 152 SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock sampled during the "
                           f"timed region)"}


def hbm_roofline(kernel, algo_bytes, ms, what, traffic=None):
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    achieved = algo_bytes / (ms * 1e-3) / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "algorithmic_bytes": algo_bytes, "bytes": what,
            "peak_source": "measured copy bandwidth (MEASURED_PEAKS hbm_gbs)"}


def g2p_bytes(N, nodes, F, dim=2):
    """Minimal bytes of one G2P: positions (4 dim B) in and F values (4 B
    each) out per particle, F mesh values (4 B each) in per node."""
    return N * (4 * dim + 4 * F) + nodes * 4 * F


def chain_step_bytes(N, nodes, F, dim):
    """Minimal bytes of one G2P -> move -> P2G step: the G2P, the positions
    read and written by the move, and the P2G's positions and values in and
    mesh fields out."""
    return g2p_bytes(N, nodes, F, dim) + N * 8 * dim + N * (4 * dim + 4 * F) + nodes * 4 * F


def max_over_ranks(torch, dist, value, device):
    """The slowest rank's value (the job's time); the value itself on one rank."""
    if not dist:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(torch, stream, flush, steps, fn):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def timed_arm(ctx, torch, stream, flush, args, dist, dev, fn, pm):
    """Warm-up, then exactly args.steps timed steps with per-phase profiling;
    returns (mean ms over the slowest rank, launches, phase ms per step)."""
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = pm.kernel_launches()
    ms = time_steps(torch, stream, flush, args.steps, fn)
    launches = pm.kernel_launches() - l0
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    t = max_over_ranks(torch, dist, sum(ms) / len(ms), dev)
    return t, launches, {k: v[0] / args.steps for k, v in prof.items() if v[0] > 0}


def solve_report(info):
    return {"iters": [i.iters for i in info], "init_rel_resid": [i.init_rel_resid for i in info],
            "rel_resid": [i.rel_resid for i in info], "cons_err": [i.cons_err for i in info],
            "energy_mesh": [i.energy_mesh for i in info], "energy_particles": [i.energy_particles for i in info]}


def finish(args, dist, line):
    if args.rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def base_line(args, value, ms, config, **extra):
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config, **extra}


# ---------------------------------------------------------------------------
# mixture (learned warm start configuration), the default
# ---------------------------------------------------------------------------
def run_mixture(args, pm, torch, dist, local):
    """One mass assignment of 16.8M mixture particles and 4 fields on a 2048^2
    mesh per step, plain (delta start) and learned (network start), both to
    1e-6 relative residual; other starts, right-hand sides, solvers and mesh
    functions as extra arms; the mesh -> particle projections of the result."""
    from paper_1610_05258_gb300 import warmstart as WS

    dev = torch.device("cuda", local)
    n, F, ppc = args.n, 4, 4
    L = 2.0 * math.pi
    px, py, vals = WS.mixture_gpu(torch, n, ppc, F, seed=16105 + 7919 * args.rank, device=dev)
    N = px.numel()
    ctx = pm.Context(2, n, L, N, F, device=dev)
    net = pm.Net(n, F, device=dev)
    WS.load_weights(net)
    out = torch.empty(F, n * n, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    arms = {"plain": {"warm_start": "delta"}, "learned": {"net": net}, "direct": {"warm_start": "direct"},
            "appb": {"warm_start": "delta", "rhs": "appb"}, "cheb": {"warm_start": "delta", "solver": "chebyshev"}}
    res = {}
    clocks = Clocks(local)
    for name, kw in arms.items():
        _, info = ctx.assign_mass(px, py, vals, out=out, **kw)
        if name == "plain":
            clocks.start()
        t, launches, phases = timed_arm(ctx, torch, stream, flush, args, dist, dev,
                                        lambda: ctx.assign_mass(px, py, vals, out=out, info=False, **kw), pm)
        if name == "plain":
            ck = clocks.stop()
        res[name] = {"ms": t, "launches": launches, "info": info, "phase_ms": phases}

    # ---- end to end through the public API: pinned host positions and values
    # in, converged mesh fields out, every step (pm_assign_mass_host: the
    # values upload under the sort and the particle functions)
    e2e = None
    if not args.no_e2e:
        hpx, hpy, hvals = px.cpu().pin_memory(), py.cpu().pin_memory(), vals.cpu().pin_memory()
        hout = torch.empty(F, n * n).pin_memory()
        bi = (hpx.numel() + hpy.numel() + hvals.numel()) * 4
        bo = hout.numel() * 4

        def e2e_step():
            ctx.assign_mass_host(hpx, hpy, hvals, out=hout, info=False)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks(torch, dist, sum(time_steps(torch, stream, flush, args.steps, e2e_step)) / args.steps, dev)
        e2e = {"value": args.world * N * F / (te * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": te}

    plain, learned, direct, appb, cheb = res["plain"], res["learned"], res["direct"], res["appb"], res["cheb"]
    # the same step with P1 mesh functions (cells split by the (0,0)-(1,1) diagonal)
    ctx_p1 = pm.Context(2, n, L, N, F, device=dev, mesh="p1")
    _, p1_info = ctx_p1.assign_mass(px, py, vals, out=out)
    p1_t, _, p1_phases = timed_arm(ctx_p1, torch, stream, flush, args, dist, dev,
                                   lambda: ctx_p1.assign_mass(px, py, vals, out=out, info=False), pm)
    del ctx_p1
    # mesh -> particle projections of the assigned fields back onto the same
    # particles: full mass (Eq. proj2, CG to 1e-6), lumped (Eq. lumped), delta
    mesh_fields = out.clone()
    back = torch.empty(F, N, device=dev)
    _, pinfo = ctx.interpolate_mass(mesh_fields, px, py, out=back)
    proj = {}
    for name, fn in (("full_mass", lambda: ctx.interpolate_mass(mesh_fields, px, py, out=back, info=False)),
                     ("lumped", lambda: ctx.interpolate_lumped(mesh_fields, px, py, out=back)),
                     ("delta", lambda: ctx.interpolate(mesh_fields, px, py, out=back)),
                     # the same particles, already sorted by the calls above: results in sorted order
                     ("delta_sorted", lambda: ctx.interpolate_sorted(mesh_fields, N, out=back))):
        t, _, phases = timed_arm(ctx, torch, stream, flush, args, dist, dev, fn, pm)
        proj[name] = {"ms_per_step": t, "value": args.world * N * F / (t * 1e-3),
                      "phase_ms_per_step": {k: round(v, 4) for k, v in phases.items()}}
    proj["full_mass"]["solve"] = solve_report(pinfo)
    g2p_ms = proj["delta"]["ms_per_step"]
    g2p_sorted_ms = proj["delta_sorted"]["ms_per_step"]
    # one untimed pass of the counting build of the triangulation
    ctx.profile(True, count_work=True)
    ctx.assign_mass(px, py, vals, out=out, info=False)
    counts = ctx.work_read()
    ctx.profile(False)
    sm = ck.get("sm_mhz") or float(measured_peaks().get("sm_max_mhz", 2070.0))
    dom = max(plain["phase_ms"], key=plain["phase_ms"].get)
    roof = alu_roofline("k_delaunay (phase triangulate)", counts, plain["phase_ms"]["triangulate"], sm, N)
    roof["dominant_phase"] = dom
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    minimal = N * (8 + 4 * F) + n * n * 4 * F  # positions + values in, fields out
    roof["hbm_minimal_io"] = {"bytes_per_step": minimal, "achieved_gbs": minimal / (plain["ms"] * 1e-3) / 1e9,
                              "peak_gbs": hbm, "frac": minimal / (plain["ms"] * 1e-3) / 1e9 / hbm}
    rooflines = [hbm_roofline("k_interleave + k_g2p (mesh -> particle, Eq. delta2)", g2p_bytes(N, n * n, F), g2p_ms,
                              "8 B position + 4F B values per particle, 4F B per node"),
                 hbm_roofline("k_interleave + k_g2p_sorted (Eq. delta2 at the sorted particles, sorted results)",
                              g2p_bytes(N, n * n, F), g2p_sorted_ms,
                              "8 B position + 4F B values per particle, 4F B per node")]

    cpu = cpu_baseline("mixture", 10.0, pm, torch, dev) if (args.rank == 0 and not args.no_cpu) else None

    def arm(r, what=None):
        d = {"value": args.world * N * F / (r["ms"] * 1e-3), "ms_per_step": r["ms"],
             "speedup_vs_plain": plain["ms"] / r["ms"],
             "phase_ms_per_step": {k: round(v, 4) for k, v in r["phase_ms"].items()},
             "solve": solve_report(r["info"]), "gpu_launches": r["launches"]}
        if what:
            d["what"] = what
        return d

    line = base_line(
        args, args.world * N * F / (plain["ms"] * 1e-3), plain["ms"],
        {"workload": f"mixture_{n}x{n}_ppc{ppc}_F{F}: {N} particles by rejection from a 10x-contrast "
                     f"Gaussian mixture, F={F} (Taylor-Green u, v, two random-phase fields), {n}x{n} "
                     f"periodic bilinear mesh, L=2pi; step = one mass assignment to 1e-6 relative "
                     f"residual (delta warm start)",
         "l2": "flushed before every timed step (512 MB write)", "parallelism": f"replicas x{args.world}"},
        phase_ms_per_step={k: round(v, 4) for k, v in plain["phase_ms"].items()},
        solve=solve_report(plain["info"]),
        learned={**arm(learned, "4-layer 3x3 conv 2-32-32-32-1, BF16 tcgen05, shipped weights"),
                 "network": "4-layer 3x3 conv 2-32-32-32-1, BF16 tcgen05, shipped weights"},
        direct_start=arm(direct, "start = exact inverse of the periodic mass matrix (separable circulant "
                                 "convolutions), then CG confirms the residual"),
        appb_rhs=arm(appb, "the same step with the App. B quadrature right-hand side (delta on the twice refined "
                           "mesh, 3x3 box sum) instead of the exact one; not conservative"),
        chebyshev=arm(cheb, "the same step with the mesh system solved by Chebyshev iteration on the closed-form "
                            "spectrum (no inner products) instead of CG"),
        p1_mesh={"value": args.world * N * F / (p1_t * 1e-3), "ms_per_step": p1_t,
                 "phase_ms_per_step": {k: round(v, 4) for k, v in p1_phases.items()},
                 "solve": solve_report(p1_info),
                 "what": "the same step with P1 mesh functions on cells split by the (0,0)-(1,1) diagonal "
                         "(7-point mass stencil) instead of bilinear ones"},
        mesh_to_particle={"what": "the step's mesh fields projected back onto the same particles; each entry is "
                                  "one call per step (full mass includes the sort and triangulation; delta_sorted "
                                  "interpolates at the particles the previous calls sorted, results in sorted order)",
                          **proj},
        roofline=roof, rooflines=rooflines, cpu_baseline=cpu, e2e=e2e, gpu_launches=plain["launches"], clocks=ck)
    finish(args, dist, line)


# ---------------------------------------------------------------------------
# time-stepping chains: tophat (1D), zalesak, taylor_green
# ---------------------------------------------------------------------------
def run_chain(args, pm, torch, dist, local):
    import numpy as np
    from paper_1610_05258_gb300 import workloads as W

    dev = torch.device("cuda", local)
    wl = args.workload
    if wl == "tophat":
        inst = W.tophat_1d(seed=16101 + args.rank)
    elif wl == "zalesak":
        inst = W.zalesak(256, seed=16102 + args.rank)
    else:
        inst = W.taylor_green(args.n, 4, seed=16103 + args.rank)
    dim, n, L, N = inst.dim, inst.n, inst.L, inst.np
    mesh0 = _initial_mesh(wl, inst)
    F = mesh0.shape[0]
    h = L / n
    dt = 1.0 / 256 if wl == "tophat" else 0.5 * h
    decay = math.exp(-2.0 * NU * dt)
    nodes = n ** dim
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    ctx = pm.Context(dim, n, L, N, F, device=dev)
    px0, py0 = t(inst.px), t(inst.py)
    px, py = px0.clone(), (py0.clone() if py0 is not None else None)
    vel = torch.empty(F, N, device=dev)
    mesh = [t(mesh0), torch.empty(F, nodes, device=dev)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def advect(m_in, qx, qy, v):
        if wl == "tophat":
            ctx.advect_shift(qx, None, dt)
        elif wl == "zalesak":
            ctx.advect_rotate(qx, qy, 0.5, 0.5, 2 * math.pi / 1000)
        else:
            ctx.advect_rk2(m_in, v, qx, qy, dt, vals=v, factor=decay)

    def make_step(method):
        def step():
            m_in, m_out = mesh
            ctx.interpolate(m_in, px, py, out=vel)
            advect(m_in, px, py, vel)
            if method == "mass":
                ctx.assign_mass(px, py, vel, out=m_out, info=False)
            elif method == "delta":
                ctx.assign_delta(px, py, vel, out=m_out)
            else:
                ctx.assign_flip(px, py, vel, out=m_out)
            mesh.reverse()
        return step

    clocks = Clocks(local)
    arms = ["mass"] if wl == "taylor_green" else ["mass", "delta", "flip"]
    res = {}
    for method in arms:
        px.copy_(px0)
        if py is not None:
            py.copy_(py0)
        mesh[0].copy_(t(mesh0))
        if method == "mass":
            clocks.start()
        tm, launches, phases = timed_arm(ctx, torch, stream, flush, args, dist, dev, make_step(method), pm)
        if method == "mass":
            ck = clocks.stop()
            ctx.interpolate(mesh[0], px, py, out=vel)
            advect(mesh[0], px, py, vel)
            _, info = ctx.assign_mass(px, py, vel, out=mesh[1])
        res[method] = {"ms": tm, "launches": launches, "phase_ms": phases}
    mass = res["mass"]

    # ---- end to end: the step's inputs (positions and the mesh fields) from
    # pinned host memory, its results (the new mesh fields and the moved
    # positions) back into host memory, every step. The next step starts from
    # those host copies, so this chain passes through the same states as the
    # device-resident one (same start, same number of steps).
    e2e = None
    if not args.no_e2e:
        hpx = px0.cpu().pin_memory()
        hpy = py0.cpu().pin_memory() if py0 is not None else None
        hmesh = [t(mesh0).cpu().pin_memory(), torch.empty(F, nodes).pin_memory()]
        dpx = torch.empty_like(px0)
        dpy = torch.empty_like(py0) if py0 is not None else None
        dmesh, dout = torch.empty_like(mesh[0]), torch.empty_like(mesh[0])
        bi = (hpx.numel() + (hpy.numel() if hpy is not None else 0) + hmesh[0].numel()) * 4
        bo = bi

        def e2e_step():
            dpx.copy_(hpx, non_blocking=True)
            if dpy is not None:
                dpy.copy_(hpy, non_blocking=True)
            dmesh.copy_(hmesh[0], non_blocking=True)
            ctx.interpolate(dmesh, dpx, dpy, out=vel)
            advect(dmesh, dpx, dpy, vel)
            ctx.assign_mass(dpx, dpy, vel, out=dout, info=False)
            hmesh[1].copy_(dout, non_blocking=True)
            hpx.copy_(dpx, non_blocking=True)
            if dpy is not None:
                hpy.copy_(dpy, non_blocking=True)
            hmesh.reverse()

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks(torch, dist, sum(time_steps(torch, stream, flush, args.steps, e2e_step)) / args.steps, dev)
        e2e = {"value": args.world * N * F / (te * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": te}

    sm = ck.get("sm_mhz") or float(measured_peaks().get("sm_max_mhz", 2070.0))
    dom = max(mass["phase_ms"], key=mass["phase_ms"].get)
    if dim == 2:
        ctx.profile(True, count_work=True)
        ctx.assign_mass(px, py, vel, out=mesh[1], info=False)
        counts = ctx.work_read()
        ctx.profile(False)
        roof = alu_roofline("k_delaunay (phase triangulate)", counts, mass["phase_ms"]["triangulate"], sm, N)
    else:
        roof = hbm_roofline("whole step (every kernel of 128 particles is launch-latency bound)",
                            chain_step_bytes(N, nodes, F, dim), mass["ms"], "G2P + shift + mass P2G minimal I/O")
    roof["dominant_phase"] = dom
    rooflines = []
    if "g2p" in mass["phase_ms"]:
        rooflines.append(hbm_roofline("k_g2p (mesh -> particle, Eq. delta2)", g2p_bytes(N, nodes, F, dim),
                                      mass["phase_ms"]["g2p"], "8 B position + 4F B values per particle, "
                                                               "4F B per node"))
    cpu = cpu_baseline(wl, 10.0, pm, torch, dev) if (args.rank == 0 and not args.no_cpu) else None
    desc = {"tophat": f"tophat_1d: {n} nodes, {N} uniform random particles on [0, 1), top-hat on [0.25, 0.5), "
                      f"u = 1, dt = 1/256; step = G2P -> shift -> mass P2G (1e-6)",
            "zalesak": f"zalesak_{n}x{n}: {N} particles (2x2 jittered lattice per cell), slotted-disk indicator, "
                       f"rotation by 2pi/1000 about (0.5, 0.5) per step; step = G2P -> rotation -> mass P2G (1e-6)",
            "taylor_green": f"taylor_green_{n}x{n}: {N} particles (4 per cell, uniform random), F=2 (u, v), L=2pi, "
                            f"nu=0.01, dt=h/2; step = G2P -> midpoint move with the mesh velocity and "
                            f"exp(-2 nu dt) decay -> mass P2G (1e-6)"}[wl]
    extra = {m: {"value": args.world * N * F / (r["ms"] * 1e-3), "ms_per_step": r["ms"],
                 "phase_ms_per_step": {k: round(v, 4) for k, v in r["phase_ms"].items()}}
             for m, r in res.items() if m != "mass"}
    line = base_line(args, args.world * N * F / (mass["ms"] * 1e-3), mass["ms"],
                     {"workload": desc, "l2": "flushed before every timed step (512 MB write)",
                      "parallelism": f"replicas x{args.world}"},
                     phase_ms_per_step={k: round(v, 4) for k, v in mass["phase_ms"].items()},
                     solve=solve_report(info), other_assignments=extra, roofline=roof, rooflines=rooflines,
                     cpu_baseline=cpu, e2e=e2e, gpu_launches=mass["launches"], clocks=ck)
    finish(args, dist, line)


# ---------------------------------------------------------------------------
# batched instances
# ---------------------------------------------------------------------------
def run_batched(args, pm, torch, dist, local):
    """Many independent 2D instances (sides uniform in 64..512, 1..8 uniform
    random particles per cell, F = 3 smooth random fields), one mass
    assignment of every instance per step."""
    from paper_1610_05258_gb300 import workloads as W

    dev = torch.device("cuda", local)
    insts = W.batched(args.instances, seed=16104 + 7919 * args.rank)
    F = insts[0].F
    N = sum(i.np for i in insts)
    nodes = sum(i.n * i.n for i in insts)
    b = pm.Batch([i.n for i in insts], [i.L for i in insts], [i.np for i in insts], max_fields=F, device=dev)
    pxs = [torch.from_numpy(i.px).to(dev) for i in insts]
    pys = [torch.from_numpy(i.py).to(dev) for i in insts]
    vals = [torch.from_numpy(i.vals).to(dev) for i in insts]
    outs = [torch.empty(F, i.n * i.n, device=dev) for i in insts]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    info = b.assign_mass(pxs, pys, vals, outs)
    for _ in range(args.warmup):
        b.assign_mass(pxs, pys, vals, outs, info=False)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = pm.kernel_launches()
    ms = time_steps(torch, stream, flush, args.steps, lambda: b.assign_mass(pxs, pys, vals, outs, info=False))
    launches = pm.kernel_launches() - l0
    ck = clocks.stop()
    t = max_over_ranks(torch, dist, sum(ms) / len(ms), dev)

    # ---- end to end: every instance's positions and values from pinned host
    # memory and its mesh fields back, every step. The instances sit packed
    # in one host and one device buffer per array (views per instance), so a
    # step is one copy per array rather than one per instance and array.
    e2e = None
    if not args.no_e2e:
        hpx = torch.cat([x.cpu() for x in pxs]).pin_memory()
        hpy = torch.cat([y.cpu() for y in pys]).pin_memory()
        hv = torch.cat([v.cpu().reshape(-1) for v in vals]).pin_memory()
        ho = torch.empty(sum(F * i.n * i.n for i in insts)).pin_memory()
        dpx, dpy, dv, dout = (torch.empty_like(a, device=dev) for a in (hpx, hpy, hv, ho))
        vpx, vpy, vv, vout = [], [], [], []
        po = vo = oo = 0
        for i in insts:
            vpx.append(dpx[po:po + i.np])
            vpy.append(dpy[po:po + i.np])
            vv.append(dv[vo:vo + F * i.np].view(F, i.np))
            vout.append(dout[oo:oo + F * i.n * i.n].view(F, i.n * i.n))
            po, vo, oo = po + i.np, vo + F * i.np, oo + F * i.n * i.n
        bi = (hpx.numel() + hpy.numel() + hv.numel()) * 4
        bo = ho.numel() * 4

        def e2e_step():
            dpx.copy_(hpx, non_blocking=True)
            dpy.copy_(hpy, non_blocking=True)
            dv.copy_(hv, non_blocking=True)
            b.assign_mass(vpx, vpy, vv, vout, info=False)
            ho.copy_(dout, non_blocking=True)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks(torch, dist, sum(time_steps(torch, stream, flush, args.steps, e2e_step)) / args.steps, dev)
        e2e = {"value": args.world * N * F / (te * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": te}

    flat = [x for row in info for x in row]
    minimal = N * (8 + 4 * F) + nodes * 4 * F
    roof = hbm_roofline("whole batched step (triangulation-dominated, ALU-bound like the single-instance step)",
                        minimal, t, "minimal I/O: 8 + 4F B per particle in, 4F B per node out")
    cpu = cpu_baseline("batched", 10.0, pm, torch, dev) if (args.rank == 0 and not args.no_cpu) else None
    tune = b.tuning()
    line = base_line(
        args, args.world * N * F / (t * 1e-3), t,
        {"workload": f"batched: {len(insts)} instances, sides 64..512, 1..8 particles/cell, F={F}, "
                     f"{N} particles, {nodes} nodes; one mass assignment of every instance per step to 1e-6",
         "l2": "flushed before every timed step (512 MB write)", "parallelism": f"replicas x{args.world}",
         "tuning": tune},
        solve={"max_iters": max(x.iters for x in flat), "max_rel_resid": max(x.rel_resid for x in flat),
               "max_cons_err": max(x.cons_err for x in flat),
               "stability_holds": all(x.energy_mesh <= x.energy_particles * (1 + 1e-6) for x in flat)},
        gpu_launches=launches, clocks=ck, cpu_baseline=cpu, e2e=e2e, roofline=roof)
    finish(args, dist, line)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixture", choices=list(WORKLOADS))
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--n", type=int, default=0, help="mesh side (default 2048 mixture, 1024 taylor_green)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-procs", type=int, default=0, help="oracle processes of the reference arm (0 = all cores)")
    args = ap.parse_args()
    if not args.n:
        args.n = 2048 if args.workload == "mixture" else 1024
    args.rank = int(os.environ.get("RANK", "0"))
    args.world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    import paper_1610_05258_gb300 as pm
    from paper_1610_05258_gb300 import build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if args.world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.rank == 0:
        build.build()
    if dist:
        dist.barrier()
    pm.load_library()

    if args.workload == "batched":
        return run_batched(args, pm, torch, dist, local)
    if args.workload == "mixture":
        return run_mixture(args, pm, torch, dist, local)
    return run_chain(args, pm, torch, dist, local)


if __name__ == "__main__":
    main()
