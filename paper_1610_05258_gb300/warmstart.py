"""Training and evaluation of the learned warm start of the mass solve.

Pairs come from the library itself: for a particle set and its fields,
``Context.net_features`` gives the network input (delta assignment / max|A|,
64 (b - M delta) / (h^2 max|A|)) and ``Context.assign_mass`` (plain CG from
the delta start, 1e-6 residual) gives the target; the network learns
64 (mass - delta) / max|A|. Particle sets follow the benchmark's mixture
workload: a 10x density contrast from 8 periodic Gaussians, Taylor-Green and
random-phase fields; inputs are drawn on the GPU with torch (input
generation only, none of the method's arithmetic).

    python -m paper_1610_05258_gb300.warmstart --pairs 2000 --steps 1500 --out ckpt.npz
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

RSCALE = 64.0  # the library's residual / output scale of the network


def mixture_gpu(torch, n, ppc, F, seed, device, contrast=10.0, ncomp=8, grid=256):
    """Particles by rejection from rho ~ 1 + (contrast - 1) g / max g (g: sum of
    periodic Gaussians of width 0.05 L), fields: Taylor-Green u, v and
    random-phase fields with spectral slope -3 (zero mean, unit RMS)."""
    L = 2.0 * math.pi
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    cen = torch.rand(ncomp, 2, generator=gen, device=device, dtype=torch.float64) * L
    sig = 0.05 * L
    c = (torch.arange(grid, device=device, dtype=torch.float64) + 0.5) * (L / grid)
    X, Y = torch.meshgrid(c, c, indexing="xy")
    dens = torch.zeros(grid, grid, device=device, dtype=torch.float64)
    for k in range(ncomp):
        dx = torch.remainder(X - cen[k, 0] + L / 2, L) - L / 2
        dy = torch.remainder(Y - cen[k, 1] + L / 2, L) - L / 2
        dens += torch.exp(-(dx * dx + dy * dy) / (2 * sig * sig))
    rho = 1.0 + (contrast - 1.0) * dens / dens.max()
    rho = (rho / rho.max()).float()
    N = ppc * n * n
    xs, ys, have = [], [], 0
    while have < N:
        k = int((N - have) * 3.5) + 1024
        x = torch.rand(k, generator=gen, device=device) * L
        y = torch.rand(k, generator=gen, device=device) * L
        ix = torch.clamp((x / L * grid).long(), 0, grid - 1)
        iy = torch.clamp((y / L * grid).long(), 0, grid - 1)
        acc = torch.rand(k, generator=gen, device=device) < rho[iy, ix]
        xs.append(x[acc])
        ys.append(y[acc])
        have += int(acc.sum().item())
    px = torch.cat(xs)[:N].contiguous()
    py = torch.cat(ys)[:N].contiguous()
    px = torch.where(px >= L, torch.zeros_like(px), px)
    py = torch.where(py >= L, torch.zeros_like(py), py)
    # particles must be distinct under the library's torus coordinates
    # (x -> floor(frac(fl32(x fl32(1/L))) 2^32)); redraw the rare coincident ones
    invL = torch.tensor(1.0 / L, dtype=torch.float32, device=device)
    for _ in range(8):
        tx = px * invL
        ty = py * invL
        kx = ((tx - torch.floor(tx)) * 4294967296.0).to(torch.int64) & 0xFFFFFFFF
        ky = ((ty - torch.floor(ty)) * 4294967296.0).to(torch.int64) & 0xFFFFFFFF
        key = (kx << 32) | ky
        srt, order = torch.sort(key)
        dup = torch.zeros_like(key, dtype=torch.bool)
        dup[order[1:]] = srt[1:] == srt[:-1]
        nd = int(dup.sum().item())
        if nd == 0:
            break
        for arr in (px, py):
            arr[dup] = torch.rand(nd, generator=gen, device=device) * L
    vals = [torch.sin(px) * torch.cos(py), -torch.cos(px) * torch.sin(py)]
    m = 128
    kf = torch.fft.fftfreq(m, device=device) * m
    kk = torch.sqrt(kf[None, :] ** 2 + kf[:, None] ** 2)
    amp = torch.where(kk > 0, kk.clamp(min=1e-9) ** -1.5, torch.zeros_like(kk))
    for f in range(F - 2):
        re = torch.randn(m, m, generator=gen, device=device)
        im = torch.randn(m, m, generator=gen, device=device)
        fld = torch.fft.ifft2((re + 1j * im) * amp).real
        fld = (fld - fld.mean()) / fld.std().clamp(min=1e-30)
        gx = px / L * m
        gy = py / L * m
        i0 = torch.floor(gx).long()
        j0 = torch.floor(gy).long()
        s = gx - i0
        t = gy - j0
        i0 %= m
        j0 %= m
        i1 = (i0 + 1) % m
        j1 = (j0 + 1) % m
        vals.append(fld[j0, i0] * (1 - s) * (1 - t) + fld[j0, i1] * s * (1 - t) + fld[j1, i0] * (1 - s) * t +
                    fld[j1, i1] * s * t)
    return px.float(), py.float(), torch.stack(vals[:F]).float().contiguous()


def make_pairs(ctx, px, py, vals):
    """(features [F,2,n,n], target [F,n,n], delta [F,n^2], scale [F])."""
    n = ctx.n
    delta, feat, scale = ctx.net_features(px, py, vals)
    mass = ctx.assign_mass(px, py, vals, warm_start="delta", info=False)
    sc = ctx.torch.tensor(scale, device=delta.device).clamp(min=1e-30)[:, None]
    target = (RSCALE * (mass - delta) / sc).reshape(-1, n, n)
    return feat.reshape(-1, 2, n, n).clone(), target.contiguous()


def generate(torch, n, count, seed0, F=8, ppc=4, device="cuda"):
    from . import Context
    ctx = Context(2, n, 2.0 * math.pi, ppc * n * n, F, device=device)
    feats, tgts = [], []
    k = 0
    while sum(f.shape[0] for f in feats) < count:
        px, py, vals = mixture_gpu(torch, n, ppc, F, seed0 + k, device)
        f, t = make_pairs(ctx, px, py, vals)
        feats.append(f)
        tgts.append(t)
        k += 1
    return torch.cat(feats)[:count].contiguous(), torch.cat(tgts)[:count].contiguous()


def train(net, feats, tgts, steps, batch=8, lr=2e-3, seed=0, log=None):
    torch = net.torch
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    losses = []
    P = feats.shape[0]
    for s in range(steps):
        idx = torch.randint(0, P, (batch,), generator=gen).to(feats.device)
        x = feats.index_select(0, idx).contiguous()
        t = tgts.index_select(0, idx).contiguous()
        rate = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
        want = (s % 50 == 0) or s == steps - 1
        loss = net.train_step(x, t, rate, want_loss=want)
        if want:
            losses.append((s, loss))
            if log:
                log(f"step {s} loss {loss:.4e}")
    return losses


def save(path, net, meta=None):
    theta, mom, step = net.state()
    np.savez(path, theta=theta, moments=mom, step=step, **(meta or {}))


def load(path, net, with_moments=False):
    d = np.load(path)
    net.load(d["theta"], d["moments"] if with_moments else None, int(d["step"]))
    return d


def main():
    import torch

    from . import Net, build

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default="warmstart.npz")
    ap.add_argument("--eval-n", type=int, default=0)
    args = ap.parse_args()
    build.build()
    t0 = time.time()
    feats, tgts = generate(torch, args.n, args.pairs + args.heldout, seed0=1000)
    tr_f, tr_t = feats[: args.pairs], tgts[: args.pairs]
    ho_f, ho_t = feats[args.pairs:], tgts[args.pairs:]
    print(f"generated {feats.shape[0]} pairs in {time.time() - t0:.1f} s")
    net = Net(args.n, args.batch)
    theta0 = init_theta(seed=0)
    net.load(theta0)
    t0 = time.time()
    train(net, tr_f, tr_t, args.steps, args.batch, args.lr, log=print)
    torch.cuda.synchronize()
    print(f"trained {args.steps} steps in {time.time() - t0:.1f} s")
    # held-out relative error of the prediction vs the delta start
    num = den = 0.0
    for k in range(0, ho_f.shape[0], args.batch):
        x = ho_f[k:k + args.batch].contiguous()
        out = net.forward(x)
        t = ho_t[k:k + args.batch]
        num += float(((out - t) ** 2).sum())
        den += float((t ** 2).sum())
    print(f"held-out relative error of the correction: {math.sqrt(num / den):.4f} (delta start: 1.0)")
    save(args.out, net, {"n": args.n, "pairs": args.pairs, "steps": args.steps})
    if args.eval_n:
        inf = Net(args.eval_n, 4)
        inf.load(net.state()[0])
        r = evaluate(torch, inf, args.eval_n, seed=999999)
        print("evaluation", r)


def evaluate(torch, net_or_none, n, seed, F=4, ppc=4, reps=3, device="cuda"):
    """Plain (delta start) vs learned warm start on one mixture instance:
    CG iterations, start residual and time of pm_assign_mass (CUDA events)."""
    from . import Context
    px, py, vals = mixture_gpu(torch, n, ppc, F, seed, device)
    ctx = Context(2, n, 2.0 * math.pi, px.numel(), F, device=device)
    out = {}
    for name, kw in (("plain", {"warm_start": "delta"}), ("learned", {"net": net_or_none})):
        if name == "learned" and net_or_none is None:
            continue
        res, info = ctx.assign_mass(px, py, vals, **kw)
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.assign_mass(px, py, vals, out=res, info=False, **kw)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        out[name] = {"ms": min(ms), "iters": [i.iters for i in info],
                     "init_rel_resid": [i.init_rel_resid for i in info], "rel_resid": [i.rel_resid for i in info]}
    return out


def init_theta(seed=0):
    """He-normal initial parameters in the library's layout (last layer scaled
    by 0.1 so the untrained network starts close to the delta start)."""
    g = np.random.default_rng(seed)
    chans = [2, 32, 32, 32, 1]
    th = []
    for li, (ci, co) in enumerate(zip(chans[:-1], chans[1:])):
        std = math.sqrt(2.0 / (9 * ci)) * (0.1 if li == len(chans) - 2 else 1.0)
        th.append(g.standard_normal(co * ci * 9) * std)
        th.append(np.zeros(co))
    return np.concatenate(th).astype(np.float32)


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_mixture.npz")


def load_weights(net, path=None):
    """Load the trained parameters shipped with the package (trained by this
    module's main() on 2000 pairs of 256^2 mixture instances)."""
    d = np.load(path or WEIGHTS)
    net.load(d["theta"], None, int(d["step"]))
    return d


if __name__ == "__main__":
    main()
