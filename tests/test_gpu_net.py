"""Learned warm start network on the GPU (tcgen05 for the 32 -> 32 layers)
against the FP64 reference, with the GPU's BF16 storage points emulated in
the reference (weights, inputs, activations and stored gradients rounded to
BF16, round to nearest even). Tolerance rel L2 <= 1e-2."""
import numpy as np
import pytest

from oracle import net as ON
from gpu_util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def bf16(a):
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def rounded_params(theta):
    ps = ON.unflatten(theta)
    return [bf16(p) if k % 2 == 0 else np.asarray(p, np.float64) for k, p in enumerate(ps)]


def fwd_bf16(theta, x):
    """Forward with the GPU's storage precision; returns out and activations."""
    ps = rounded_params(theta)
    acts = [bf16(x)]
    h = acts[0]
    for l in range(4):
        h = ON.conv(h, ps[2 * l], ps[2 * l + 1])
        if l < 3:
            h = bf16(np.maximum(h, 0.0))
        acts.append(h)
    return h[0], acts, ps


def grad_bf16(theta, x, tgt):
    out, acts, ps = fwd_bf16(theta, x)
    r = out - tgt
    g = (r / r.size)[None]
    grads = [None] * 8
    for l in range(3, -1, -1):
        if l < 3:
            g = bf16(g * (acts[l + 1] > 0))
        gx, gW, gb = ON.conv_backward(acts[l], ps[2 * l], g)
        grads[2 * l], grads[2 * l + 1] = gW, gb
        g = gx
    return np.concatenate([q.ravel() for q in grads]), 0.5 * float(np.mean(r * r))


@pytest.fixture(scope="module")
def built():
    from paper_1610_05258_gb300 import build
    build.build()


def _inputs(B, n, seed):
    g = np.random.default_rng(seed)
    x = g.standard_normal((B, 2, n, n)).astype(np.float32)
    t = (0.3 * np.roll(x[:, 0], 1, axis=-1) - 0.2 * x[:, 1]).astype(np.float32)
    return x, t


def _theta(seed):
    th = ON.init_params(seed)
    th[-289:-1] *= 10.0  # last layer at full scale for a meaningful comparison
    th[-1] = 0.05
    return th.astype(np.float32)


@pytest.mark.parametrize("B,n", [(1, 128), (2, 256)])
def test_forward_matches_reference(built, B, n):
    from paper_1610_05258_gb300 import Net
    x, _ = _inputs(B, n, 1)
    theta = _theta(2)
    net = Net(n, B)
    net.load(theta)
    out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    for b in range(B):
        want, _, _ = fwd_bf16(theta.astype(np.float64), x[b])
        assert rel_l2(out[b], want) <= 1e-2


def test_gradient_matches_reference(built):
    from paper_1610_05258_gb300 import Net
    B, n = 2, 128
    x, t = _inputs(B, n, 3)
    theta = _theta(4)
    net = Net(n, B)
    net.load(theta)
    loss = net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), lr=0.0)
    g = net.grad()
    want = np.zeros_like(g, dtype=np.float64)
    wl = 0.0
    for b in range(B):
        gb, lb = grad_bf16(theta.astype(np.float64), x[b], t[b])
        want += gb / B
        wl += lb / B
    assert loss == pytest.approx(wl, rel=1e-3)
    # per parameter block
    offs = np.cumsum([0] + [int(np.prod(s)) for s in ON.param_shapes()])
    for k in range(8):
        assert rel_l2(g[offs[k]:offs[k + 1]], want[offs[k]:offs[k + 1]]) <= 1e-2, k


def test_training_reduces_loss_and_checkpoint_resumes(built):
    from paper_1610_05258_gb300 import Net
    B, n = 2, 128
    x, t = _inputs(B, n, 5)
    dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    net = Net(n, B)
    net.load(ON.init_params(6).astype(np.float32))
    losses = [net.train_step(dx, dt, lr=3e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0]
    theta, mom, step = net.state()
    a = [net.train_step(dx, dt, lr=3e-3) for _ in range(5)]
    net2 = Net(n, B)
    net2.load(theta, mom, step)
    b = [net2.train_step(dx, dt, lr=3e-3) for _ in range(5)]
    assert a == b
    np.testing.assert_array_equal(net.state()[0], net2.state()[0])


def test_net_warm_start_keeps_the_solution(built):
    import oracle
    from paper_1610_05258_gb300 import Context, Net, workloads as W
    inst = W.uniform_instance(128, 3, F=2, seed=77)
    c = Context(2, 128, inst.L, inst.np, 2)
    px, py, vals = (torch.from_numpy(a).cuda() for a in (inst.px, inst.py, inst.vals))
    net = Net(128, 2)
    net.load(ON.init_params(8).astype(np.float32))
    out, info = c.assign_mass(px, py, vals, net=net)
    want = oracle.assign_mass(2, inst.n, inst.L, inst.px, inst.py, inst.vals)
    for f in range(2):
        assert rel_l2(out.cpu().numpy()[f], want[f]) <= 1e-5
        assert info[f].rel_resid <= 1e-6 and info[f].cons_err <= 1e-6


def test_trained_network_gains_over_delta_start(built):
    """The shipped network (trained on 2000 delta -> mass pairs of 256^2
    mixture instances) on a held-out 512^2 instance: for the random-phase
    fields, where the delta start is poor, the start residual drops and CG
    needs fewer iterations; every field still reaches the residual."""
    import math
    from paper_1610_05258_gb300 import Context, Net, warmstart
    n, F = 512, 4
    px, py, vals = warmstart.mixture_gpu(torch, n, 4, F, seed=424242, device="cuda")
    ctx = Context(2, n, 2.0 * math.pi, px.numel(), F)
    net = Net(n, F)
    warmstart.load_weights(net)
    _, plain = ctx.assign_mass(px, py, vals)
    _, learned = ctx.assign_mass(px, py, vals, net=net)
    for f in (2, 3):
        assert learned[f].init_rel_resid < 0.3 * plain[f].init_rel_resid, (f, learned[f], plain[f])
        assert learned[f].iters < plain[f].iters
    for f in range(F):
        assert learned[f].rel_resid <= 1e-6 and learned[f].cons_err <= 1e-6
        if plain[f].init_rel_resid < 1e-4:
            # gated: a field whose delta start is already this close keeps it
            assert learned[f].init_rel_resid == plain[f].init_rel_resid, (f, learned[f], plain[f])
