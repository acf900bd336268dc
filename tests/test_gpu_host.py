"""Mass assignment from host buffers (pm_assign_mass_host): the same result,
bit for bit, as the device-buffer call on the same inputs (the values are
uploaded on a second stream and gathered after the particle functions; the
arithmetic is unchanged), in 1D and 2D, from page-locked and pageable host
memory, over consecutive calls with different values; parity with the oracle;
the device-only start rejected."""
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


CASES = [
    ("uniform_n40_ppc4_F3", lambda: W.uniform_instance(40, 4, F=3, seed=601)),
    ("mixture_n64_F4", lambda: W.mixture(64, 4, 4, seed=602)),
    ("tophat_203_517", lambda: W.tophat_1d(203, 517, seed=603)),
]


def _host(a, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("name,mk", CASES)
def test_host_call_matches_device_call(built, name, mk, pinned):
    from paper_1610_05258_gb300 import Context
    inst = mk()
    F = inst.vals.shape[0]
    c = Context(inst.dim, inst.n, inst.L, inst.np, 4)
    dpx, dpy, dv = to_dev(torch, inst.px, inst.py, inst.vals)
    want, winfo = c.assign_mass(dpx, dpy, dv)
    hpx, hv = _host(inst.px, pinned), _host(inst.vals, pinned)
    hpy = _host(inst.py, pinned) if inst.dim == 2 else None
    got, ginfo = c.assign_mass_host(hpx, hpy, hv)
    assert torch.equal(got, want.cpu())
    for f in range(F):
        assert ginfo[f].iters == winfo[f].iters
        assert ginfo[f].rel_resid == winfo[f].rel_resid
        assert ginfo[f].energy_particles == winfo[f].energy_particles
    # a second call on the same context with other values (staging reused;
    # the upload of the new values must wait for the earlier call's work)
    vals2 = (np.cos(3.0 * inst.vals) + 0.5).astype(np.float32)
    want2 = c.assign_mass(dpx, dpy, to_dev(torch, vals2)[0], info=False).cpu()
    out = torch.empty(F, inst.n ** inst.dim, dtype=torch.float32)
    out = out.pin_memory() if pinned else out
    c.assign_mass_host(hpx, hpy, _host(vals2, pinned), out=out, info=False)
    c.sync()
    assert torch.equal(out, want2)


def test_host_call_oracle_parity_and_rejects_device_start(built):
    from paper_1610_05258_gb300 import Context, PMError
    inst = W.uniform_instance(33, 3, F=2, seed=604)
    c = Context(2, inst.n, inst.L, inst.np, 2)
    got, info = c.assign_mass_host(_host(inst.px, True), _host(inst.py, True), _host(inst.vals, True))
    want = oracle.assign_mass(2, inst.n, inst.L, inst.px, inst.py, inst.vals)
    assert rel_l2(got.double().numpy(), want) <= 1e-5
    for x in info:
        assert x.rel_resid <= 1e-6 and x.cons_err <= 1e-6
    with pytest.raises(PMError):
        c.assign_mass_host(_host(inst.px, True), _host(inst.py, True), _host(inst.vals, True), warm_start="user")


@pytest.mark.parametrize("mesh_kind,rhs,warm", [("p1", "exact", "delta"), ("q1", "appb", "delta"),
                                                 ("q1", "exact", "direct"), ("q1", "exact", "zero")])
def test_host_call_other_modes(built, mesh_kind, rhs, warm):
    """The deferred value gather feeds every right-hand side and start: the
    host call equals the device call bit for bit on the P1 mesh, with the
    App. B right-hand side, and from the direct and zero starts."""
    from paper_1610_05258_gb300 import Context
    inst = W.uniform_instance(48, 4, F=2, seed=610)
    c = Context(2, inst.n, inst.L, inst.np, 2, mesh=mesh_kind)
    dpx, dpy, dv = to_dev(torch, inst.px, inst.py, inst.vals)
    want = c.assign_mass(dpx, dpy, dv, rhs=rhs, warm_start=warm, info=False).cpu()
    got = c.assign_mass_host(_host(inst.px, True), _host(inst.py, True), _host(inst.vals, True), rhs=rhs,
                             warm_start=warm, info=False)
    c.sync()
    assert torch.equal(got, want)
