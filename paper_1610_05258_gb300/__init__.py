"""GB300-native particle <-> mesh field transfer (arXiv 1610.05258).

A thin ctypes binding over the C ABI in ``include/pmt.h``; every step of the
transfer runs in the library's CUDA kernels. PyTorch provides device memory
and the current stream only. Importing this package does not load the
library; the first Context does, and raises if it is missing or no CUDA
device is present. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

__all__ = ["Context", "Batch", "Net", "PMError", "SolveInfo", "load_library", "library_path", "kernel_launches"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.environ.get("PM_LIBRARY") or os.path.join(
    _HERE, "_build_checked" if os.environ.get("PM_CHECKED") == "1" else "_build", "libpmt.so")
_lib = None

PM_WS_DELTA, PM_WS_ZERO, PM_WS_USER, PM_WS_NET, PM_WS_DIRECT = 0, 1, 2, 3, 4
PM_RHS_EXACT, PM_RHS_APPB = 0, 1
PM_MESH_Q1, PM_MESH_P1 = 0, 1
MESH_KINDS = {"q1": PM_MESH_Q1, "p1": PM_MESH_P1}
RHS_MODES = {"exact": PM_RHS_EXACT, "appb": PM_RHS_APPB}
PM_SOLVER_CG, PM_SOLVER_CHEBYSHEV = 0, 1
SOLVERS = {"cg": PM_SOLVER_CG, "chebyshev": PM_SOLVER_CHEBYSHEV}
_STATUS = {0: "PM_OK", 1: "PM_EINVAL", 2: "PM_ENOMEM", 3: "PM_ENOTCONV", 4: "PM_ETIMEOUT", 5: "PM_EDEGENERATE",
           6: "PM_ECUDA"}

EXPORTS = [
    "pm_ctx_create", "pm_ctx_create_mesh", "pm_ctx_destroy", "pm_ctx_set_stream", "pm_sync", "pm_last_error", "pm_ctx_workspace_bytes",
    "pm_interpolate", "pm_interpolate_sorted", "pm_interpolate_lumped", "pm_interpolate_mass", "pm_assign_lumped", "pm_assign_delta", "pm_assign_flip", "pm_assign_mass", "pm_assign_mass_host", "pm_mass_rhs", "pm_mass_rhs_mode", "pm_mass_apply",
    "pm_mass_solve", "pm_particle_volumes", "pm_triangulate", "pm_sort", "pm_advect_shift", "pm_advect_rotate",
    "pm_advect_rk2", "pm_profile", "pm_profile_read", "pm_work_read", "pm_phase_name", "pm_kernel_launches",
    "pm_batch_create", "pm_batch_destroy", "pm_batch_last_error", "pm_batch_tuning", "pm_batch_assign_mass",
    "pm_net_num_params", "pm_net_create", "pm_net_destroy", "pm_net_set_stream", "pm_net_state", "pm_net_load",
    "pm_net_forward", "pm_net_train_step", "pm_net_grad", "pm_net_features",
]
WORK_COUNTERS = ["candidates", "tested", "vertex_tests", "clips", "cell_size_sum", "retried", "retried_last",
                 "exact_tests"]
PHASES = ["sort", "triangulate", "delta", "flip", "rhs", "solve", "g2p", "advect", "other", "net"]


class PMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("warm_start", ctypes.c_int), ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("x0", ctypes.c_void_p), ("net", ctypes.c_void_p), ("rhs_mode", ctypes.c_int),
                ("solver", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("init_rel_resid", ctypes.c_double), ("rel_resid", ctypes.c_double),
                ("sum_particles", ctypes.c_double), ("sum_mesh", ctypes.c_double), ("cons_err", ctypes.c_double),
                ("energy_mesh", ctypes.c_double), ("energy_particles", ctypes.c_double)]


@dataclass
class SolveInfo:
    iters: int
    init_rel_resid: float
    rel_resid: float
    sum_particles: float
    sum_mesh: float
    cons_err: float
    energy_mesh: float = 0.0       # int Ab^2 = Ab^T M Ab (Eq. stab, integral form)
    energy_particles: float = 0.0  # int A^2 = A^T M_p A


def _info(x) -> SolveInfo:
    return SolveInfo(x.iters, x.init_rel_resid, x.rel_resid, x.sum_particles, x.sum_mesh, x.cons_err, x.energy_mesh,
                     x.energy_particles)


def library_path() -> str:
    return _LIBPATH


def load_library(path: str | None = None):
    """Load libpmt.so (built by paper_1610_05258_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIBPATH
    if not os.path.exists(p):
        raise ImportError(f"libpmt.so not built ({p}); run `python -m paper_1610_05258_gb300.build`")
    lib = ctypes.CDLL(p)
    vp, ll, i, d = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_double
    sig = {
        "pm_ctx_create": [ctypes.POINTER(vp), i, i, d, ll, i, vp],
        "pm_ctx_create_mesh": [ctypes.POINTER(vp), i, i, d, ll, i, i, vp],
        "pm_ctx_destroy": [vp],
        "pm_ctx_set_stream": [vp, vp],
        "pm_sync": [vp],
        "pm_last_error": [vp],
        "pm_ctx_workspace_bytes": [vp],
        "pm_interpolate": [vp, vp, i, vp, vp, ll, vp],
        "pm_interpolate_lumped": [vp, vp, i, vp, vp, ll, vp],
        "pm_interpolate_mass": [vp, vp, i, vp, vp, ll, vp, ctypes.POINTER(_Opts), vp],
        "pm_assign_lumped": [vp, vp, vp, ll, vp, i, vp],
        "pm_assign_delta": [vp, vp, vp, ll, vp, i, vp],
        "pm_assign_flip": [vp, vp, vp, ll, vp, i, vp, vp, ctypes.POINTER(ll)],
        "pm_assign_pic": [vp, vp, vp, ll, vp, i, vp],
        "pm_assign_mass": [vp, vp, vp, ll, vp, i, vp, ctypes.POINTER(_Opts), vp],
        "pm_assign_mass_host": [vp, vp, vp, ll, vp, i, vp, ctypes.POINTER(_Opts), vp],
        "pm_interpolate_sorted": [vp, vp, i, ll, vp],
        "pm_mass_rhs": [vp, vp, vp, ll, vp, i, vp],
        "pm_mass_rhs_mode": [vp, vp, vp, ll, vp, i, i, vp],
        "pm_mass_apply": [vp, vp, i, vp],
        "pm_mass_solve": [vp, vp, i, vp, ctypes.POINTER(_Opts), vp],
        "pm_particle_volumes": [vp, vp, vp, ll, vp],
        "pm_triangulate": [vp, vp, vp, ll, vp, vp, ll, ctypes.POINTER(ll)],
        "pm_sort": [vp, vp, vp, ll, vp, vp],
        "pm_advect_shift": [vp, vp, vp, ll, d, d],
        "pm_advect_rotate": [vp, vp, vp, ll, d, d, d],
        "pm_advect_rk2": [vp, vp, vp, vp, vp, ll, d, vp, i, d],
        "pm_profile": [vp, i],
        "pm_profile_read": [vp, vp, vp, i],
        "pm_work_read": [vp, vp, i, i],
        "pm_phase_name": [i],
        "pm_kernel_launches": [],
        "pm_batch_create": [ctypes.POINTER(vp), i, vp, vp, vp, i, i, vp],
        "pm_batch_destroy": [vp],
        "pm_batch_last_error": [vp],
        "pm_batch_tuning": [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d)],
        "pm_batch_set_tuning": [vp, i, i, i],
        "pm_batch_assign_mass": [vp, vp, vp, vp, vp, i, vp, d, i, vp],
        "pm_batch_set_start": [vp, i],
        "pm_net_num_params": [],
        "pm_net_create": [ctypes.POINTER(vp), i, i, vp],
        "pm_net_destroy": [vp],
        "pm_net_set_stream": [vp, vp],
        "pm_net_state": [vp, vp, ctypes.POINTER(ll)],
        "pm_net_load": [vp, vp, i, ll],
        "pm_net_forward": [vp, vp, i, i, vp],
        "pm_net_train_step": [vp, vp, vp, i, i, ctypes.c_float, ctypes.POINTER(d)],
        "pm_net_grad": [vp, vp],
        "pm_net_features": [vp, vp, vp, ll, vp, i, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.pm_last_error.restype = ctypes.c_char_p
    lib.pm_phase_name.restype = ctypes.c_char_p
    lib.pm_batch_last_error.restype = ctypes.c_char_p
    lib.pm_batch_destroy.restype = None
    lib.pm_net_destroy.restype = None
    lib.pm_kernel_launches.restype = ctypes.c_longlong
    lib.pm_ctx_workspace_bytes.restype = ctypes.c_longlong
    lib.pm_ctx_destroy.restype = None
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels this library has launched in the process so far."""
    return load_library().pm_kernel_launches()


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One periodic mesh (dim 1 or 2, n nodes per side, box length L) with
    workspace for up to max_particles particles and max_fields fields; mesh
    functions "q1" (bilinear) or "p1" (linear on cells split by the (0,0)-(1,1)
    diagonal), pm_ctx_create_mesh."""

    def __init__(self, dim: int, n: int, L: float, max_particles: int, max_fields: int = 1, device=None,
                 mesh: str = "q1"):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_1610_05258_gb300 needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device if device is not None else "cuda")
        self.dim, self.n, self.L = dim, n, float(L)
        self.max_particles, self.max_fields = max_particles, max_fields
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = torch.cuda.current_stream().cuda_stream
            s = self.lib.pm_ctx_create_mesh(ctypes.byref(h), dim, n, ctypes.c_double(L), max_particles, max_fields,
                                            MESH_KINDS[mesh], ctypes.c_void_p(st))
        if s != 0:
            raise PMError(s, "pm_ctx_create failed")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and self.lib is not None:
            self.lib.pm_ctx_destroy(self.h)
            self.h = None

    @property
    def workspace_bytes(self) -> int:
        return self.lib.pm_ctx_workspace_bytes(self.h)

    def _stream(self):
        self.lib.pm_ctx_set_stream(self.h, ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream))

    def _check(self, s):
        if s != 0:
            raise PMError(s, self.lib.pm_last_error(self.h).decode())

    def _f32(self, t):
        if t is None:
            return None
        if not (t.is_cuda and t.dtype == self.torch.float32 and t.is_contiguous()):
            raise TypeError("expected a contiguous float32 CUDA tensor")
        return t

    def _empty(self, *shape):
        return self.torch.empty(*shape, dtype=self.torch.float32, device=self.device)

    @property
    def nodes(self) -> int:
        return self.n ** self.dim

    def sync(self):
        self._check(self.lib.pm_sync(self.h))

    def interpolate(self, mesh, px, py=None, out=None):
        mesh, px, py = self._f32(mesh), self._f32(px), self._f32(py)
        F = mesh.numel() // self.nodes
        out = out if out is not None else self._empty(F, px.numel())
        self._stream()
        self._check(self.lib.pm_interpolate(self.h, _ptr(mesh), F, _ptr(px), _ptr(py), px.numel(), _ptr(out)))
        return out

    def interpolate_lumped(self, mesh, px, py=None, out=None):
        """Lumped mesh -> particle projection, c_mu / v_mu (pm_interpolate_lumped)."""
        mesh, px, py = self._f32(mesh), self._f32(px), self._f32(py)
        F = mesh.numel() // self.nodes
        out = out if out is not None else self._empty(F, px.numel())
        self._stream()
        self._check(self.lib.pm_interpolate_lumped(self.h, _ptr(mesh), F, _ptr(px), _ptr(py), px.numel(), _ptr(out)))
        return out

    def interpolate_sorted(self, mesh, np_, out=None):
        """Delta G2P at the particles of the context's last sort, results in
        that sorted order (pm_interpolate_sorted); np_ = that call's count."""
        mesh = self._f32(mesh)
        F = mesh.numel() // self.nodes
        out = out if out is not None else self._empty(F, np_)
        self._stream()
        self._check(self.lib.pm_interpolate_sorted(self.h, _ptr(mesh), F, np_, _ptr(out)))
        return out

    def interpolate_mass(self, mesh, px, py=None, out=None, rtol=1e-6, max_iter=200, info=True):
        """Full mass mesh -> particle projection (pm_interpolate_mass)."""
        mesh, px, py = self._f32(mesh), self._f32(px), self._f32(py)
        F = mesh.numel() // self.nodes
        out = out if out is not None else self._empty(F, px.numel())
        o = self._opts("delta", rtol, max_iter, None)
        inf = (_Info * F)() if info else None
        self._stream()
        self._check(self.lib.pm_interpolate_mass(self.h, _ptr(mesh), F, _ptr(px), _ptr(py), px.numel(), _ptr(out),
                                                 ctypes.byref(o), inf))
        if not info:
            return out
        return out, [_info(x)
                     for x in inf]

    def assign_lumped(self, px, py, vals, out=None):
        """Lumped assignment, int A psi_i / h^dim (pm_assign_lumped)."""
        px, py, vals = self._f32(px), self._f32(py), self._f32(vals)
        F = vals.numel() // max(1, px.numel())
        out = out if out is not None else self._empty(F, self.nodes)
        self._stream()
        self._check(self.lib.pm_assign_lumped(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F, _ptr(out)))
        return out

    def assign_delta(self, px, py, vals, out=None):
        px, py, vals = self._f32(px), self._f32(py), self._f32(vals)
        F = vals.numel() // max(1, px.numel())
        out = out if out is not None else self._empty(F, self.nodes)
        self._stream()
        self._check(self.lib.pm_assign_delta(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F, _ptr(out)))
        return out

    def assign_flip(self, px, py, vals, out=None, node_volume=None, count_empty=False):
        px, py, vals = self._f32(px), self._f32(py), self._f32(vals)
        F = vals.numel() // max(1, px.numel())
        out = out if out is not None else self._empty(F, self.nodes)
        e = ctypes.c_longlong(0)
        self._stream()
        self._check(self.lib.pm_assign_flip(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F, _ptr(out),
                                            _ptr(node_volume), ctypes.byref(e) if count_empty else None))
        return (out, e.value) if count_empty else out

    def assign_pic(self, px, py, vals, out=None):
        """PIC assignment with the mesh volumes h^dim (pm_assign_pic)."""
        px, py, vals = self._f32(px), self._f32(py), self._f32(vals)
        F = vals.numel() // max(1, px.numel())
        out = out if out is not None else self._empty(F, self.nodes)
        self._stream()
        self._check(self.lib.pm_assign_pic(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F, _ptr(out)))
        return out

    def _opts(self, warm_start, rtol, max_iter, x0, net=None, rhs="exact", solver="cg"):
        ws = {"delta": PM_WS_DELTA, "zero": PM_WS_ZERO, "user": PM_WS_USER, "net": PM_WS_NET,
              "direct": PM_WS_DIRECT}[warm_start]
        return _Opts(ws, rtol, max_iter, x0.data_ptr() if x0 is not None else None, net.h.value if net else None,
                     RHS_MODES[rhs], SOLVERS[solver])

    def assign_mass(self, px, py, vals, out=None, warm_start="delta", rtol=1e-6, max_iter=200, x0=None,
                    info=True, net=None, rhs="exact", solver="cg"):
        """Mass assignment; rhs "exact" (Eq. proj) or "appb" (App. B quadrature);
        solver "cg" or "chebyshev" for the mesh system."""
        px, py, vals, x0 = self._f32(px), self._f32(py), self._f32(vals), self._f32(x0)
        F = vals.numel() // max(1, px.numel())
        out = out if out is not None else self._empty(F, self.nodes)
        if net is not None:
            warm_start = "net"
        o = self._opts(warm_start, rtol, max_iter, x0, net, rhs, solver)
        inf = (_Info * F)() if info else None
        self._stream()
        s = self.lib.pm_assign_mass(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F, _ptr(out),
                                    ctypes.byref(o), inf)
        self._check(s)
        if not info:
            return out
        return out, [_info(x)
                     for x in inf]

    def assign_mass_host(self, px, py, vals, out=None, warm_start="delta", rtol=1e-6, max_iter=200, info=True,
                         net=None, rhs="exact", solver="cg"):
        """Mass assignment from CPU tensors into a CPU tensor (pm_assign_mass_host):
        pinned tensors let the uploads overlap the kernels. Without info the
        result is valid after the context's stream completes (sync())."""
        def host(t):
            if t is None:
                return None
            if t.is_cuda or t.dtype != self.torch.float32 or not t.is_contiguous():
                raise TypeError("expected a contiguous float32 CPU tensor")
            return t
        px, py, vals = host(px), host(py), host(vals)
        F = vals.numel() // max(1, px.numel())
        out = out if out is not None else self.torch.empty(F, self.nodes, dtype=self.torch.float32).pin_memory()
        host(out)
        if net is not None:
            warm_start = "net"
        o = self._opts(warm_start, rtol, max_iter, None, net, rhs, solver)
        inf = (_Info * F)() if info else None
        self._stream()
        s = self.lib.pm_assign_mass_host(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F, _ptr(out),
                                         ctypes.byref(o), inf)
        self._check(s)
        if not info:
            return out
        return out, [_info(x) for x in inf]

    def net_features(self, px, py, vals):
        """(delta [F, n^2], features [F, 2, n^2], max|A_f| list) for the network."""
        px, py, vals = self._f32(px), self._f32(py), self._f32(vals)
        F = vals.numel() // max(1, px.numel())
        delta = self._empty(F, self.nodes)
        feat = self._empty(F, 2, self.nodes)
        scale = (ctypes.c_float * F)()
        self._stream()
        self._check(self.lib.pm_net_features(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F, _ptr(delta),
                                             _ptr(feat), scale))
        return delta, feat, list(scale)

    def mass_rhs(self, px, py, vals, out=None, rhs="exact"):
        """b_j = int A psi_j; rhs "exact" (Eq. proj) or "appb" (App. B quadrature)."""
        px, py, vals = self._f32(px), self._f32(py), self._f32(vals)
        F = vals.numel() // max(1, px.numel())
        out = out if out is not None else self._empty(F, self.nodes)
        self._stream()
        self._check(self.lib.pm_mass_rhs_mode(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(vals), F,
                                              RHS_MODES[rhs], _ptr(out)))
        return out

    def mass_apply(self, x, out=None):
        x = self._f32(x)
        F = x.numel() // self.nodes
        out = out if out is not None else self._empty(F, self.nodes)
        self._stream()
        self._check(self.lib.pm_mass_apply(self.h, _ptr(x), F, _ptr(out)))
        return out

    def mass_solve(self, b, out=None, rtol=1e-6, max_iter=200, x0=None, info=True, warm_start=None, solver="cg"):
        b, x0 = self._f32(b), self._f32(x0)
        F = b.numel() // self.nodes
        out = out if out is not None else self._empty(F, self.nodes)
        ws = warm_start or ("user" if x0 is not None else "zero")
        o = self._opts(ws, rtol, max_iter, x0, solver=solver)
        inf = (_Info * F)() if info else None
        self._stream()
        self._check(self.lib.pm_mass_solve(self.h, _ptr(b), F, _ptr(out), ctypes.byref(o), inf))
        if not info:
            return out
        return out, [_info(x)
                     for x in inf]

    def particle_volumes(self, px, py=None, out=None):
        px, py = self._f32(px), self._f32(py)
        out = out if out is not None else self._empty(px.numel())
        self._stream()
        self._check(self.lib.pm_particle_volumes(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(out)))
        return out

    def triangulate(self, px, py):
        px, py = self._f32(px), self._f32(py)
        cap = 2 * px.numel() + 64
        tri = self.torch.empty((cap, 3), dtype=self.torch.int32, device=self.device)
        off = self.torch.empty((cap, 4), dtype=self.torch.int32, device=self.device)
        nt = ctypes.c_longlong(0)
        self._stream()
        self._check(self.lib.pm_triangulate(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(tri), _ptr(off), cap,
                                            ctypes.byref(nt)))
        return tri[: nt.value], off[: nt.value]

    def sort(self, px, py=None):
        px, py = self._f32(px), self._f32(py)
        perm = self.torch.empty(px.numel(), dtype=self.torch.int32, device=self.device)
        cs = self.torch.empty(self.nodes + 1, dtype=self.torch.int32, device=self.device)
        self._stream()
        self._check(self.lib.pm_sort(self.h, _ptr(px), _ptr(py), px.numel(), _ptr(perm), _ptr(cs)))
        return perm, cs

    # ---------------------------------------------------------------- advection
    def advect_shift(self, px, py, dx, dy=0.0):
        px, py = self._f32(px), self._f32(py)
        self._stream()
        self._check(self.lib.pm_advect_shift(self.h, _ptr(px), _ptr(py), px.numel(), float(dx), float(dy)))

    def advect_rotate(self, px, py, cx, cy, angle):
        px, py = self._f32(px), self._f32(py)
        self._stream()
        self._check(self.lib.pm_advect_rotate(self.h, _ptr(px), _ptr(py), px.numel(), float(cx), float(cy),
                                              float(angle)))

    def advect_rk2(self, mesh_vel, vel, px, py, dt, vals=None, factor=1.0):
        mesh_vel, vel, px, py, vals = (self._f32(t) for t in (mesh_vel, vel, px, py, vals))
        F = vals.numel() // max(1, px.numel()) if vals is not None else 0
        self._stream()
        self._check(self.lib.pm_advect_rk2(self.h, _ptr(mesh_vel), _ptr(vel), _ptr(px), _ptr(py), px.numel(),
                                           float(dt), _ptr(vals), F, float(factor)))

    # ---------------------------------------------------------- instrumentation
    def profile(self, enable=True, count_work=False):
        """Per-phase CUDA-event timing; with count_work, the triangulation
        runs its counting build (same results, not for timing)."""
        self._check(self.lib.pm_profile(self.h, (2 if count_work else 1) if enable else 0))

    def work_read(self, reset=True):
        """Triangulation work counters collected in counting mode."""
        c = (ctypes.c_longlong * 8)()
        self._check(self.lib.pm_work_read(self.h, c, 8, 1 if reset else 0))
        return dict(zip(WORK_COUNTERS, list(c)[:len(WORK_COUNTERS)]))

    def profile_read(self, reset=True):
        ms = (ctypes.c_double * len(PHASES))()
        calls = (ctypes.c_longlong * len(PHASES))()
        self._check(self.lib.pm_profile_read(self.h, ms, calls, 1 if reset else 0))
        return {PHASES[k]: (ms[k], calls[k]) for k in range(len(PHASES))}


class Batch:
    """Many independent 2D instances advanced together in one packed
    workspace, one launch per phase (pm_batch_*). tune: 0 = choose the solve
    block size and packing order by timing the first step; 256, 512 or 1024 =
    that solve block size."""

    def __init__(self, sizes, Ls, max_particles, max_fields=1, tune=0, device=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_1610_05258_gb300 needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device if device is not None else "cuda")
        self.k = len(sizes)
        self.sizes = list(sizes)
        n = (ctypes.c_int * self.k)(*sizes)
        L = (ctypes.c_double * self.k)(*Ls)
        mp = (ctypes.c_longlong * self.k)(*max_particles)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = torch.cuda.current_stream().cuda_stream
            s = self.lib.pm_batch_create(ctypes.byref(h), self.k, n, L, mp, max_fields, tune, ctypes.c_void_p(st))
        if s != 0:
            raise PMError(s, "pm_batch_create failed")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and self.lib is not None:
            self.lib.pm_batch_destroy(self.h)
            self.h = None

    def tuning(self):
        """(solve threads per CTA, CTAs per instance, packed largest first, step
        ms measured when tuning)."""
        th, cl, lf, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        self.lib.pm_batch_tuning(self.h, ctypes.byref(th), ctypes.byref(cl), ctypes.byref(lf), ctypes.byref(ms))
        return th.value, cl.value, bool(lf.value), ms.value

    def set_tuning(self, threads, cluster=1, largest_first=False):
        s = self.lib.pm_batch_set_tuning(self.h, threads, cluster, int(largest_first))
        if s != 0:
            raise PMError(s, self.lib.pm_batch_last_error(self.h).decode())

    def set_start(self, warm_start="direct"):
        ws = {"direct": PM_WS_DIRECT, "delta": PM_WS_DELTA, "zero": PM_WS_ZERO, "user": PM_WS_USER,
              "net": PM_WS_NET}.get(warm_start, -1)  # the library rejects all but the first three
        s = self.lib.pm_batch_set_start(self.h, ws)
        if s != 0:
            raise PMError(s, self.lib.pm_batch_last_error(self.h).decode())

    def assign_mass(self, pxs, pys, vals, outs, rtol=1e-6, max_iter=200, info=True):
        K = self.k
        arr = lambda ts: (ctypes.c_void_p * K)(*[t.data_ptr() for t in ts])
        np_ = (ctypes.c_longlong * K)(*[t.numel() for t in pxs])
        F = vals[0].numel() // max(1, pxs[0].numel())
        inf = (_Info * (K * F))() if info else None
        s = self.lib.pm_batch_assign_mass(self.h, arr(pxs), arr(pys), np_, arr(vals), F, arr(outs), rtol, max_iter,
                                          inf)
        if s != 0:
            raise PMError(s, self.lib.pm_batch_last_error(self.h).decode())
        if not info:
            return None
        return [[_info(x)
                 for x in inf[k * F:(k + 1) * F]] for k in range(K)]


class Net:
    """The learned warm start's network (pm_net_*)."""

    def __init__(self, max_n, max_batch=1, device=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_1610_05258_gb300 needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device if device is not None else "cuda")
        self.num_params = self.lib.pm_net_num_params()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = torch.cuda.current_stream().cuda_stream
            s = self.lib.pm_net_create(ctypes.byref(h), max_n, max_batch, ctypes.c_void_p(st))
        if s != 0:
            raise PMError(s, "pm_net_create failed")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and self.lib is not None:
            self.lib.pm_net_destroy(self.h)
            self.h = None

    def _stream(self):
        self.lib.pm_net_set_stream(self.h, ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream))

    def load(self, theta, moments=None, step=0):
        import numpy as np
        P = self.num_params
        buf = np.zeros(3 * P, dtype=np.float32)
        buf[:P] = np.asarray(theta, dtype=np.float32)
        if moments is not None:
            buf[P:] = np.asarray(moments, dtype=np.float32)
        s = self.lib.pm_net_load(self.h, buf.ctypes.data_as(ctypes.c_void_p), 1 if moments is not None else 0, step)
        if s != 0:
            raise PMError(s, "pm_net_load failed")

    def state(self):
        import numpy as np
        P = self.num_params
        buf = np.zeros(3 * P, dtype=np.float32)
        step = ctypes.c_longlong(0)
        s = self.lib.pm_net_state(self.h, buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(step))
        if s != 0:
            raise PMError(s, "pm_net_state failed")
        return buf[:P].copy(), buf[P:].copy(), step.value

    def forward(self, x, out=None):
        B, _, n, _ = x.shape
        out = out if out is not None else self.torch.empty(B, n, n, device=self.device)
        self._stream()
        s = self.lib.pm_net_forward(self.h, _ptr(x), B, n, _ptr(out))
        if s != 0:
            raise PMError(s, "pm_net_forward failed")
        return out

    def train_step(self, x, target, lr, want_loss=True):
        B, _, n, _ = x.shape
        loss = ctypes.c_double(0.0)
        self._stream()
        s = self.lib.pm_net_train_step(self.h, _ptr(x), _ptr(target), B, n, ctypes.c_float(lr),
                                       ctypes.byref(loss) if want_loss else None)
        if s != 0:
            raise PMError(s, "pm_net_train_step failed")
        return loss.value if want_loss else None

    def grad(self):
        import numpy as np
        g = np.zeros(self.num_params, dtype=np.float32)
        s = self.lib.pm_net_grad(self.h, g.ctypes.data_as(ctypes.c_void_p))
        if s != 0:
            raise PMError(s, "pm_net_grad failed")
        return g
