// C ABI (include/pmt.h): context, workspace and the entry points. Each entry
// validates its arguments on the host, then queues the kernels of its path on
// the context's stream.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

static std::atomic<long long> g_launch_total{0};
void count_launches(int k) { g_launch_total += k; }

struct PendingEvent {
    cudaEvent_t a, b;
    int ph;
};

struct pm_ctx {
    Geo g;
    Work w;
    cudaStream_t st;
    std::string err;
    ll bytes;
    int dev;
    // profiling: CUDA events around every phase, on the context's stream
    bool prof = false;
    bool count_work = false;  // counting instantiation of the triangulation
    std::vector<PendingEvent> ev;
    size_t nev = 0;
    double acc_ms[PM_NPHASE] = {0};
    ll acc_calls[PM_NPHASE] = {0};
    ll sorted_np = -1;  // particles of the most recent sort (w.pos, w.perm); -1: none yet
    // host-buffer mass assignment: device copies of the inputs and output,
    // the stream that uploads the values and its events (made on first use)
    float *hx = nullptr, *hy = nullptr, *hv = nullptr, *hout = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_start = nullptr, ev_vals = nullptr;
};

namespace {

pm_status fail(pm_ctx *c, pm_status s, const char *msg) {
    if (c) c->err = msg;
    return s;
}

pm_status cuda_fail(pm_ctx *c, cudaError_t e, const char *where) {
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return PM_ECUDA;
}

template <class T>
bool alloc(pm_ctx *c, T **p, ll count) {
    size_t b = sizeof(T) * (size_t)(count > 0 ? count : 1);
    if (cudaMalloc((void **)p, b) != cudaSuccess) return false;
    c->bytes += (ll)b;
    return true;
}

pm_status map_status(pm_ctx *c, int s) {
    if (s & (ST_NONFINITE | ST_DUP | ST_SPARSE | ST_DEGREE | ST_RANGE)) {
        char buf[256];
        snprintf(buf, sizeof buf, "degenerate input (device status 0x%x:%s%s%s%s%s)", s,
                 s & ST_NONFINITE ? " non-finite value" : "", s & ST_DUP ? " coincident particles" : "",
                 s & ST_SPARSE ? " triangulation not certified within the searched cells" : "",
                 s & ST_DEGREE ? " Delaunay degree above capacity" : "", s & ST_RANGE ? " internal range" : "");
        c->err = buf;
        return PM_EDEGENERATE;
    }
    if (s & ST_TIMEOUT) return fail(c, PM_ETIMEOUT, "a device-side wait timed out");
    if (s & ST_NOTCONV) return fail(c, PM_ENOTCONV, "mass solve did not reach the requested residual");
    return PM_OK;
}

// Wait for the stream, fetch and clear the device status word.
pm_status wait_status(pm_ctx *c) {
    cudaError_t e = cudaMemcpyAsync(c->w.hstatus, c->w.status, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    int s = *c->w.hstatus;
    if (s) cudaMemsetAsync(c->w.status, 0, sizeof(int), c->st);
    return map_status(c, s);
}

void resolve_events(pm_ctx *c) {
    if (!c->nev) return;
    cudaStreamSynchronize(c->st);
    for (size_t k = 0; k < c->nev; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->ev[k].a, c->ev[k].b) == cudaSuccess) {
            c->acc_ms[c->ev[k].ph] += ms;
            c->acc_calls[c->ev[k].ph] += 1;
        }
    }
    c->nev = 0;
}

// RAII phase marker: records a CUDA event pair around the phase's kernels.
struct Phase {
    pm_ctx *c;
    size_t k;
    Phase(pm_ctx *c_, int ph) : c(c_), k((size_t)-1) {
        if (!c->prof) return;
        if (c->nev == 256) resolve_events(c);
        if (c->nev == c->ev.size()) {
            PendingEvent e;
            cudaEventCreate(&e.a);
            cudaEventCreate(&e.b);
            c->ev.push_back(e);
        }
        k = c->nev++;
        c->ev[k].ph = ph;
        cudaEventRecord(c->ev[k].a, c->st);
    }
    ~Phase() {
        if (k != (size_t)-1) cudaEventRecord(c->ev[k].b, c->st);
    }
};

// PM_DEBUG_SYNC=1 in the environment: wait for the stream after every phase
// so that an execution error is reported with the phase that caused it.
bool debug_sync() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("PM_DEBUG_SYNC");
        v = e && e[0] == '1';
    }
    return v == 1;
}

pm_status check_launch(pm_ctx *c, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && debug_sync()) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(c->st, &cs);
        if (cs == cudaStreamCaptureStatusNone) e = cudaStreamSynchronize(c->st);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return PM_OK;
}

pm_status check_particles(pm_ctx *c, const float *px, const float *py, ll np, int F, const float *vals,
                          ll min_np) {
    if (!c) return PM_EINVAL;
    if (np < min_np || np > c->w.np_max) return fail(c, PM_EINVAL, "particle count out of range");
    if (np > 0 && (!px || (c->g.dim == 2 && !py))) return fail(c, PM_EINVAL, "null position array");
    if (F < 0 || F > c->w.F_max) return fail(c, PM_EINVAL, "field count out of range");
    if (F > 0 && np > 0 && !vals) return fail(c, PM_EINVAL, "null particle field array");
    return PM_OK;
}

// Sort + particle functions: everything the assignments share.
pm_status prepare(pm_ctx *c, const float *px, const float *py, ll np, const float *vals, int F, bool need_tri) {
    {
        Phase ph(c, PM_PH_SORT);
        launch_sort(c->g, c->w, px, py, np, vals, F, c->st);
    }
    if (pm_status s = check_launch(c, "sort")) return s;
    c->sorted_np = np;
    if (need_tri) {
        Phase ph(c, PM_PH_TRIANGULATE);
        if (c->g.dim == 2)
            launch_triangulate(c->g, c->w, np, c->st, c->count_work);
        else
            launch_volumes_1d(c->g, c->w, np, c->st);
    }
    return check_launch(c, "particle functions");
}

}  // namespace

extern "C" {

pm_status pm_ctx_create(pm_ctx **out, int dim, int n, double L, long long max_particles, int max_fields,
                        void *stream) {
    return pm_ctx_create_mesh(out, dim, n, L, max_particles, max_fields, PM_MESH_Q1, stream);
}

pm_status pm_ctx_create_mesh(pm_ctx **out, int dim, int n, double L, long long max_particles, int max_fields,
                             int mesh_kind, void *stream) {
    if (!out) return PM_EINVAL;
    *out = nullptr;
    if ((dim != 1 && dim != 2) || n < 4 || !(L > 0.0) || max_particles < 0 || max_fields < 1 ||
        max_fields > PM_MAXF || (mesh_kind != PM_MESH_Q1 && mesh_kind != PM_MESH_P1))
        return PM_EINVAL;
    if (max_particles >= (1LL << 28) - 16) return PM_EINVAL;  // star entries: 28-bit index, top 16 reserved
    if (dim == 2 && (ll)n * n > (1LL << 30)) return PM_EINVAL;
    pm_ctx *c = new pm_ctx();
    c->bytes = 0;
    c->st = (cudaStream_t)stream;
    cudaGetDevice(&c->dev);
    Geo &g = c->g;
    g.dim = dim;
    g.n = n;
    g.L = L;
    g.invL = (float)(1.0 / L);
    g.h = (float)(L / n);
    g.ncell = dim == 1 ? n : (ll)n * n;
    g.p1 = dim == 2 && mesh_kind == PM_MESH_P1 ? 1 : 0;
    Work &w = c->w;
    memset(&w, 0, sizeof(w));
    w.np_max = max_particles;
    w.F_max = max_fields;
    const ll np = max_particles, nc = g.ncell, F = max_fields;
    w.nblk_psum = 4 * 152;  // enough loads in flight to stream the particle arrays
    bool ok = alloc(c, &w.fx, np) && alloc(c, &w.key, np) && alloc(c, &w.slot, np) && alloc(c, &w.count, nc) &&
              alloc(c, &w.cell_start, nc + 1) && alloc(c, &w.scan_tmp, nc / 4096 + 2) && alloc(c, &w.tmp, np) &&
              alloc(c, &w.perm, np) && alloc(c, &w.pos, np) && alloc(c, &w.vals, np * F) &&
              alloc(c, &w.maxabs, PM_MAXF) && alloc(c, &w.deg, np) && alloc(c, &w.vol, np) &&
              alloc(c, &w.part, (dim == 2 ? 4 : 2) * (F + 1) * nc) && alloc(c, &w.bfix, F * nc) &&
              alloc(c, &w.psum, 2 * PM_MAXF * (ll)w.nblk_psum) &&
              alloc(c, &w.epart, 2 * PM_MAXF * (ll)energy_blocks()) && alloc(c, &w.r, F * nc) &&
              alloc(c, &w.p, F * nc) && alloc(c, &w.q, F * nc) && alloc(c, &w.b, F * nc) &&
              alloc(c, &w.red, 6LL * PM_MAXF * 4096) && alloc(c, &w.scal, 16LL * PM_MAXF) &&
              alloc(c, &w.bar, 2) && alloc(c, &w.status, 1) && alloc(c, &w.empty, 1) && alloc(c, &w.ntri, 1) &&
              alloc(c, &w.wsum, 8) && alloc(c, &w.nretry, 1) && alloc(c, &w.meshmax, PM_MAXF) &&
              alloc(c, &w.pc, F * np) && alloc(c, &w.px, pcg_width((int)F) * np) &&
              alloc(c, &w.pq, pcg_width((int)F) * np) && alloc(c, &w.prp, 2LL * pcg_width((int)F) * np) &&
              alloc(c, &w.pp2, pcg_width((int)F) * np);
    w.cfix = (ll *)w.prp;
    w.red_blocks = 4096;
    if (ok && dim == 2)
        ok = alloc(c, &w.nbr, (ll)PM_MAXDEG * np) && alloc(c, &w.pcoef, (ll)PM_MAXDEG * np) && alloc(c, &w.r2, F * nc);
    if (ok && F > 1) ok = alloc(c, &w.mesh_il, (ll)g2p_width((int)F) * nc);
    if (ok && dim == 2 && n % 128 == 0 && !g.p1)  // the network start: bilinear meshes
        ok = alloc(c, &w.feat, 2 * F * nc) && alloc(c, &w.corr, F * nc);
    if (ok && cudaMallocHost((void **)&w.hstatus, sizeof(int)) != cudaSuccess) ok = false;
    if (ok && cudaMallocHost((void **)&w.hres, sizeof(double) * PM_MAXF) != cudaSuccess) ok = false;
    if (!ok) {
        pm_ctx_destroy(c);
        cudaGetLastError();
        return PM_ENOMEM;
    }
    rhs_prepare_device();
    cudaMemset(w.status, 0, sizeof(int));
    cudaMemset(w.scal, 0, sizeof(double) * 16 * PM_MAXF);
    cudaMemset(w.wsum, 0, sizeof(ull) * 8);
    cudaMemset(w.deg, 0, (size_t)(np > 0 ? np : 1));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        pm_ctx_destroy(c);
        return PM_ECUDA;
    }
    *out = c;
    return PM_OK;
}

void pm_ctx_destroy(pm_ctx *c) {
    if (!c) return;
    Work &w = c->w;
    void *ptrs[] = {w.fx,  w.key, w.slot, w.count, w.cell_start, w.scan_tmp, w.tmp,  w.perm,  w.pos,
                    w.vals, w.maxabs, w.nbr, w.deg,  w.vol,  w.part,  w.bfix, w.psum, w.epart, w.r, w.p,
                    w.q,   w.b,   w.red,  w.scal,  w.bar,  w.status, w.empty, w.ntri, w.feat, w.corr,
                    w.wsum, w.nretry, w.meshmax, w.pc, w.px, w.pq, w.prp, w.pp2, w.pcoef, w.mesh_il, w.r2};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w.hstatus) cudaFreeHost(w.hstatus);
    if (w.hres) cudaFreeHost(w.hres);
    for (float *p : {c->hx, c->hy, c->hv, c->hout})
        if (p) cudaFree(p);
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    if (c->ev_vals) cudaEventDestroy(c->ev_vals);
    if (c->side) cudaStreamDestroy(c->side);
    for (auto &e : c->ev) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    delete c;
}

pm_status pm_ctx_set_stream(pm_ctx *c, void *stream) {
    if (!c) return PM_EINVAL;
    c->st = (cudaStream_t)stream;
    return PM_OK;
}

pm_status pm_sync(pm_ctx *c) {
    if (!c) return PM_EINVAL;
    return wait_status(c);
}

const char *pm_last_error(const pm_ctx *c) { return c ? c->err.c_str() : "null context"; }

long long pm_ctx_workspace_bytes(const pm_ctx *c) { return c ? c->bytes : 0; }

pm_status pm_interpolate(pm_ctx *c, const float *mesh, int F, const float *px, const float *py, long long np,
                         float *out) {
    pm_status s = check_particles(c, px, py, np, 0, nullptr, 0);
    if (s) return s;
    if (F < 1 || F > c->w.F_max) return fail(c, PM_EINVAL, "field count out of range");
    if (np > 0 && (!mesh || !out)) return fail(c, PM_EINVAL, "null mesh or output array");
    {
        Phase ph(c, PM_PH_G2P);
        launch_g2p(c->g, mesh, F, px, py, np, out, c->w.mesh_il, c->w.status, c->st);
    }
    return check_launch(c, "pm_interpolate");
}

pm_status pm_interpolate_sorted(pm_ctx *c, const float *mesh, int F, long long np, float *out) {
    if (!c) return PM_EINVAL;
    if (c->sorted_np < 0) return fail(c, PM_EINVAL, "no particles sorted yet");
    if (np != c->sorted_np) return fail(c, PM_EINVAL, "np differs from the particles of the last sort");
    if (F < 1 || F > c->w.F_max) return fail(c, PM_EINVAL, "field count out of range");
    if (np > 0 && (!mesh || !out)) return fail(c, PM_EINVAL, "null mesh or output array");
    {
        Phase ph(c, PM_PH_G2P);
        launch_g2p_sorted(c->g, mesh, F, c->w.pos, np, out, c->w.mesh_il, c->st);
    }
    return check_launch(c, "pm_interpolate_sorted");
}

pm_status pm_assign_delta(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                          float *mesh_out) {
    pm_status s = check_particles(c, px, py, np, F, vals, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (F < 1 || !mesh_out) return fail(c, PM_EINVAL, "null output or no field");
    if ((s = prepare(c, px, py, np, vals, F, c->g.dim == 2))) return s;
    {
        Phase ph(c, PM_PH_DELTA);
        launch_delta(c->g, c->w, np, F, mesh_out, c->st);
    }
    return check_launch(c, "pm_assign_delta");
}

pm_status pm_assign_flip(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                         float *mesh_out, float *node_volume_out, long long *empty_nodes) {
    pm_status s = check_particles(c, px, py, np, F, vals, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (F < 1 || !mesh_out) return fail(c, PM_EINVAL, "null output or no field");
    if ((s = prepare(c, px, py, np, vals, F, true))) return s;
    {
        Phase ph(c, PM_PH_FLIP);
        launch_flip(c->g, c->w, np, F, mesh_out, node_volume_out, c->st);
    }
    if ((s = check_launch(c, "pm_assign_flip"))) return s;
    if (empty_nodes) {
        int e = 0;
        cudaMemcpyAsync(c->w.hstatus, c->w.empty, sizeof(int), cudaMemcpyDeviceToHost, c->st);
        cudaError_t ce = cudaStreamSynchronize(c->st);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "pm_assign_flip");
        e = *c->w.hstatus;
        *empty_nodes = e;
        return wait_status(c);
    }
    return PM_OK;
}

pm_status pm_assign_pic(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                        float *mesh_out) {
    pm_status s = check_particles(c, px, py, np, F, vals, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (F < 1 || !mesh_out) return fail(c, PM_EINVAL, "null output or no field");
    if ((s = prepare(c, px, py, np, vals, F, true))) return s;
    {
        Phase ph(c, PM_PH_FLIP);
        const double h = c->g.L / c->g.n;
        launch_flip(c->g, c->w, np, F, mesh_out, nullptr, c->st, (float)(c->g.dim == 2 ? h * h : h));
    }
    return check_launch(c, "pm_assign_pic");
}

static void default_opts(const pm_solve_opts *o, pm_solve_opts &d) {
    d.warm_start = PM_WS_DELTA;
    d.rtol = 1e-6;
    d.max_iter = 200;
    d.x0 = nullptr;
    d.net = nullptr;
    d.rhs_mode = PM_RHS_EXACT;
    d.solver = PM_SOLVER_CG;
    if (o) d = *o;
    if (!(d.rtol > 0.0)) d.rtol = 1e-6;
    if (d.max_iter <= 0) d.max_iter = 200;
}

static pm_status fill_info(pm_ctx *c, int F, pm_solve_info *info) {
    pm_status s = wait_status(c);
    double sc[16 * PM_MAXF];
    cudaError_t e = cudaMemcpy(sc, c->w.scal, sizeof(double) * 16 * F, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "info");
    for (int f = 0; f < F; ++f) {
        const double *v = sc + 16 * f;
        info[f].iters = (int)v[0];
        info[f].init_rel_resid = v[1];
        info[f].rel_resid = v[2];
        info[f].sum_mesh = v[3];
        info[f].sum_particles = v[4];
        double den = v[5] > 0.0 ? v[5] : fabs(v[4]);
        info[f].cons_err = den > 0.0 ? fabs(v[3] - v[4]) / den : fabs(v[3] - v[4]);
        info[f].energy_mesh = v[6];
        info[f].energy_particles = v[7];
    }
    return s;
}

// The report of a solve: stability diagnostics of the mesh fields and, if
// given, of the sorted particle values (see launch_energies), then the
// solver's scalars.
static pm_status report(pm_ctx *c, int F, pm_solve_info *info, const float *mesh, ll np, const float *pvals, ll fs,
                        ll ss) {
    {
        Phase ph(c, PM_PH_OTHER);
        launch_energies(c->g, c->w, F, mesh, np, pvals, fs, ss, c->st);
    }
    if (pm_status s = check_launch(c, "diagnostics")) return s;
    return fill_info(c, F, info);
}

// Everything of a mass assignment before the solve: sort, particle
// functions, particle sums, right-hand side and the warm start.
// vals_ready (may be NULL): the values are still arriving, and become
// readable on the context's stream once that event completes. The sort and
// the particle functions run without them, and their gather waits for it.
static pm_status mass_front(pm_ctx *c, const float *px, const float *py, ll np, const float *vals, int F,
                            float *mesh_out, const pm_solve_opts &o, bool &start, cudaEvent_t vals_ready = nullptr) {
    pm_status s;
    if (vals_ready) {
        if ((s = prepare(c, px, py, np, nullptr, 0, true))) return s;
        Phase ph(c, PM_PH_SORT);
        cudaStreamWaitEvent(c->st, vals_ready, 0);
        launch_gather_vals(c->w, np, vals, F, c->st);
        if ((s = check_launch(c, "value gather"))) return s;
    } else if ((s = prepare(c, px, py, np, vals, F, true))) {
        return s;
    }
    {
        Phase ph(c, PM_PH_RHS);
        launch_psum(c->g, c->w, np, F, c->st);
        if ((s = check_launch(c, "particle sums"))) return s;
        if (o.rhs_mode == PM_RHS_APPB)
            launch_rhs_appb(c->g, c->w, np, F, c->st);
        else
            launch_rhs(c->g, c->w, np, F, c->st);
        if ((s = check_launch(c, "right-hand side"))) return s;
    }
    start = true;
    if (o.warm_start == PM_WS_DELTA) {
        Phase ph(c, PM_PH_DELTA);
        launch_delta(c->g, c->w, np, F, mesh_out, c->st);
    } else if (o.warm_start == PM_WS_NET) {
        {
            Phase ph(c, PM_PH_DELTA);
            launch_delta(c->g, c->w, np, F, mesh_out, c->st);
            launch_features(c->g, c->w, F, mesh_out, c->st);
        }
        {
            Phase ph(c, PM_PH_NET);
            // Gate: the network runs only on the fields whose delta start is
            // still above PM_NET_GATE in relative residual (the others need a
            // CG iteration or two, far less than the network costs). The
            // residuals come back to the host, so this start waits once.
            double *dres = c->w.red + 4LL * PM_MAXF * 608;  // past the residual kernel's partials
            launch_start_resid(c->g, c->w, F, dres, c->st);
            cudaMemcpyAsync(c->w.hres, dres, sizeof(double) * F, cudaMemcpyDeviceToHost, c->st);
            cudaError_t ce = cudaStreamSynchronize(c->st);
            if (ce != cudaSuccess) return cuda_fail(c, ce, "network gate");
            pm_net_set_stream(o.net, c->st);
            int f = 0;
            while (f < F) {
                const bool on = c->w.hres[f] > PM_NET_GATE;
                int e = f + 1;
                while (e < F && (c->w.hres[e] > PM_NET_GATE) == on) ++e;
                float *corr = c->w.corr + (ll)f * c->g.ncell;
                if (on) {
                    pm_status s2 = pm_net_forward(o.net, c->w.feat + 2LL * f * c->g.ncell, e - f, c->g.n, corr);
                    if (s2)
                        return fail(c, s2, "network forward failed (n must be a multiple of 128 within the net's size)");
                } else {
                    // no correction: alpha = 0 for these fields
                    cudaMemsetAsync(corr, 0, sizeof(float) * (e - f) * c->g.ncell, c->st);
                }
                f = e;
            }
            launch_apply_correction(c->g, c->w, F, mesh_out, c->st);
        }
    } else if (o.warm_start == PM_WS_DIRECT) {
        // exact inverse of the uniform periodic mass matrix applied to b
        Phase ph(c, PM_PH_SOLVE);
        launch_rhs_to_float(c->g, c->w, F, c->w.b, c->st);
        launch_mass_direct(c->g, c->w.b, F, mesh_out, c->w.r, c->st);
    } else if (o.warm_start == PM_WS_USER) {
        cudaMemcpyAsync(mesh_out, o.x0, sizeof(float) * F * c->g.ncell, cudaMemcpyDeviceToDevice, c->st);
    } else {
        start = false;
    }
    return check_launch(c, "warm start");
}

static pm_status mass_solve_launch(pm_ctx *c, int F, float *mesh_out, bool start, const pm_solve_opts &o) {
    int e;
    {
        Phase ph(c, PM_PH_SOLVE);
        e = (o.solver == PM_SOLVER_CHEBYSHEV ? launch_cheb : launch_cg)(c->g, c->w, F, nullptr, true, mesh_out,
                                                                       start, o.rtol, o.max_iter, c->st);
    }
    if (e) return cuda_fail(c, (cudaError_t)e, "pm_assign_mass solve launch");
    return check_launch(c, "solve");
}

static pm_status mass_args(pm_ctx *c, const float *px, const float *py, ll np, const float *vals, int F,
                           float *mesh_out, const pm_solve_opts *opts, pm_solve_opts &o) {
    pm_status s = check_particles(c, px, py, np, F, vals, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (F < 1 || !mesh_out) return fail(c, PM_EINVAL, "null output or no field");
    default_opts(opts, o);
    if (o.warm_start < PM_WS_DELTA || o.warm_start > PM_WS_DIRECT) return fail(c, PM_EINVAL, "unknown warm start");
    if (o.rhs_mode != PM_RHS_EXACT && o.rhs_mode != PM_RHS_APPB) return fail(c, PM_EINVAL, "unknown rhs_mode");
    if (o.solver != PM_SOLVER_CG && o.solver != PM_SOLVER_CHEBYSHEV) return fail(c, PM_EINVAL, "unknown solver");
    if (c->g.p1 && (o.rhs_mode == PM_RHS_APPB || o.warm_start == PM_WS_DIRECT))
        return fail(c, PM_EINVAL, "PM_RHS_APPB and PM_WS_DIRECT need the bilinear mesh");
    if (o.warm_start == PM_WS_USER && !o.x0) return fail(c, PM_EINVAL, "PM_WS_USER without x0");
    if (o.warm_start == PM_WS_NET && (!o.net || !c->w.feat)) return fail(c, PM_EINVAL, "PM_WS_NET needs a network and a 2D bilinear mesh with n % 128 == 0");
    return PM_OK;
}

pm_status pm_assign_mass(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                         float *mesh_out, const pm_solve_opts *opts, pm_solve_info *info) {
    pm_solve_opts o;
    pm_status s = mass_args(c, px, py, np, vals, F, mesh_out, opts, o);
    if (s) return s;
    bool start = true;
    if ((s = mass_front(c, px, py, np, vals, F, mesh_out, o, start))) return s;
    if ((s = mass_solve_launch(c, F, mesh_out, start, o))) return s;
    if (info) return report(c, F, info, mesh_out, np, c->w.vals, np, 1);
    return PM_OK;
}

// Device copies for the host-buffer call: inputs at the context's maximum
// sizes, one mesh-sized output, the upload stream and its events.
static pm_status host_staging(pm_ctx *c) {
    if (c->hx) return PM_OK;
    Work &w = c->w;
    const ll np = w.np_max, F = w.F_max;
    bool ok = alloc(c, &c->hx, np) && (c->g.dim == 1 || alloc(c, &c->hy, np)) && alloc(c, &c->hv, F * np) &&
              alloc(c, &c->hout, F * c->g.ncell);
    ok = ok && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_vals, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(c, PM_ENOMEM, "host-buffer staging: allocation failed");
    }
    return PM_OK;
}

pm_status pm_assign_mass_host(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                              float *mesh_out, const pm_solve_opts *opts, pm_solve_info *info) {
    pm_solve_opts o;
    pm_status s = mass_args(c, px, py, np, vals, F, mesh_out, opts, o);
    if (s) return s;
    if (o.warm_start == PM_WS_USER) return fail(c, PM_EINVAL, "PM_WS_USER takes a device x0: use pm_assign_mass");
    if ((s = host_staging(c))) return s;
    const size_t pb = sizeof(float) * (size_t)np;
    // Positions first, on the context's stream. The values follow on the side
    // stream once the positions are up (copies share the copy engine, so
    // queued first they would hold the positions back) and everything queued
    // before on the context's stream is done (an earlier call may still be
    // reading them); the sort and the particle functions run meanwhile.
    cudaMemcpyAsync(c->hx, px, pb, cudaMemcpyHostToDevice, c->st);
    if (c->g.dim == 2) cudaMemcpyAsync(c->hy, py, pb, cudaMemcpyHostToDevice, c->st);
    cudaEventRecord(c->ev_start, c->st);
    cudaStreamWaitEvent(c->side, c->ev_start, 0);
    cudaMemcpyAsync(c->hv, vals, pb * F, cudaMemcpyHostToDevice, c->side);
    cudaEventRecord(c->ev_vals, c->side);
    if ((s = check_launch(c, "host-buffer uploads"))) return s;
    bool start = true;
    if ((s = mass_front(c, c->hx, c->g.dim == 2 ? c->hy : nullptr, np, c->hv, F, c->hout, o, start, c->ev_vals)))
        return s;
    if ((s = mass_solve_launch(c, F, c->hout, start, o))) return s;
    cudaMemcpyAsync(mesh_out, c->hout, sizeof(float) * F * (size_t)c->g.ncell, cudaMemcpyDeviceToHost, c->st);
    if ((s = check_launch(c, "host-buffer download"))) return s;
    if (info) return report(c, F, info, c->hout, np, c->w.vals, np, 1);
    return PM_OK;
}

// ---------------------------------------------------------------------------
// Mesh -> particle projections other than delta, and the lumped assignment
// (Table 1): c_mu = int Ab psi_mu, then c/v (lumped) or M_p^-1 c (full mass).
// ---------------------------------------------------------------------------
static pm_status proj_front(pm_ctx *c, const float *mesh, int F, const float *px, const float *py, ll np,
                            float *out) {
    pm_status s = check_particles(c, px, py, np, 0, nullptr, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (F < 1 || F > c->w.F_max) return fail(c, PM_EINVAL, "field count out of range");
    if (!mesh || !out) return fail(c, PM_EINVAL, "null mesh or output array");
    if ((s = prepare(c, px, py, np, nullptr, 0, true))) return s;
    {
        Phase ph(c, PM_PH_RHS);
        launch_g2p_integral(c->g, c->w, np, F, mesh, c->w.pc, c->st);
    }
    return check_launch(c, "mesh-to-particle integral");
}

static void unsort_fields(pm_ctx *c, ll np, int F, const float *src, float *out) {
    for (int f = 0; f < F; ++f) launch_scatter_sorted(np, c->w.perm, src + (ll)f * np, out + (ll)f * np, c->st);
}

pm_status pm_interpolate_lumped(pm_ctx *c, const float *mesh, int F, const float *px, const float *py, long long np,
                                float *out) {
    pm_status s = proj_front(c, mesh, F, px, py, np, out);
    if (s) return s;
    {
        Phase ph(c, PM_PH_G2P);
        launch_div_vol(np, F, c->w.vol, c->w.pc, c->st);
        unsort_fields(c, np, F, c->w.pc, out);
    }
    return check_launch(c, "pm_interpolate_lumped");
}

pm_status pm_interpolate_mass(pm_ctx *c, const float *mesh, int F, const float *px, const float *py, long long np,
                              float *out, const pm_solve_opts *opts, pm_solve_info *info) {
    pm_solve_opts o = opts ? *opts : pm_solve_opts{PM_WS_DELTA, 1e-6, 200, nullptr, nullptr, PM_RHS_EXACT, PM_SOLVER_CG};
    if (!(o.rtol > 0.0) || o.max_iter < 0) return fail(c, PM_EINVAL, "bad solve options");
    pm_status s = proj_front(c, mesh, F, px, py, np, out);
    if (s) return s;
    int e;
    {
        Phase ph(c, PM_PH_SOLVE);
        e = launch_pcg(c->g, c->w, np, F, c->w.pc, out, o.rtol, o.max_iter, c->st);
    }
    if (e) return cuda_fail(c, (cudaError_t)e, "pm_interpolate_mass solve launch");
    if ((s = check_launch(c, "pm_interpolate_mass"))) return s;
    if (info) return report(c, F, info, mesh, np, c->w.pq, 1, pcg_width(F));
    return PM_OK;
}

pm_status pm_assign_lumped(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                           float *mesh_out) {
    pm_status s = check_particles(c, px, py, np, F, vals, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (F < 1 || !mesh_out) return fail(c, PM_EINVAL, "null output or no field");
    if ((s = prepare(c, px, py, np, vals, F, true))) return s;
    {
        Phase ph(c, PM_PH_RHS);
        launch_rhs(c->g, c->w, np, F, c->st);
        launch_rhs_to_float(c->g, c->w, F, mesh_out, c->st);
        const double hd = c->g.dim == 2 ? (double)c->g.h * c->g.h : (double)c->g.h;
        launch_scale((ll)F * c->g.ncell, (float)(1.0 / hd), mesh_out, c->st);
    }
    return check_launch(c, "pm_assign_lumped");
}

pm_status pm_mass_rhs_mode(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                           int rhs_mode, float *b_out) {
    pm_status s = check_particles(c, px, py, np, F, vals, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (F < 1 || !b_out) return fail(c, PM_EINVAL, "null output or no field");
    if (rhs_mode != PM_RHS_EXACT && rhs_mode != PM_RHS_APPB) return fail(c, PM_EINVAL, "unknown rhs_mode");
    if (c->g.p1 && rhs_mode == PM_RHS_APPB) return fail(c, PM_EINVAL, "PM_RHS_APPB needs the bilinear mesh");
    if ((s = prepare(c, px, py, np, vals, F, true))) return s;
    {
        Phase ph(c, PM_PH_RHS);
        if (rhs_mode == PM_RHS_APPB)
            launch_rhs_appb(c->g, c->w, np, F, c->st);
        else
            launch_rhs(c->g, c->w, np, F, c->st);
        launch_rhs_to_float(c->g, c->w, F, b_out, c->st);
    }
    return check_launch(c, "pm_mass_rhs");
}

pm_status pm_mass_rhs(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                      float *b_out) {
    return pm_mass_rhs_mode(c, px, py, np, vals, F, PM_RHS_EXACT, b_out);
}

pm_status pm_mass_apply(pm_ctx *c, const float *x, int F, float *y) {
    if (!c) return PM_EINVAL;
    if (F < 1 || F > c->w.F_max || !x || !y) return fail(c, PM_EINVAL, "bad mass_apply arguments");
    launch_mass_apply(c->g, x, F, y, c->st);
    return check_launch(c, "pm_mass_apply");
}

pm_status pm_mass_solve(pm_ctx *c, const float *b, int F, float *x, const pm_solve_opts *opts,
                        pm_solve_info *info) {
    if (!c) return PM_EINVAL;
    if (F < 1 || F > c->w.F_max || !b || !x) return fail(c, PM_EINVAL, "bad mass_solve arguments");
    pm_solve_opts o;
    default_opts(opts, o);
    if (o.solver != PM_SOLVER_CG && o.solver != PM_SOLVER_CHEBYSHEV) return fail(c, PM_EINVAL, "unknown solver");
    bool start = false;
    if (o.warm_start == PM_WS_USER) {
        if (!o.x0) return fail(c, PM_EINVAL, "PM_WS_USER without x0");
        if (o.x0 != x) cudaMemcpyAsync(x, o.x0, sizeof(float) * F * c->g.ncell, cudaMemcpyDeviceToDevice, c->st);
        start = true;
    } else if (o.warm_start == PM_WS_DIRECT) {
        if (b == x) return fail(c, PM_EINVAL, "PM_WS_DIRECT needs distinct b and x");
        if (c->g.p1) return fail(c, PM_EINVAL, "PM_WS_DIRECT needs the bilinear mesh");
        launch_mass_direct(c->g, b, F, x, c->w.r, c->st);
        start = true;
    }
    int e;
    {
        Phase ph(c, PM_PH_SOLVE);
        e = (o.solver == PM_SOLVER_CHEBYSHEV ? launch_cheb : launch_cg)(c->g, c->w, F, b, false, x, start, o.rtol,
                                                                       o.max_iter, c->st);
    }
    if (e) return cuda_fail(c, (cudaError_t)e, "pm_mass_solve launch");
    if (info) return report(c, F, info, x, 0, nullptr, 0, 0);
    return PM_OK;
}

pm_status pm_particle_volumes(pm_ctx *c, const float *px, const float *py, long long np, float *v_out) {
    pm_status s = check_particles(c, px, py, np, 0, nullptr, c && c->g.dim == 2 ? 3 : 2);
    if (s) return s;
    if (!v_out) return fail(c, PM_EINVAL, "null output");
    if ((s = prepare(c, px, py, np, nullptr, 0, true))) return s;
    launch_scatter_sorted(np, c->w.perm, c->w.vol, v_out, c->st);
    return check_launch(c, "pm_particle_volumes");
}

pm_status pm_triangulate(pm_ctx *c, const float *px, const float *py, long long np, int *tri_out, int *off_out,
                         long long max_tri, long long *ntri) {
    pm_status s = check_particles(c, px, py, np, 0, nullptr, 3);
    if (s) return s;
    if (c->g.dim != 2) return fail(c, PM_EINVAL, "pm_triangulate needs dim == 2");
    if (!tri_out || !off_out || !ntri || max_tri < 0) return fail(c, PM_EINVAL, "bad output arguments");
    if ((s = prepare(c, px, py, np, nullptr, 0, true))) return s;
    launch_export_tris(c->g, c->w, np, tri_out, off_out, max_tri, c->st);
    if ((s = check_launch(c, "pm_triangulate"))) return s;
    ll cnt = 0;
    cudaMemcpyAsync(&cnt, c->w.ntri, sizeof(ll), cudaMemcpyDeviceToHost, c->st);
    s = wait_status(c);
    *ntri = cnt;
    if (!s && cnt > max_tri) return fail(c, PM_EINVAL, "max_tri too small");
    return s;
}

pm_status pm_net_features(pm_ctx *c, const float *px, const float *py, long long np, const float *vals, int F,
                          float *delta_out, float *feat_out, float *scale_out) {
    pm_status s = check_particles(c, px, py, np, F, vals, 3);
    if (s) return s;
    if (!c->w.feat || F < 1 || !delta_out || !feat_out) return fail(c, PM_EINVAL, "bad pm_net_features arguments");
    if ((s = prepare(c, px, py, np, vals, F, true))) return s;
    {
        Phase ph(c, PM_PH_RHS);
        launch_rhs(c->g, c->w, np, F, c->st);
    }
    {
        Phase ph(c, PM_PH_DELTA);
        launch_delta(c->g, c->w, np, F, delta_out, c->st);
        launch_features(c->g, c->w, F, delta_out, c->st);
    }
    cudaMemcpyAsync(feat_out, c->w.feat, sizeof(float) * 2 * F * c->g.ncell, cudaMemcpyDeviceToDevice, c->st);
    if (scale_out) {
        // max|A_f| as float
        cudaStreamSynchronize(c->st);
        unsigned m[PM_MAXF];
        cudaMemcpy(m, c->w.maxabs, sizeof(unsigned) * F, cudaMemcpyDeviceToHost);
        for (int f = 0; f < F; ++f) memcpy(&scale_out[f], &m[f], sizeof(float));
    }
    return check_launch(c, "pm_net_features");
}

pm_status pm_advect_shift(pm_ctx *c, float *px, float *py, long long np, double dx, double dy) {
    pm_status s = check_particles(c, px, py, np, 0, nullptr, 0);
    if (s) return s;
    {
        Phase ph(c, PM_PH_ADVECT);
        launch_advect_shift(c->g, px, py, np, dx, dy, c->st);
    }
    return check_launch(c, "pm_advect_shift");
}

pm_status pm_advect_rotate(pm_ctx *c, float *px, float *py, long long np, double cx, double cy, double angle) {
    pm_status s = check_particles(c, px, py, np, 0, nullptr, 0);
    if (s) return s;
    if (c->g.dim != 2) return fail(c, PM_EINVAL, "pm_advect_rotate needs dim == 2");
    {
        Phase ph(c, PM_PH_ADVECT);
        launch_advect_rotate(c->g, px, py, np, cx, cy, cos(angle), sin(angle), c->st);
    }
    return check_launch(c, "pm_advect_rotate");
}

pm_status pm_advect_rk2(pm_ctx *c, const float *mesh_vel, const float *vel, float *px, float *py, long long np,
                        double dt, float *vals, int F, double factor) {
    pm_status s = check_particles(c, px, py, np, F, vals, 0);
    if (s) return s;
    if (np > 0 && (!mesh_vel || !vel)) return fail(c, PM_EINVAL, "null velocity array");
    {
        Phase ph(c, PM_PH_ADVECT);
        launch_advect_rk2(c->g, mesh_vel, vel, px, py, np, (float)dt, vals, vals ? F : 0, (float)factor,
                          c->w.status, c->st);
    }
    return check_launch(c, "pm_advect_rk2");
}

pm_status pm_profile(pm_ctx *c, int enable) {
    if (!c) return PM_EINVAL;
    if (!enable) resolve_events(c);
    c->prof = enable != 0;
    c->count_work = enable == 2;
    return PM_OK;
}

pm_status pm_work_read(pm_ctx *c, long long *counts, int ncounts, int reset) {
    if (!c || !counts || ncounts < 0) return PM_EINVAL;
    ull h[8];
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "pm_work_read");
    if (cudaMemcpy(h, c->w.wsum, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "pm_work_read");
    for (int k = 0; k < ncounts; ++k) counts[k] = k < 8 ? (long long)h[k] : 0;
    if (reset && cudaMemset(c->w.wsum, 0, sizeof(h)) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "pm_work_read");
    return PM_OK;
}

pm_status pm_profile_read(pm_ctx *c, double *ms, long long *calls, int reset) {
    if (!c) return PM_EINVAL;
    resolve_events(c);
    for (int k = 0; k < PM_NPHASE; ++k) {
        if (ms) ms[k] = c->acc_ms[k];
        if (calls) calls[k] = c->acc_calls[k];
        if (reset) {
            c->acc_ms[k] = 0.0;
            c->acc_calls[k] = 0;
        }
    }
    return PM_OK;
}

const char *pm_phase_name(int ph) {
    static const char *names[PM_NPHASE] = {"sort", "triangulate", "delta", "flip", "rhs",
                                           "solve", "g2p", "advect", "other", "net"};
    return ph >= 0 && ph < PM_NPHASE ? names[ph] : "?";
}

long long pm_kernel_launches(void) { return g_launch_total.load(); }

#ifdef PM_CHECKED
}  // extern "C"
void pm_dbg_fetch_sort(int *);
void pm_dbg_fetch_delaunay(int *);
void pm_dbg_fetch_transfer(int *);
void pm_dbg_fetch_solve(int *);
extern "C" {
// Checked build only: first violated site code and violation count of each
// file (sort, delaunay, transfer, solve), then reset.
int pm_debug_read(int *out) {
    pm_dbg_fetch_sort(out);
    pm_dbg_fetch_delaunay(out + 2);
    pm_dbg_fetch_transfer(out + 4);
    pm_dbg_fetch_solve(out + 6);
    return 0;
}
#endif

}  // extern "C"

extern "C" {

pm_status pm_sort(pm_ctx *c, const float *px, const float *py, long long np, int *perm_out, int *cell_start_out) {
    pm_status s = check_particles(c, px, py, np, 0, nullptr, 0);
    if (s) return s;
    if (!perm_out || !cell_start_out) return fail(c, PM_EINVAL, "null output");
    if ((s = prepare(c, px, py, np, nullptr, 0, false))) return s;
    if (np > 0) cudaMemcpyAsync(perm_out, c->w.perm, sizeof(int) * np, cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(cell_start_out, c->w.cell_start, sizeof(int) * (c->g.ncell + 1), cudaMemcpyDeviceToDevice, c->st);
    return check_launch(c, "pm_sort");
}

}  // extern "C"
