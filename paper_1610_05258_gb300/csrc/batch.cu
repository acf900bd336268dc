// Batches of independent 2D instances (no counterpart in the paper: many
// periodic problems of uneven mesh and particle sizes advanced together).
//
// Every instance lives in one packed workspace: instance k owns the particle
// slots [poff[k], poff[k+1]) and the cells/nodes [coff[k], coff[k+1]), so one
// launch per phase covers all instances. A mass assignment of the whole
// batch (Sec. 2.4, Eqs. proj and phi_def, as pm_assign_mass with the exact
// inverse as start) is
//
//   pack       caller arrays -> packed arrays                (per particle)
//   sort       cell keys, one scan over all cells, canonical
//              order, gather with max|A| per instance         (per particle / cell)
//   stars      periodic Delaunay stars, two retry passes       (per particle)
//   rhs        exact right-hand side                           (per 16x16-cell tile)
//   start      M^-1 b by separable circulant convolutions      (per 32x32 tile;
//              or the delta assignment per particle, or zero)
//   solve      mean mode, true residual, CG if it is not yet
//              below rtol, conservation and stability report,
//              result written to the caller's array             (one cluster per instance)
//
// about 18 launches per step whatever the number of instances, captured once
// into a CUDA graph and replayed while the arguments stay the same. Tables
// resolve a particle, cell or tile to its instance (binary search over the
// offsets). The autotuner times one step for each candidate setting the first
// time a batch of a given size class runs on a device and keeps the fastest:
// the threads per CTA and the CTAs per instance (a thread-block cluster that
// reduces through distributed shared memory) of the solve, and the packing
// order of the instances (as given, or largest first so that the longest
// solves start first).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace {

// Cluster-wide sum of one double per thread (every thread of the cluster
// receives it): warp shuffle tree, the warps' sums in index order, then the
// CTAs' sums read from each CTA's shared memory (DSMEM) in rank order, so the
// result is the same on every CTA and every run. slot[2] alternates between
// calls: a CTA writes slot[ph] only after every CTA has passed the barrier of
// the previous call, which follows its reads of slot[ph] two calls back.
template <int NT, int CS>
__device__ __forceinline__ double cluster_sum(double v, double *sh, double *slot, int &ph) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < NT / 32; ++k) s += sh[k];
        slot[ph] = s;
    }
    double tot = 0.0;
    if (CS == 1) {
        __syncthreads();
        tot = slot[ph];
    } else {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        for (int r = 0; r < CS; ++r) tot += *cl.map_shared_rank(&slot[ph], r);
    }
    ph ^= 1;
    return tot;
}

// Barrier over the instance's threads (the CTA, or its cluster), ordering
// their global-memory writes before the reads that follow.
template <int CS>
__device__ __forceinline__ void instance_sync() {
    if (CS == 1)
        __syncthreads();
    else
        cg::this_cluster().sync();
}

__global__ void k_pack(BTab t, const float *const *__restrict__ px, const float *const *__restrict__ py,
                       const float *const *__restrict__ vals, int F, float *__restrict__ opx,
                       float *__restrict__ opy, float *__restrict__ ovals) {
    const ll j = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= t.NP) return;
    const int k = find_slot(t.poff, t.ninst, j);
    const ll p0 = __ldg(t.poff + k), npk = __ldg(t.poff + k + 1) - p0, l = j - p0;
    opx[j] = px[k][l];
    opy[j] = py[k][l];
    for (int f = 0; f < F; ++f) ovals[(ll)f * t.NP + j] = vals[k][(ll)f * npk + l];
}

struct SolveArgs {
    BTab t;
    const int *order;        // block -> instance (packing order)
    int F;
    const float *b;          // [F][NC] right-hand side (float)
    float *x, *r, *p, *q;    // [F][NC]: start (the direct solve), CG vectors
    const float *vals;       // [F][NP] sorted particle values
    const float *vol;        // [NP] particle volumes
    float *const *out;       // [ninst] caller mesh arrays [F][n_k^2]
    double *scal;            // [ninst][PM_MAXF][16] report
    int *status;
    double rtol;
    int max_iter;
    int report;              // also the stability integrals
    const uint2 *pos;
    const int *nbr;
    const unsigned char *deg;
};

// One cluster of CS CTAs per instance: the same steps as the grid-wide CG kernel on one
// mesh (power-of-two field scale, exact mean mode from sum b, true residual
// with the compensated stencil, CG iterations only while it is above rtol),
// then the conservation sums and the result in the caller's array.
template <int NT, int CS>
__global__ void __launch_bounds__(NT) k_batch_solve(SolveArgs a) {
    __shared__ double sh[NT / 32];
    __shared__ double slot[2];
    int ph = 0;
    const BTab &t = a.t;
    // instance = cluster index; this CTA's threads take every CS-th chunk of NT
    const int k = a.order[blockIdx.x / CS];
    const int rank = CS == 1 ? 0 : (int)(blockIdx.x % CS);
    const ll t0 = (ll)rank * NT + threadIdx.x, TS = (ll)NT * CS;
    const BInst I = t.inst[k];
    const int n = I.n;
    const ll nn = (ll)n * n, co = t.coff[k], p0 = t.poff[k], p1 = t.poff[k + 1];
    const float c = I.h * I.h / 36.0f;
    const double hd = (double)I.h * I.h;
    const double tol2 = a.rtol * a.rtol;
    bool bad = false;
    for (int f = 0; f < a.F; ++f) {
        const ll fo = (ll)f * t.NC + co;
        const float *bf = a.b + fo;
        float *xf = a.x + fo, *rf = a.r + fo, *pf = a.p + fo, *qf = a.q + fo;
        // sums of b, |b| and the start
        Dot2 sb, sa, sx;
        for (ll i = t0; i < nn; i += TS) {
            const float bv = bf[i];
            sb.add(bv);
            sa.add(fabsf(bv));
            sx.add(xf[i]);
        }
        const double sumb = cluster_sum<NT, CS>((double)sb.hi + (double)sb.lo, sh, slot, ph);
        const double suma = cluster_sum<NT, CS>((double)sa.hi + (double)sa.lo, sh, slot, ph);
        const double sumx = cluster_sum<NT, CS>((double)sx.hi + (double)sx.lo, sh, slot, ph);
        const float S = solve_scale(suma / (double)nn);
        const float shv = (float)((double)S * (sumb / ((double)nn * hd) - sumx / (double)nn));
        // scaled start with the exact mean mode, scaled b (into q) and |S b|^2
        Dot2 s2;
        for (ll i = t0; i < nn; i += TS) {
            xf[i] = xf[i] * S + shv;
            const float bv = bf[i] * S;
            qf[i] = bv;
            s2.fma_acc(bv, bv);
        }
        const double bb = cluster_sum<NT, CS>((double)s2.hi + (double)s2.lo, sh, slot, ph);
        instance_sync<CS>();
        // r = S b - M x, p = r (q keeps S b until the first iteration)
        auto residual = [&](bool set_p) {
            Dot2 s;
            for (ll i = t0; i < nn; i += TS) {
                float hi, lo;
                stencil<2, 0>(xf, n, i, hi, lo);
                const float rv = fmaf(-c, hi, qf[i]) - c * lo;
                rf[i] = rv;
                if (set_p) pf[i] = rv;
                s.fma_acc(rv, rv);
            }
            return cluster_sum<NT, CS>((double)s.hi + (double)s.lo, sh, slot, ph);
        };
        double rr = residual(true);
        const double init = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        int it = 0;
        if (bb > 0.0 && rr > tol2 * bb) {
            // conjugate gradients on the instance (q holds M p during the
            // iterations; S b is rebuilt from b afterwards, the scale being an
            // exact power of two)
            for (it = 0; it < a.max_iter && rr > tol2 * bb; ++it) {
                Dot2 pq;
                for (ll i = t0; i < nn; i += TS) {
                    float hi, lo;
                    stencil<2, 0>(pf, n, i, hi, lo);
                    const float qv = c * hi + c * lo;
                    qf[i] = qv;
                    pq.fma_acc(pf[i], qv);
                }
                const double dpq = cluster_sum<NT, CS>((double)pq.hi + (double)pq.lo, sh, slot, ph);
                if (!(dpq > 0.0)) break;
                const float al = (float)(rr / dpq);
                Dot2 s;
                for (ll i = t0; i < nn; i += TS) {
                    xf[i] = fmaf(al, pf[i], xf[i]);
                    const float rv = fmaf(-al, qf[i], rf[i]);
                    rf[i] = rv;
                    s.fma_acc(rv, rv);
                }
                const double rn = cluster_sum<NT, CS>((double)s.hi + (double)s.lo, sh, slot, ph);
                const float be = (float)(rn / rr);
                rr = rn;
                for (ll i = t0; i < nn; i += TS) pf[i] = fmaf(be, pf[i], rf[i]);
                instance_sync<CS>();
            }
            // true residual against S b (rebuilt in q)
            for (ll i = t0; i < nn; i += TS) qf[i] = bf[i] * S;
            instance_sync<CS>();
            rr = residual(false);
        }
        // result, conservation and stability
        const float inv = 1.0f / S;  // a power of two: exact
        float *o = a.out[k] + (ll)f * nn;
        Dot2 sxx, em;
        for (ll i = t0; i < nn; i += TS) {
            const float xv = xf[i] * inv;
            o[i] = xv;
            sxx.add(xv);
        }
        const double sum_mesh = cluster_sum<NT, CS>((double)sxx.hi + (double)sxx.lo, sh, slot, ph) * hd;
        instance_sync<CS>();
        if (a.report) {
            for (ll i = t0; i < nn; i += TS) {
                float hi, lo;
                stencil<2, 0>(o, n, i, hi, lo);
                em.fma_acc(o[i], hi);
                em.fma_acc(o[i], lo);
            }
        }
        const double emesh = cluster_sum<NT, CS>((double)em.hi + (double)em.lo, sh, slot, ph) * ((double)I.L / n) * ((double)I.L / n) / 36.0;
        Dot2 pa, pb;
        const float *vf = a.vals + (ll)f * t.NP;
        for (ll s = p0 + t0; s < p1; s += TS) {
            const float v = a.vol[s], y = vf[s];
            pa.fma_acc(v, y);
            pb.fma_acc(v, fabsf(y));
        }
        const double sp = cluster_sum<NT, CS>((double)pa.hi + (double)pa.lo, sh, slot, ph);
        const double spa = cluster_sum<NT, CS>((double)pb.hi + (double)pb.lo, sh, slot, ph);
        // int A^2 over the instance's owned triangles (A^T M_p A)
        double ep = 0.0;
        if (a.report) {
            Dot2 e;
            for (ll s = p0 + t0; s < p1; s += TS) {
                const int m = a.deg[s];
                if (m < 3) continue;
                const uint2 Xp = a.pos[s];
                int ida = a.nbr[(ll)(m - 1) * t.NP + s] & 0x0fffffff;
                int ca = (unsigned)a.nbr[(ll)(m - 1) * t.NP + s] >> 28;
                for (int kk = 0; kk < m; ++kk) {
                    const int eb = a.nbr[(ll)kk * t.NP + s];
                    const int idb = eb & 0x0fffffff, cb = (unsigned)eb >> 28;
                    if (ida > s && idb > s) {
                        const uint2 A = a.pos[ida], B = a.pos[idb];
                        const ll ax = (ll)A.x + (ll)(ca / 3 - 1) * 4294967296LL - Xp.x;
                        const ll ay = (ll)A.y + (ll)(ca % 3 - 1) * 4294967296LL - Xp.y;
                        const ll bx = (ll)B.x + (ll)(cb / 3 - 1) * 4294967296LL - Xp.x;
                        const ll by = (ll)B.y + (ll)(cb % 3 - 1) * 4294967296LL - Xp.y;
                        const float w2 = (float)(ax * by - ay * bx) * 5.421010862427522e-20f;
                        const float u = vf[s], v = vf[ida], z = vf[idb];
                        e.fma_acc(w2, u * u + v * v + z * z + u * v + v * z + z * u);
                    }
                    ida = idb;
                    ca = cb;
                }
            }
            ep = cluster_sum<NT, CS>((double)e.hi + (double)e.lo, sh, slot, ph) * I.L * I.L / 12.0;
        }
        if (t0 == 0) {
            double *r = a.scal + ((ll)k * PM_MAXF + f) * 16;
            const double res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
            r[0] = it;
            r[1] = init;
            r[2] = res;
            r[3] = sum_mesh;
            r[4] = sp;
            r[5] = spa;
            r[6] = emesh;
            r[7] = ep;
            if (res > a.rtol) bad = true;
        }
        instance_sync<CS>();
    }
    if (t0 == 0 && bad) atomicOr(a.status, ST_NOTCONV);
}

}  // namespace

struct pm_batch {
    int ninst = 0, F_max = 0, dev = 0;
    std::vector<int> n;
    std::vector<double> L;
    std::vector<ll> max_np;
    cudaStream_t main = nullptr, user = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr, t0 = nullptr, t1 = nullptr;
    // packed workspace (sized for the sum of max_np and of n^2)
    Work w{};
    ll NPmax = 0, NC = 0;
    float *in_px = nullptr, *in_py = nullptr, *in_vals = nullptr;
    BInst *d_inst = nullptr;
    ll *d_poff = nullptr, *d_coff = nullptr;
    int *d_rtile = nullptr, *d_dtile = nullptr, *d_order = nullptr;
    void *d_taps = nullptr;
    const float **d_px = nullptr, **d_py = nullptr, **d_vals = nullptr;
    float **d_out = nullptr;
    double *hscal = nullptr;
    // the current layout
    std::vector<int> order;  // packing order: position -> instance
    std::vector<ll> np;      // particles per instance of the current layout
    BTab tab{};
    int ntiles_rhs = 0, ntiles_dir = 0;
    // tuning
    int threads = 0;     // solve block threads (256, 512, 1024); 0 = autotune
    int cluster = 1;     // CTAs per instance in the solve (a thread-block cluster of 1, 4 or 8)
    int largest_first = 0;
    int start = PM_WS_DIRECT;  // start of the solves
    double tuned_ms = 0.0;
    bool fixed = false;  // tuning given by the caller
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;
    long long graph_kernels = 0;
    std::string err;
};

namespace {

std::mutex g_tune_mu;
struct Tune {
    int threads = 0, cluster = 1, largest_first = 0;
};
std::map<std::tuple<int, int, int, int, int>, Tune> g_tune;  // (device, size class) -> setting

pm_status bfail(pm_batch *b, pm_status s, const std::string &m) {
    b->err = m;
    return s;
}

template <class T>
bool balloc(T **p, ll count) {
    return cudaMalloc((void **)p, sizeof(T) * (size_t)(count > 0 ? count : 1)) == cudaSuccess;
}

// Offsets, tables and taps of the layout (np per instance, packing order):
// host -> device copies on the batch's stream, outside any capture.
pm_status set_layout(pm_batch *b, const ll *np, int largest_first) {
    const int K = b->ninst;
    std::vector<int> order(K);
    for (int k = 0; k < K; ++k) order[k] = k;
    if (largest_first)
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (ll)b->n[x] * b->n[x] + np[x] > (ll)b->n[y] * b->n[y] + np[y];
        });
    // slot s of the packed layout holds instance order[s]; the tables are
    // indexed by slot, the caller's pointers and reports by instance
    std::vector<BInst> inst(K);
    std::vector<ll> poff(K + 1, 0), coff(K + 1, 0);
    std::vector<int> rt(K + 1, 0), dt(K + 1, 0);
    std::vector<unsigned char> taps((size_t)K * direct_taps_bytes());
    const int RT = rhs_tile_side();
    for (int s = 0; s < K; ++s) {
        const int k = order[s];
        const int n = b->n[k];
        const double L = b->L[k];
        inst[s].n = n;
        inst[s].invL = (float)(1.0 / L);
        inst[s].h = (float)(L / n);
        inst[s].L = L;
        const double u = L / 4294967296.0;
        inst[s].vol_scale = (float)(u * u / 6.0);
        poff[s + 1] = poff[s] + np[k];
        coff[s + 1] = coff[s] + (ll)n * n;
        const int tx = (n + RT - 1) / RT;
        rt[s + 1] = rt[s] + tx * tx;
        dt[s + 1] = dt[s] + direct_tile_count(n);
        make_direct_taps(n, L, taps.data() + (size_t)s * direct_taps_bytes());
    }
    // the solve blocks visit slots in packing order; order[] maps to instances
    // for the caller's arrays, so the slot tables use instance = slot here and
    // the caller pointer tables are permuted to slot order below
    std::vector<int> ident(K);
    for (int s = 0; s < K; ++s) ident[s] = s;
    cudaStream_t st = b->main;
    bool ok = cudaMemcpyAsync(b->d_inst, inst.data(), sizeof(BInst) * K, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_poff, poff.data(), sizeof(ll) * (K + 1), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_coff, coff.data(), sizeof(ll) * (K + 1), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_rtile, rt.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_dtile, dt.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_order, ident.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_taps, taps.data(), taps.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) return bfail(b, PM_ECUDA, "batch layout upload");
    b->order = order;
    b->np.assign(np, np + K);
    b->largest_first = largest_first;
    b->tab.inst = b->d_inst;
    b->tab.poff = b->d_poff;
    b->tab.coff = b->d_coff;
    b->tab.ninst = K;
    b->tab.NP = poff[K];
    b->tab.NC = coff[K];
    b->ntiles_rhs = rt[K];
    b->ntiles_dir = dt[K];
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->key.clear();
    return PM_OK;
}

// Caller pointers in slot order (device tables read by pack and solve).
pm_status set_pointers(pm_batch *b, const float *const *px, const float *const *py, const float *const *vals,
                       float *const *out) {
    const int K = b->ninst;
    std::vector<const float *> a(K), c(K), d(K);
    std::vector<float *> o(K);
    for (int s = 0; s < K; ++s) {
        const int k = b->order[s];
        a[s] = px[k];
        c[s] = py[k];
        d[s] = vals[k];
        o[s] = out[k];
    }
    cudaStream_t st = b->main;
    bool ok = cudaMemcpyAsync(b->d_px, a.data(), sizeof(void *) * K, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_py, c.data(), sizeof(void *) * K, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_vals, d.data(), sizeof(void *) * K, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(b->d_out, o.data(), sizeof(void *) * K, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaStreamSynchronize(st) == cudaSuccess;
    return ok ? PM_OK : bfail(b, PM_ECUDA, "batch pointer upload");
}

using SolveKernel = void (*)(SolveArgs);

SolveKernel solve_kernel(int threads, int cs) {
    if (threads == 1024)
        return cs == 8 ? k_batch_solve<1024, 8> : (cs == 4 ? k_batch_solve<1024, 4> : k_batch_solve<1024, 1>);
    if (threads == 256)
        return cs == 8 ? k_batch_solve<256, 8> : (cs == 4 ? k_batch_solve<256, 4> : k_batch_solve<256, 1>);
    return cs == 8 ? k_batch_solve<512, 8> : (cs == 4 ? k_batch_solve<512, 4> : k_batch_solve<512, 1>);
}

cudaLaunchConfig_t solve_config(int K, int threads, int cs, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K * cs);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Whether a (threads, cluster) setting of the solve can run on this device.
bool solve_fits(int threads, int cs) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = solve_config(1, threads, cs, nullptr, attr);
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, solve_kernel(threads, cs), &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

// Queue one step on the batch's main stream.
int enqueue_step(pm_batch *b, int F, double rtol, int max_iter, int report) {
    const BTab &t = b->tab;
    Work &w = b->w;
    cudaStream_t st = b->main;
    cudaMemsetAsync(w.status, 0, sizeof(int), st);
    k_pack<<<div_up(t.NP, 256), 256, 0, st>>>(t, b->d_px, b->d_py, b->d_vals, F, b->in_px, b->in_py, b->in_vals);
    count_launches(1);
    launch_sort_batched(t, w, b->in_px, b->in_py, b->in_vals, F, st);
    launch_triangulate_batched(t, w, st);
    launch_rhs_batched(t, w, F, b->d_rtile, b->ntiles_rhs, st);
    launch_rhs_to_float_batched(t, w, F, w.b, st);
    if (b->start == PM_WS_DELTA)
        launch_delta_batched(t, w, F, w.r, st);
    else if (b->start == PM_WS_ZERO)
        cudaMemsetAsync(w.r, 0, sizeof(float) * F * t.NC, st);
    else
        launch_mass_direct_batched(t, b->d_taps, b->d_dtile, b->ntiles_dir, w.b, F, w.r, w.p, st);
    SolveArgs a;
    a.t = t;
    a.order = b->d_order;
    a.F = F;
    a.b = w.b;
    a.x = w.r;  // the start (direct solve, delta assignment or zero)
    a.r = w.q;
    a.p = w.p;
    a.q = w.bfix ? (float *)w.bfix : nullptr;  // [F][NC] floats fit in the fixed-point array
    a.vals = w.vals;
    a.vol = w.vol;
    a.out = b->d_out;
    a.scal = w.scal;
    a.status = w.status;
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.report = report;
    a.pos = w.pos;
    a.nbr = w.nbr;
    a.deg = w.deg;
    const int K = b->ninst;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = solve_config(K, b->threads, b->cluster, st, attr);
    cudaError_t e = cudaLaunchKernelEx(&cfg, solve_kernel(b->threads, b->cluster), a);
    count_launches(1);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

}  // namespace

extern "C" {

pm_status pm_batch_create(pm_batch **out, int ninst, const int *n, const double *L, const long long *max_np,
                          int max_fields, int tune, void *stream) {
    if (!out || ninst < 1 || !n || !L || !max_np || max_fields < 1 || max_fields > PM_MAXF) return PM_EINVAL;
    if (tune != 0 && tune != 256 && tune != 512 && tune != 1024) return PM_EINVAL;
    *out = nullptr;
    ll NP = 0, NC = 0;
    for (int k = 0; k < ninst; ++k) {
        if (n[k] < 4 || !(L[k] > 0.0) || max_np[k] < 3) return PM_EINVAL;
        NP += max_np[k];
        NC += (ll)n[k] * n[k];
    }
    if (NP >= (1LL << 28) - 16 || NC >= (1LL << 31) - 1) return PM_EINVAL;
    pm_batch *b = new pm_batch();
    b->ninst = ninst;
    b->F_max = max_fields;
    b->n.assign(n, n + ninst);
    b->L.assign(L, L + ninst);
    b->max_np.assign(max_np, max_np + ninst);
    b->user = (cudaStream_t)stream;
    b->NPmax = NP;
    b->NC = NC;
    b->threads = tune;
    b->fixed = tune != 0;
    cudaGetDevice(&b->dev);
    Work &w = b->w;
    const ll F = max_fields;
    bool ok = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&b->t0) == cudaSuccess && cudaEventCreate(&b->t1) == cudaSuccess;
    ok = ok && balloc(&w.fx, NP) && balloc(&w.key, NP) && balloc(&w.slot, NP) && balloc(&w.count, NC) &&
         balloc(&w.cell_start, NC + 1) && balloc(&w.scan_tmp, NC / 4096 + 2) && balloc(&w.tmp, NP) &&
         balloc(&w.perm, NP) && balloc(&w.pos, NP) && balloc(&w.vals, NP * F) &&
         balloc(&w.maxabs, (ll)PM_MAXF * ninst) && balloc(&w.deg, NP) && balloc(&w.vol, NP) &&
         balloc(&w.nbr, (ll)PM_MAXDEG * NP) && balloc(&w.bfix, F * NC) && balloc(&w.b, F * NC) &&
         balloc(&w.r, F * NC) && balloc(&w.p, F * NC) && balloc(&w.q, F * NC) &&
         balloc(&w.scal, 16LL * PM_MAXF * ninst) && balloc(&w.status, 1) && balloc(&w.nretry, 1) &&
         balloc(&b->in_px, NP) && balloc(&b->in_py, NP) && balloc(&b->in_vals, NP * F) &&
         balloc(&b->d_inst, ninst) && balloc(&b->d_poff, ninst + 1) && balloc(&b->d_coff, ninst + 1) &&
         balloc(&b->d_rtile, ninst + 1) && balloc(&b->d_dtile, ninst + 1) && balloc(&b->d_order, ninst) &&
         balloc((unsigned char **)&b->d_taps, (ll)direct_taps_bytes() * ninst) && balloc(&b->d_px, ninst) &&
         balloc(&b->d_py, ninst) && balloc(&b->d_vals, ninst) && balloc(&b->d_out, ninst) &&
         cudaMallocHost((void **)&w.hstatus, sizeof(int)) == cudaSuccess &&
         cudaMallocHost((void **)&b->hscal, sizeof(double) * 16 * PM_MAXF * ninst) == cudaSuccess;
    w.np_max = NP;
    w.F_max = max_fields;
    if (ok) {
        rhs_prepare_device();
        ok = cudaMemset(w.deg, 0, (size_t)NP) == cudaSuccess && cudaMemset(w.scal, 0, sizeof(double) * 16 * PM_MAXF * ninst) == cudaSuccess &&
             cudaDeviceSynchronize() == cudaSuccess;
    }
    if (ok) ok = set_layout(b, b->max_np.data(), 0) == PM_OK;
    if (!ok) {
        pm_batch_destroy(b);
        cudaGetLastError();
        return PM_ENOMEM;
    }
    *out = b;
    return PM_OK;
}

void pm_batch_destroy(pm_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    Work &w = b->w;
    void *ptrs[] = {w.fx,     w.key,      w.slot,     w.count,    w.cell_start, w.scan_tmp, w.tmp,
                    w.perm,   w.pos,      w.vals,     w.maxabs,   w.deg,        w.vol,      w.nbr,
                    w.bfix,   w.b,        w.r,        w.p,        w.q,          w.scal,     w.status,
                    w.nretry, b->in_px,   b->in_py,   b->in_vals, b->d_inst,    b->d_poff,  b->d_coff,
                    b->d_rtile, b->d_dtile, b->d_order, b->d_taps, (void *)b->d_px, (void *)b->d_py,
                    (void *)b->d_vals, (void *)b->d_out};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w.hstatus) cudaFreeHost(w.hstatus);
    if (b->hscal) cudaFreeHost(b->hscal);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->main) cudaStreamDestroy(b->main);
    delete b;
}

const char *pm_batch_last_error(const pm_batch *b) { return b ? b->err.c_str() : "null batch"; }

pm_status pm_batch_set_start(pm_batch *b, int warm_start) {
    if (!b) return PM_EINVAL;
    if (warm_start != PM_WS_DIRECT && warm_start != PM_WS_DELTA && warm_start != PM_WS_ZERO)
        return bfail(b, PM_EINVAL, "batch start must be PM_WS_DIRECT, PM_WS_DELTA or PM_WS_ZERO");
    if (warm_start != b->start) {
        b->start = warm_start;
        b->key.clear();  // recapture
    }
    return PM_OK;
}

pm_status pm_batch_tuning(const pm_batch *b, int *threads, int *cluster, int *largest_first, double *step_ms) {
    if (!b) return PM_EINVAL;
    if (threads) *threads = b->threads;
    if (cluster) *cluster = b->cluster;
    if (largest_first) *largest_first = b->largest_first;
    if (step_ms) *step_ms = b->tuned_ms;
    return PM_OK;
}

pm_status pm_batch_set_tuning(pm_batch *b, int threads, int cluster, int largest_first) {
    if (!b) return PM_EINVAL;
    if ((threads != 256 && threads != 512 && threads != 1024) || (cluster != 1 && cluster != 4 && cluster != 8))
        return bfail(b, PM_EINVAL, "threads must be 256, 512 or 1024 and cluster 1, 4 or 8");
    if (!solve_fits(threads, cluster)) return bfail(b, PM_EINVAL, "this cluster does not fit the device");
    b->threads = threads;
    b->cluster = cluster;
    b->fixed = true;
    if ((largest_first != 0) != (b->largest_first != 0)) {
        pm_status s = set_layout(b, b->np.data(), largest_first != 0);
        if (s) return s;
    }
    b->key.clear();  // recapture
    return PM_OK;
}

pm_status pm_batch_assign_mass(pm_batch *b, const float *const *px, const float *const *py, const long long *np,
                               const float *const *vals, int F, float *const *mesh_out, double rtol, int max_iter,
                               pm_solve_info *info) {
    if (!b || !px || !py || !np || !vals || !mesh_out || F < 1 || F > b->F_max) return PM_EINVAL;
    const int K = b->ninst;
    for (int k = 0; k < K; ++k) {
        if (np[k] < 3 || np[k] > b->max_np[k]) return bfail(b, PM_EINVAL, "instance " + std::to_string(k) + ": particle count out of range");
        if (!px[k] || !py[k] || !vals[k] || !mesh_out[k]) return bfail(b, PM_EINVAL, "instance " + std::to_string(k) + ": null array");
    }
    if (!(rtol > 0.0)) rtol = 1e-6;
    if (max_iter <= 0) max_iter = 200;
    // the main stream follows the caller's stream
    cudaEventRecord(b->fork, b->user);
    cudaStreamWaitEvent(b->main, b->fork, 0);
    bool same_np = b->np.size() == (size_t)K && std::equal(b->np.begin(), b->np.end(), np);
    // autotune once per (device, size class): the solve's threads per CTA and
    // CTAs per instance (cluster) x the packing order
    if (!b->fixed && b->threads == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        ll NPt = 0;
        for (int k = 0; k < K; ++k) NPt += np[k];
        const auto cls = std::make_tuple(dev, K, (int)std::log2((double)NPt + 1.0), (int)std::log2((double)b->NC + 1.0), F);
        Tune best;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(cls);
            if (it != g_tune.end()) best = it->second;
        }
        if (!best.threads) {
            double best_ms = 1e30;
            const int cand[5][2] = {{1024, 1}, {512, 4}, {1024, 4}, {512, 8}, {1024, 8}};
            for (int lf : {1, 0}) {
                pm_status s = set_layout(b, np, lf);
                if (s) return s;
                if ((s = set_pointers(b, px, py, vals, mesh_out))) return s;
                for (const auto &c : cand) {
                    if (!solve_fits(c[0], c[1])) continue;
                    b->threads = c[0];
                    b->cluster = c[1];
                    int e = enqueue_step(b, F, rtol, max_iter, 0);  // warm
                    cudaEventRecord(b->t0, b->main);
                    e |= enqueue_step(b, F, rtol, max_iter, 0);
                    cudaEventRecord(b->t1, b->main);
                    if (e || cudaEventSynchronize(b->t1) != cudaSuccess) return bfail(b, PM_ECUDA, "autotune step");
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, b->t0, b->t1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best.threads = c[0];
                        best.cluster = c[1];
                        best.largest_first = lf;
                    }
                }
            }
            b->tuned_ms = best_ms;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[cls] = best;
        }
        b->threads = best.threads;
        b->cluster = best.cluster;
        if (best.largest_first != b->largest_first || !same_np) {
            pm_status s = set_layout(b, np, best.largest_first);
            if (s) return s;
        }
    } else if (!same_np) {
        pm_status s = set_layout(b, np, b->largest_first);
        if (s) return s;
    }
    // capture one step into a CUDA graph, replay it while the arguments match
    std::vector<const void *> key;
    key.push_back((const void *)(ll)F);
    key.push_back((const void *)(ll)b->threads);
    key.push_back((const void *)(ll)b->cluster);
    key.push_back((const void *)(ll)b->largest_first);
    key.push_back((const void *)(ll)b->start);
    for (int k = 0; k < K; ++k) {
        key.push_back(px[k]);
        key.push_back(py[k]);
        key.push_back(vals[k]);
        key.push_back(mesh_out[k]);
    }
    key.push_back((const void *)(ll)max_iter);
    key.push_back((const void *)(ll)(rtol * 1e12));
    if (!b->exec || key != b->key) {
        pm_status s = set_pointers(b, px, py, vals, mesh_out);
        if (s) return s;
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) return bfail(b, PM_ECUDA, std::string("capture: ") + cudaGetErrorString(ce));
        const long long l0 = pm_kernel_launches();
        const int e = enqueue_step(b, F, rtol, max_iter, 0);
        b->graph_kernels = pm_kernel_launches() - l0;
        count_launches(-(int)b->graph_kernels);  // counted when the graph runs
        ce = cudaStreamEndCapture(b->main, &b->graph);
        if (e) return bfail(b, PM_ECUDA, std::string("batch step: ") + cudaGetErrorString((cudaError_t)e));
        if (ce != cudaSuccess) return bfail(b, PM_ECUDA, std::string("end capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (ce != cudaSuccess) return bfail(b, PM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
        b->key = key;
    }
    if (info) {
        // a reported step runs outside the graph, with the stability integrals
        const int e = enqueue_step(b, F, rtol, max_iter, 1);
        if (e) return bfail(b, PM_ECUDA, std::string("batch step: ") + cudaGetErrorString((cudaError_t)e));
    } else {
        cudaError_t ce = cudaGraphLaunch(b->exec, b->main);
        if (ce != cudaSuccess) return bfail(b, PM_ECUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
        count_launches((int)b->graph_kernels);
    }
    cudaEventRecord(b->done, b->main);
    cudaStreamWaitEvent(b->user, b->done, 0);
    if (!info) return PM_OK;
    cudaMemcpyAsync(b->hscal, b->w.scal, sizeof(double) * 16 * PM_MAXF * K, cudaMemcpyDeviceToHost, b->main);
    cudaMemcpyAsync(b->w.hstatus, b->w.status, sizeof(int), cudaMemcpyDeviceToHost, b->main);
    if (cudaStreamSynchronize(b->main) != cudaSuccess) return bfail(b, PM_ECUDA, "batch report");
    for (int s = 0; s < K; ++s) {
        const int k = b->order[s];
        for (int f = 0; f < F; ++f) {
            const double *v = b->hscal + ((ll)s * PM_MAXF + f) * 16;
            pm_solve_info &o = info[(ll)k * F + f];
            o.iters = (int)v[0];
            o.init_rel_resid = v[1];
            o.rel_resid = v[2];
            o.sum_mesh = v[3];
            o.sum_particles = v[4];
            const double den = v[5] > 0.0 ? v[5] : fabs(v[4]);
            o.cons_err = den > 0.0 ? fabs(v[3] - v[4]) / den : fabs(v[3] - v[4]);
            o.energy_mesh = v[6];
            o.energy_particles = v[7];
        }
    }
    const int st = *b->w.hstatus;
    if (st & (ST_NONFINITE | ST_DUP | ST_SPARSE | ST_DEGREE | ST_RANGE))
        return bfail(b, PM_EDEGENERATE, "degenerate input in an instance (device status " + std::to_string(st) + ")");
    if (st & ST_TIMEOUT) return bfail(b, PM_ETIMEOUT, "a device-side wait timed out");
    if (st & ST_NOTCONV) return bfail(b, PM_ENOTCONV, "an instance's solve did not reach the requested residual");
    return PM_OK;
}

}  // extern "C"
