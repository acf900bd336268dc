// Mesh mass matrix m_ij = int psi_i psi_j (Sec. 2.4) and the solve M Ab = b
// (Eq. phi_def).
//
// M is applied matrix-free: 1D (h/6)(x_{i-1} + 4 x_i + x_{i+1}); 2D bilinear
// elements give the tensor product (h^2/36) [1 4 1; 4 16 4; 1 4 1]. Stencil
// sums are compensated (error-free transformations), so M x is accurate to
// about one rounding whatever the cancellation.
//
// The solve is conjugate gradients in ONE persistent cooperative kernel:
// every block owns a strided share of the nodes of all F fields, vectors stay
// in L2, and the three reductions per iteration go through per-block FP64
// partials that every block then sums in the same fixed order (deterministic
// and identical on all blocks, so all blocks take the same branch). Per-node
// products are accumulated per thread in compensated FP32 before entering
// FP64. Before iterating, the mean mode of x is set exactly from sum_j b_j
// (1 is an eigenvector of the circulant M with eigenvalue h^dim, and CG keeps
// the mean of the start vector), which makes the result conservative (Eq.
// cons) to rounding at any iteration count.
#include <cooperative_groups.h>

#include "internal.cuh"

PM_DEBUG_DECL(solve)

namespace {

struct CG {
    Geo g;
    int F;
    const float *bsrc;      // float right-hand side (or null)
    const ll *bfix;         // fixed-point right-hand side (or null)
    const unsigned *maxabs; // fixed-point scale source
    float *x, *r, *p, *q, *b;
    double *red;            // [6 * PM_MAXF][grid]
    double *scal;           // [F][16]
    unsigned *bar;          // [2] barrier count, generation
    int *status;
    double rtol;
    int max_iter;
    int has_start;
    const double *psum;     // particle sums per block (or null)
    int nblk_psum;
};

enum { S_ITERS = 0, S_INIT = 1, S_RESID = 2, S_SUMMESH = 3, S_SUMPART = 4, S_SUMABS = 5 };

// Grid-wide barrier with a bounded wait (about a second); on timeout the
// status word gets ST_TIMEOUT and false is returned.
__device__ bool grid_sync(unsigned *bar, int *status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *gen = bar + 1;
        unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g0) {
                __nanosleep(64);
                if (++spins > (1LL << 24)) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Block reduction of one double per field into red[slot*F + f][block].
__device__ void block_partial(double v[PM_MAXF], int F, double *red, int slot) {
    __shared__ double sh[PM_MAXF][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int f = 0; f < F; ++f) {
        double s = v[f];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh[f][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < F) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[threadIdx.x][w];
        PM_CHK((ll)(slot * F + threadIdx.x + 1) * gridDim.x <= 6LL * PM_MAXF * 1024, 401, s = 0)
        red[(ll)(slot * F + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
}

// Sum of the partials of (slot, f) over all blocks, same order on every block.
__device__ void grid_total(const double *red, int F, int slot, double out[PM_MAXF]) {
    __shared__ double tot[PM_MAXF];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < F) {
        const double *src = red + (ll)(slot * F + wid) * gridDim.x;
        double s = 0;
        for (unsigned i = lane; i < gridDim.x; i += 32) s += src[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) tot[wid] = s;
    }
    __syncthreads();
    for (int f = 0; f < F; ++f) out[f] = tot[f];
    __syncthreads();
}

// Compensated M x at node i of field array xf; returns (hi, lo) of the
// unscaled stencil sum; the caller multiplies by c = h/6 or h^2/36.
template <int DIM>
__device__ __forceinline__ void stencil(const float *__restrict__ xf, int n, ll i, float &hi, float &lo) {
    Dot2 acc;
    if (DIM == 1) {
        int ix = (int)i, xm = ix == 0 ? n - 1 : ix - 1, xp = ix + 1 == n ? 0 : ix + 1;
        acc.add(4.0f * xf[ix]);
        acc.add(xf[xm]);
        acc.add(xf[xp]);
    } else {
        int ix = (int)(i % n), iy = (int)(i / n);
        int xm = ix == 0 ? n - 1 : ix - 1, xp = ix + 1 == n ? 0 : ix + 1;
        int ym = iy == 0 ? n - 1 : iy - 1, yp = iy + 1 == n ? 0 : iy + 1;
        const float *r0 = xf + (ll)ym * n, *r1 = xf + (ll)iy * n, *r2 = xf + (ll)yp * n;
        acc.add(16.0f * r1[ix]);
        acc.add(4.0f * r1[xm]);
        acc.add(4.0f * r1[xp]);
        acc.add(4.0f * r0[ix]);
        acc.add(4.0f * r2[ix]);
        acc.add(r0[xm]);
        acc.add(r0[xp]);
        acc.add(r2[xm]);
        acc.add(r2[xp]);
    }
    hi = acc.hi;
    lo = acc.lo;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_cg(CG a) {
    const Geo g = a.g;
    const int F = a.F, n = g.n;
    const ll nn = g.ncell;
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    const float c = DIM == 1 ? g.h / 6.0f : g.h * g.h / 36.0f;
    const double hd = DIM == 1 ? (double)g.h : (double)g.h * g.h;
    double v[PM_MAXF], w[PM_MAXF];
    double bb[PM_MAXF], rr[PM_MAXF], alpha[PM_MAXF], beta[PM_MAXF];
    bool act[PM_MAXF];
    int it_f[PM_MAXF];
    // --- phase 0: right-hand side as float, its sum and norm, sum of start
    for (int f = 0; f < F; ++f) {
        Dot2 sb, s2, sx;
        float hd32 = DIM == 1 ? g.h : g.h * g.h;
        int E = 0;
        if (a.bfix) {
            float m = __uint_as_float(a.maxabs[f]) * hd32;
            if (m > 0.0f) { frexpf(m, &E); E = 60 - E; }
        }
        for (ll i = tid; i < nn; i += nth) {
            float bv = a.bfix ? ldexpf((float)a.bfix[(ll)f * nn + i], -E) : a.bsrc[(ll)f * nn + i];
            a.b[(ll)f * nn + i] = bv;
            sb.add(bv);
            s2.fma_acc(bv, bv);
            if (a.has_start) sx.add(a.x[(ll)f * nn + i]);
        }
        v[f] = (double)sb.hi + (double)sb.lo;
        w[f] = (double)s2.hi + (double)s2.lo;
        double t = (double)sx.hi + (double)sx.lo;
        alpha[f] = t;
    }
    block_partial(v, F, a.red, 0);
    block_partial(w, F, a.red, 1);
    block_partial(alpha, F, a.red, 2);
    if (!grid_sync(a.bar, a.status)) return;
    double sumb[PM_MAXF], sumx[PM_MAXF];
    grid_total(a.red, F, 0, sumb);
    grid_total(a.red, F, 1, bb);
    grid_total(a.red, F, 2, sumx);
    // exact mean mode: mean(x) = sum b / (nn h^dim)
    for (int f = 0; f < F; ++f) {
        double shift = sumb[f] / ((double)nn * hd) - (a.has_start ? sumx[f] / (double)nn : 0.0);
        float sh = (float)shift;
        for (ll i = tid; i < nn; i += nth) {
            float xv = a.has_start ? a.x[(ll)f * nn + i] : 0.0f;
            a.x[(ll)f * nn + i] = xv + sh;
        }
    }
    if (!grid_sync(a.bar, a.status)) return;
    // --- r = b - M x, p = r
    for (int f = 0; f < F; ++f) {
        Dot2 s;
        const float *xf = a.x + (ll)f * nn;
        for (ll i = tid; i < nn; i += nth) {
            float hi, lo;
            stencil<DIM>(xf, n, i, hi, lo);
            float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
            a.r[(ll)f * nn + i] = rv;
            a.p[(ll)f * nn + i] = rv;
            s.fma_acc(rv, rv);
        }
        v[f] = (double)s.hi + (double)s.lo;
    }
    block_partial(v, F, a.red, 0);
    if (!grid_sync(a.bar, a.status)) return;
    grid_total(a.red, F, 0, rr);
    const double tol2 = a.rtol * a.rtol;
    for (int f = 0; f < F; ++f) {
        act[f] = rr[f] > tol2 * bb[f] && bb[f] > 0.0;
        it_f[f] = 0;
        if (blockIdx.x == 0 && threadIdx.x == 0)
            a.scal[f * 16 + S_INIT] = bb[f] > 0.0 ? sqrt(rr[f] / bb[f]) : 0.0;
    }
    int restarts = 0;
    for (int it = 0; it < a.max_iter; ++it) {
        bool any = false;
        for (int f = 0; f < F; ++f) any |= act[f];
        if (!any) {
            // recursive residuals converged: check the true residual once
            for (int f = 0; f < F; ++f) {
                Dot2 s;
                const float *xf = a.x + (ll)f * nn;
                for (ll i = tid; i < nn; i += nth) {
                    float hi, lo;
                    stencil<DIM>(xf, n, i, hi, lo);
                    float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
                    s.fma_acc(rv, rv);
                }
                v[f] = (double)s.hi + (double)s.lo;
            }
            block_partial(v, F, a.red, 0);
            if (!grid_sync(a.bar, a.status)) return;
            double tr[PM_MAXF];
            grid_total(a.red, F, 0, tr);
            bool again = false;
            for (int f = 0; f < F; ++f)
                if (bb[f] > 0.0 && tr[f] > tol2 * bb[f]) { act[f] = true; again = true; }
            if (!again || restarts >= 3) break;
            ++restarts;
            // restart the drifted fields from their true residual
            for (int f = 0; f < F; ++f) {
                if (!act[f]) continue;
                Dot2 s;
                const float *xf = a.x + (ll)f * nn;
                for (ll i = tid; i < nn; i += nth) {
                    float hi, lo;
                    stencil<DIM>(xf, n, i, hi, lo);
                    float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
                    a.r[(ll)f * nn + i] = rv;
                    a.p[(ll)f * nn + i] = rv;
                    s.fma_acc(rv, rv);
                }
                v[f] = (double)s.hi + (double)s.lo;
            }
            block_partial(v, F, a.red, 0);
            if (!grid_sync(a.bar, a.status)) return;
            grid_total(a.red, F, 0, w);
            for (int f = 0; f < F; ++f)
                if (act[f]) rr[f] = w[f];
        }
        // q = M p, (p, q)
        for (int f = 0; f < F; ++f) {
            v[f] = 0.0;
            if (!act[f]) continue;
            Dot2 s;
            const float *pf = a.p + (ll)f * nn;
            for (ll i = tid; i < nn; i += nth) {
                float hi, lo;
                stencil<DIM>(pf, n, i, hi, lo);
                float qv = fmaf(c, hi, c * lo);
                a.q[(ll)f * nn + i] = qv;
                s.fma_acc(pf[i], qv);
            }
            v[f] = (double)s.hi + (double)s.lo;
        }
        block_partial(v, F, a.red, 0);
        if (!grid_sync(a.bar, a.status)) return;
        grid_total(a.red, F, 0, w);
        // x += alpha p, r -= alpha q, (r, r)
        for (int f = 0; f < F; ++f) {
            v[f] = 0.0;
            if (!act[f]) continue;
            alpha[f] = rr[f] / w[f];
            const float al = (float)alpha[f];
            Dot2 s;
            for (ll i = tid; i < nn; i += nth) {
                ll o = (ll)f * nn + i;
                a.x[o] = fmaf(al, a.p[o], a.x[o]);
                float rv = fmaf(-al, a.q[o], a.r[o]);
                a.r[o] = rv;
                s.fma_acc(rv, rv);
            }
            v[f] = (double)s.hi + (double)s.lo;
        }
        block_partial(v, F, a.red, 0);
        if (!grid_sync(a.bar, a.status)) return;
        grid_total(a.red, F, 0, w);
        for (int f = 0; f < F; ++f) {
            if (!act[f]) continue;
            beta[f] = w[f] / rr[f];
            rr[f] = w[f];
            ++it_f[f];
            if (rr[f] <= tol2 * bb[f]) act[f] = false;
        }
        // p = r + beta p
        for (int f = 0; f < F; ++f) {
            if (!act[f]) continue;
            const float be = (float)beta[f];
            for (ll i = tid; i < nn; i += nth) {
                ll o = (ll)f * nn + i;
                a.p[o] = fmaf(be, a.p[o], a.r[o]);
            }
        }
        if (!grid_sync(a.bar, a.status)) return;
    }
    // --- report: true residual and sum of the mesh field
    for (int f = 0; f < F; ++f) {
        Dot2 s, sx;
        const float *xf = a.x + (ll)f * nn;
        for (ll i = tid; i < nn; i += nth) {
            float hi, lo;
            stencil<DIM>(xf, n, i, hi, lo);
            float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
            s.fma_acc(rv, rv);
            sx.add(xf[i]);
        }
        v[f] = (double)s.hi + (double)s.lo;
        w[f] = (double)sx.hi + (double)sx.lo;
    }
    block_partial(v, F, a.red, 0);
    block_partial(w, F, a.red, 1);
    if (!grid_sync(a.bar, a.status)) return;
    double tr[PM_MAXF], sx[PM_MAXF];
    grid_total(a.red, F, 0, tr);
    grid_total(a.red, F, 1, sx);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool bad = false;
        for (int f = 0; f < F; ++f) {
            double res = bb[f] > 0.0 ? sqrt(tr[f] / bb[f]) : 0.0;
            a.scal[f * 16 + S_ITERS] = it_f[f];
            a.scal[f * 16 + S_RESID] = res;
            a.scal[f * 16 + S_SUMMESH] = sx[f] * hd;
            if (a.psum) {
                double s1 = 0, s2 = 0;
                for (int k = 0; k < a.nblk_psum; ++k) {
                    s1 += a.psum[(ll)(2 * f) * a.nblk_psum + k];
                    s2 += a.psum[(ll)(2 * f + 1) * a.nblk_psum + k];
                }
                a.scal[f * 16 + S_SUMPART] = s1;
                a.scal[f * 16 + S_SUMABS] = s2;
            } else {
                a.scal[f * 16 + S_SUMPART] = sumb[f];
                a.scal[f * 16 + S_SUMABS] = 0.0;
            }
            if (res > a.rtol) bad = true;
        }
        if (bad) atomicOr(a.status, ST_NOTCONV);
    }
}

template <int DIM>
__global__ void k_mass_apply(Geo g, const float *__restrict__ x, int F, float *__restrict__ y) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const float c = DIM == 1 ? g.h / 6.0f : g.h * g.h / 36.0f;
    for (int f = 0; f < F; ++f) {
        float hi, lo;
        stencil<DIM>(x + (ll)f * g.ncell, g.n, i, hi, lo);
        y[(ll)f * g.ncell + i] = fmaf(c, hi, c * lo);
    }
}

int g_cg_grid[2] = {0, 0};

}  // namespace

void launch_mass_apply(const Geo &g, const float *x, int F, float *y, cudaStream_t st) {
    if (g.dim == 1)
        k_mass_apply<1><<<div_up(g.ncell, 256), 256, 0, st>>>(g, x, F, y);
    else
        k_mass_apply<2><<<div_up(g.ncell, 256), 256, 0, st>>>(g, x, F, y);
    count_launches(1);
}

// Returns 0 or a CUDA error code.
int launch_cg(const Geo &g, Work &w, int F, const float *b_float, bool b_from_fix, float *x, bool x_has_start,
              double rtol, int max_iter, cudaStream_t st) {
    CG a;
    a.g = g;
    a.F = F;
    a.bsrc = b_float;
    a.bfix = b_from_fix ? w.bfix : nullptr;
    a.maxabs = w.maxabs;
    a.x = x;
    a.r = w.r;
    a.p = w.p;
    a.q = w.q;
    a.b = w.b;
    a.red = w.red;
    a.scal = w.scal;
    a.bar = w.bar;
    a.status = w.status;
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.has_start = x_has_start ? 1 : 0;
    a.psum = b_from_fix ? w.psum : nullptr;
    a.nblk_psum = w.nblk_psum;
    const int di = g.dim - 1;
    void (*kern)(CG) = g.dim == 1 ? k_cg<1> : k_cg<2>;
    if (!g_cg_grid[di]) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0);
        if (per < 1) per = 1;
        if (per > 2) per = 2;
        g_cg_grid[di] = sms * per;
    }
    int grid = g_cg_grid[di];
    ll need = (g.ncell + 255) / 256;
    if (need < grid) grid = (int)(need < 1 ? 1 : need);
    cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st);
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(256), args, 0, st);
    count_launches(1);
    return (int)e;
}
