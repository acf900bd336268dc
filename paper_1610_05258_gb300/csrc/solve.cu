// Mesh mass matrix m_ij = int psi_i psi_j (Sec. 2.4) and the solve M Ab = b
// (Eq. phi_def).
//
// M is applied matrix-free: 1D (h/6)(x_{i-1} + 4 x_i + x_{i+1}); 2D bilinear
// elements give the tensor product (h^2/36) [1 4 1; 4 16 4; 1 4 1]; 2D P1
// elements on cells split by the (0,0)-(1,1) diagonal give (h^2/12) times 6 at
// the node and 1 at its six edge neighbours (row sums h^2 in every case). Stencil
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

#include <mutex>

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
    float *r2;              // second residual buffer of the blocked Chebyshev passes (2D)
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

// Totals of the per-block particle sums (sum v A, sum v |A|) of every field:
// warp f sums field f's partials (lanes stride, fixed shuffle tree), so the
// result is the same on every run. Called by all threads of one block.
__device__ void particle_sums(const double *psum, int nblk, int F, double s1[PM_MAXF], double s2[PM_MAXF]) {
    __shared__ double tot[2 * PM_MAXF];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = wid; k < 2 * F; k += (int)(blockDim.x >> 5)) {
        const double *src = psum + (ll)k * nblk;
        double s = 0;
        for (int i = lane; i < nblk; i += 32) s += src[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) tot[k] = s;
    }
    __syncthreads();
    for (int f = 0; f < F; ++f) {
        s1[f] = tot[2 * f];
        s2[f] = tot[2 * f + 1];
    }
}

template <int DIM, int P1>
__global__ void __launch_bounds__(256) k_cg(CG a) {
    // Reduction slot groups alternate (3 (k & 1) for the k-th reduction), so a
    // block that runs ahead never overwrites partials another block is summing.
    int rk = 0, rg = 0;
    const Geo g = a.g;
    const int F = a.F, n = g.n;
    const ll nn = g.ncell;
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    const float c = DIM == 1 ? g.h / 6.0f : (P1 ? g.h * g.h / 12.0f : g.h * g.h / 36.0f);
    const double hd = DIM == 1 ? (double)g.h : (double)g.h * g.h;
    double v[PM_MAXF], w[PM_MAXF];
    double bb[PM_MAXF], rr[PM_MAXF], alpha[PM_MAXF], beta[PM_MAXF];
    bool act[PM_MAXF];
    int it_f[PM_MAXF];
    // --- phase 0: right-hand side as float, its sum and sum of |b|, sum of start
    for (int f = 0; f < F; ++f) {
        Dot2 sb, sa, sx;
        const float hd32 = DIM == 1 ? g.h : g.h * g.h;
        const int E = a.bfix ? fixed_point_exp(__uint_as_float(a.maxabs[f]), hd32) : 0;
        for (ll i = tid; i < nn; i += nth) {
            float bv = a.bfix ? ldexpf((float)a.bfix[(ll)f * nn + i], -E) : a.bsrc[(ll)f * nn + i];
            a.b[(ll)f * nn + i] = bv;
            sb.add(bv);
            sa.add(fabsf(bv));
            if (a.has_start) sx.add(a.x[(ll)f * nn + i]);
        }
        v[f] = (double)sb.hi + (double)sb.lo;
        w[f] = (double)sa.hi + (double)sa.lo;
        alpha[f] = (double)sx.hi + (double)sx.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(v, F, a.red, rg);
    block_partial(w, F, a.red, rg + 1);
    block_partial(alpha, F, a.red, rg + 2);
    if (!grid_sync(a.bar, a.status)) return;
    double sumb[PM_MAXF], sumx[PM_MAXF], suma[PM_MAXF];
    grid_total(a.red, F, rg, sumb);
    grid_total(a.red, F, rg + 1, suma);
    grid_total(a.red, F, rg + 2, sumx);
    // The system is solved for S b with S a power of two that brings the mean
    // |b| to order one (exact scaling: FP32 inner products of any field stay
    // in range); x is scaled by S on entry and by 1/S on exit. Then the exact
    // mean mode: mean(x) = sum b / (nn h^dim), and the norm of S b.
    float S[PM_MAXF];
    for (int f = 0; f < F; ++f) {
        S[f] = solve_scale(suma[f] / (double)nn);
        const double shift = (double)S[f] * (sumb[f] / ((double)nn * hd) - (a.has_start ? sumx[f] / (double)nn : 0.0));
        const float sh = (float)shift;
        Dot2 s2;
        for (ll i = tid; i < nn; i += nth) {
            const float xv = a.has_start ? a.x[(ll)f * nn + i] * S[f] : 0.0f;
            a.x[(ll)f * nn + i] = xv + sh;
            const float bv = a.b[(ll)f * nn + i] * S[f];
            a.b[(ll)f * nn + i] = bv;
            s2.fma_acc(bv, bv);
        }
        w[f] = (double)s2.hi + (double)s2.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(w, F, a.red, rg);
    if (!grid_sync(a.bar, a.status)) return;
    grid_total(a.red, F, rg, bb);
    // --- r = b - M x, p = r
    for (int f = 0; f < F; ++f) {
        Dot2 s;
        const float *xf = a.x + (ll)f * nn;
        for (ll i = tid; i < nn; i += nth) {
            float hi, lo;
            stencil<DIM, P1>(xf, n, i, hi, lo);
            float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
            a.r[(ll)f * nn + i] = rv;
            a.p[(ll)f * nn + i] = rv;
            s.fma_acc(rv, rv);
        }
        v[f] = (double)s.hi + (double)s.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(v, F, a.red, rg);
    if (!grid_sync(a.bar, a.status)) return;
    grid_total(a.red, F, rg, rr);
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
                    stencil<DIM, P1>(xf, n, i, hi, lo);
                    float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
                    s.fma_acc(rv, rv);
                }
                v[f] = (double)s.hi + (double)s.lo;
            }
            rg = 3 * (rk++ & 1);
            block_partial(v, F, a.red, rg);
            if (!grid_sync(a.bar, a.status)) return;
            double tr[PM_MAXF];
            grid_total(a.red, F, rg, tr);
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
                    stencil<DIM, P1>(xf, n, i, hi, lo);
                    float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
                    a.r[(ll)f * nn + i] = rv;
                    a.p[(ll)f * nn + i] = rv;
                    s.fma_acc(rv, rv);
                }
                v[f] = (double)s.hi + (double)s.lo;
            }
            rg = 3 * (rk++ & 1);
            block_partial(v, F, a.red, rg);
            if (!grid_sync(a.bar, a.status)) return;
            grid_total(a.red, F, rg, w);
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
                stencil<DIM, P1>(pf, n, i, hi, lo);
                float qv = fmaf(c, hi, c * lo);
                a.q[(ll)f * nn + i] = qv;
                s.fma_acc(pf[i], qv);
            }
            v[f] = (double)s.hi + (double)s.lo;
        }
        rg = 3 * (rk++ & 1);
        block_partial(v, F, a.red, rg);
        if (!grid_sync(a.bar, a.status)) return;
        grid_total(a.red, F, rg, w);
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
        rg = 3 * (rk++ & 1);
        block_partial(v, F, a.red, rg);
        if (!grid_sync(a.bar, a.status)) return;
        grid_total(a.red, F, rg, w);
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
            stencil<DIM, P1>(xf, n, i, hi, lo);
            float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
            s.fma_acc(rv, rv);
            sx.add(xf[i]);
        }
        v[f] = (double)s.hi + (double)s.lo;
        w[f] = (double)sx.hi + (double)sx.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(v, F, a.red, rg);
    block_partial(w, F, a.red, rg + 1);
    if (!grid_sync(a.bar, a.status)) return;
    double tr[PM_MAXF], sx[PM_MAXF];
    grid_total(a.red, F, rg, tr);
    grid_total(a.red, F, rg + 1, sx);
    double ps1[PM_MAXF], ps2[PM_MAXF];
    if (blockIdx.x == 0 && a.psum) particle_sums(a.psum, a.nblk_psum, F, ps1, ps2);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool bad = false;
        for (int f = 0; f < F; ++f) {
            double res = bb[f] > 0.0 ? sqrt(tr[f] / bb[f]) : 0.0;
            a.scal[f * 16 + S_ITERS] = it_f[f];
            a.scal[f * 16 + S_RESID] = res;
            a.scal[f * 16 + S_SUMMESH] = sx[f] * hd / (double)S[f];
            if (a.psum) {
                a.scal[f * 16 + S_SUMPART] = ps1[f];
                a.scal[f * 16 + S_SUMABS] = ps2[f];
            } else {
                a.scal[f * 16 + S_SUMPART] = sumb[f];
                a.scal[f * 16 + S_SUMABS] = 0.0;
            }
            if (res > a.rtol) bad = true;
        }
        if (bad) atomicOr(a.status, ST_NOTCONV);
    }
    for (int f = 0; f < F; ++f) {
        const float inv = 1.0f / S[f];  // a power of two: exact
        for (ll i = tid; i < nn; i += nth) a.x[(ll)f * nn + i] *= inv;
    }
}

// ---------------------------------------------------------------------------
// Chebyshev iteration for M x = b. The spectrum of the periodic mass matrix
// is known in closed form (Fourier modes): [h/3, h] in 1D, [h^2/9, h^2] on
// the bilinear mesh, [h^2/4, h^2] on the P1 mesh. With theta and delta the
// centre and half-width of that interval, sigma = theta / delta, the
// iteration
//   d_0 = r_0 / theta, rho_0 = 1 / sigma,
//   x += d_k, r -= M d_k, rho_{k+1} = 1 / (2 sigma - rho_k),
//   d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) r
// reduces the residual by the scaled Chebyshev polynomial, whose maximum on
// the interval is at most 2 q^k, q = (sqrt(kappa) - 1) / (sqrt(kappa) + 1).
// It needs no inner products: the number of steps for the tolerance follows
// from ||r_0|| and that bound, one grid barrier per step; the true residual
// is then recomputed and, if rounding left it above the tolerance, the
// iteration restarts from it (at most three times). The mean mode is set
// exactly first, as for CG, and every update d_k has zero mean, so the result
// is conservative to rounding.
// ---------------------------------------------------------------------------
// Temporal blocking of the Chebyshev steps (2D): a tile of CT x CT nodes
// with a halo of CH nodes runs up to CH steps in shared memory, the valid
// region shrinking by one node per step, then writes its interior back.
#define CT 32
#define CH 4
#define CR (CT + 2 * CH)

// stencil<2, P1> on a CR x CR shared-memory region: the same terms in the
// same order, so the same bits as on the global array.
template <int P1>
__device__ __forceinline__ void stencil_s(const float *__restrict__ d, int i, float &hi, float &lo) {
    Dot2 acc;
    const float *r0 = d + i - CR, *r1 = d + i, *r2 = d + i + CR;
    if (P1) {
        acc.add(6.0f * r1[0]);
        acc.add(r1[-1]);
        acc.add(r1[1]);
        acc.add(r0[0]);
        acc.add(r2[0]);
        acc.add(r0[-1]);
        acc.add(r2[1]);
    } else {
        acc.add(16.0f * r1[0]);
        acc.add(4.0f * r1[-1]);
        acc.add(4.0f * r1[1]);
        acc.add(4.0f * r0[0]);
        acc.add(4.0f * r2[0]);
        acc.add(r0[-1]);
        acc.add(r0[1]);
        acc.add(r2[-1]);
        acc.add(r2[1]);
    }
    hi = acc.hi;
    lo = acc.lo;
}

template <int DIM, int P1>
__global__ void __launch_bounds__(256) k_cheb(CG a) {
    // Reduction slot groups alternate (3 (k & 1) for the k-th reduction), so a
    // block that runs ahead never overwrites partials another block is summing.
    int rk = 0, rg = 0;
    const Geo g = a.g;
    const int F = a.F, n = g.n;
    const ll nn = g.ncell;
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    const float c = DIM == 1 ? g.h / 6.0f : (P1 ? g.h * g.h / 12.0f : g.h * g.h / 36.0f);
    const double hd = DIM == 1 ? (double)g.h : (double)g.h * g.h;
    // spectrum bounds, widened by 1e-6 against rounding of the operator
    const double lmin = hd * (DIM == 1 ? 1.0 / 3.0 : (P1 ? 0.25 : 1.0 / 9.0)) * (1.0 - 1e-6);
    const double lmax = hd * (1.0 + 1e-6);
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    const double kap = lmax / lmin, q = (sqrt(kap) - 1.0) / (sqrt(kap) + 1.0);
    double v[PM_MAXF], w[PM_MAXF], u[PM_MAXF], bb[PM_MAXF], rr[PM_MAXF];
    // --- right-hand side as float, its sum and sum of |b|, sum of the start
    for (int f = 0; f < F; ++f) {
        Dot2 sb, sa, sx;
        const float hd32 = DIM == 1 ? g.h : g.h * g.h;
        const int E = a.bfix ? fixed_point_exp(__uint_as_float(a.maxabs[f]), hd32) : 0;
        for (ll i = tid; i < nn; i += nth) {
            const float bv = a.bfix ? ldexpf((float)a.bfix[(ll)f * nn + i], -E) : a.bsrc[(ll)f * nn + i];
            a.b[(ll)f * nn + i] = bv;
            sb.add(bv);
            sa.add(fabsf(bv));
            if (a.has_start) sx.add(a.x[(ll)f * nn + i]);
        }
        v[f] = (double)sb.hi + (double)sb.lo;
        w[f] = (double)sa.hi + (double)sa.lo;
        u[f] = (double)sx.hi + (double)sx.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(v, F, a.red, rg);
    block_partial(w, F, a.red, rg + 1);
    block_partial(u, F, a.red, rg + 2);
    if (!grid_sync(a.bar, a.status)) return;
    double sumb[PM_MAXF], sumx[PM_MAXF], suma[PM_MAXF];
    grid_total(a.red, F, rg, sumb);
    grid_total(a.red, F, rg + 1, suma);
    grid_total(a.red, F, rg + 2, sumx);
    // solve for S b (S a power of two, as in k_cg), exact mean mode, |S b|^2
    float S[PM_MAXF];
    for (int f = 0; f < F; ++f) {
        S[f] = solve_scale(suma[f] / (double)nn);
        const double shift = (double)S[f] * (sumb[f] / ((double)nn * hd) - (a.has_start ? sumx[f] / (double)nn : 0.0));
        const float sh = (float)shift;
        Dot2 s2;
        for (ll i = tid; i < nn; i += nth) {
            const float xv = a.has_start ? a.x[(ll)f * nn + i] * S[f] : 0.0f;
            a.x[(ll)f * nn + i] = xv + sh;
            const float bv = a.b[(ll)f * nn + i] * S[f];
            a.b[(ll)f * nn + i] = bv;
            s2.fma_acc(bv, bv);
        }
        w[f] = (double)s2.hi + (double)s2.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(w, F, a.red, rg);
    if (!grid_sync(a.bar, a.status)) return;
    grid_total(a.red, F, rg, bb);
    const double tol2 = a.rtol * a.rtol;
    int steps_done = 0, steps_f[PM_MAXF];
    for (int f = 0; f < PM_MAXF; ++f) steps_f[f] = 0;
    for (int pass = 0;; ++pass) {
        // --- r = b - M x (the true residual), d = r / theta, (r, r), sum x
        for (int f = 0; f < F; ++f) {
            Dot2 s, sx;
            const float *xf = a.x + (ll)f * nn;
            for (ll i = tid; i < nn; i += nth) {
                float hi, lo;
                stencil<DIM, P1>(xf, n, i, hi, lo);
                const float rv = fmaf(-c, hi, a.b[(ll)f * nn + i]) - c * lo;
                a.r[(ll)f * nn + i] = rv;
                a.p[(ll)f * nn + i] = (float)(rv / theta);
                s.fma_acc(rv, rv);
                sx.add(xf[i]);
            }
            v[f] = (double)s.hi + (double)s.lo;
            u[f] = (double)sx.hi + (double)sx.lo;
        }
        rg = 3 * (rk++ & 1);
        block_partial(v, F, a.red, rg);
        block_partial(u, F, a.red, rg + 1);
        if (!grid_sync(a.bar, a.status)) return;
        grid_total(a.red, F, rg, rr);
        double sx[PM_MAXF];
        grid_total(a.red, F, rg + 1, sx);
        if (pass == 0 && blockIdx.x == 0 && threadIdx.x == 0)
            for (int f = 0; f < F; ++f) a.scal[f * 16 + S_INIT] = bb[f] > 0.0 ? sqrt(rr[f] / bb[f]) : 0.0;
        // steps of each field for the bound 2 q^k ||r_0|| <= rtol ||b||; the
        // pass runs the largest, a field stops updating after its own
        int K = 0, Kf[PM_MAXF];
        for (int f = 0; f < F; ++f) {
            Kf[f] = 0;
            if (!(bb[f] > 0.0) || rr[f] <= tol2 * bb[f]) continue;
            const double ratio = a.rtol * sqrt(bb[f]) / (2.0 * sqrt(rr[f]));
            Kf[f] = min((int)ceil(log(ratio) / log(q)), a.max_iter - steps_done);
            K = max(K, Kf[f]);
        }
        if (K <= 0 || pass == 4) {
            // report: this pass computed the true residual of the final x
            double ps1[PM_MAXF], ps2[PM_MAXF];
            if (blockIdx.x == 0 && a.psum) particle_sums(a.psum, a.nblk_psum, F, ps1, ps2);
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                bool bad = false;
                for (int f = 0; f < F; ++f) {
                    const double res = bb[f] > 0.0 ? sqrt(rr[f] / bb[f]) : 0.0;
                    a.scal[f * 16 + S_ITERS] = steps_f[f];
                    a.scal[f * 16 + S_RESID] = res;
                    a.scal[f * 16 + S_SUMMESH] = sx[f] * hd / (double)S[f];
                    a.scal[f * 16 + S_SUMPART] = a.psum ? ps1[f] : sumb[f];
                    a.scal[f * 16 + S_SUMABS] = a.psum ? ps2[f] : 0.0;
                    if (res > a.rtol) bad = true;
                }
                if (bad) atomicOr(a.status, ST_NOTCONV);
            }
            for (int f = 0; f < F; ++f) {
                const float inv = 1.0f / S[f];  // a power of two: exact
                for (ll i = tid; i < nn; i += nth) a.x[(ll)f * nn + i] *= inv;
            }
            break;
        }
        // the residual partials must be read by every block before reuse
        if (!grid_sync(a.bar, a.status)) return;
        double rho = 1.0 / sigma;
        float *dc = a.p, *dn = a.q;
        if (DIM == 2) {
            // passes of up to CH steps; d and r alternate between two buffers
            // (other tiles read them as halo), x is only updated at its own
            // nodes. Every node gets the plain loop's arithmetic in the same
            // order, so the iterate is the same bits.
            __shared__ float sd[2][CR * CR], sr[CR * CR], sx[CT * CT];
            float *rc = a.r, *rn = a.r2;
            const int tside = (n + CT - 1) / CT, ntiles = tside * tside;
            for (int kb = 0; kb < K; kb += CH) {
                const int steps = min(CH, K - kb);
                float c1s[CH], c2s[CH];
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    c1s[j] = c2s[j] = 0.0f;
                    if (j < steps) {
                        const double rho1 = 1.0 / (2.0 * sigma - rho);
                        c1s[j] = (float)(rho1 * rho);
                        c2s[j] = (float)(2.0 * rho1 / delta);
                        rho = rho1;
                    }
                }
                for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                    const int tx0 = (tile % tside) * CT, ty0 = (tile / tside) * CT;
                    for (int f = 0; f < F; ++f) {
                        const int sf = min(steps, Kf[f] - kb);  // this field's steps in the pass
                        if (sf <= 0) continue;
                        const ll fo = (ll)f * nn;
                        for (int i = threadIdx.x; i < CR * CR; i += blockDim.x) {
                            const int gx = wrapi(tx0 - CH + i % CR, n), gy = wrapi(ty0 - CH + i / CR, n);
                            sd[0][i] = dc[fo + (ll)gy * n + gx];
                            sr[i] = rc[fo + (ll)gy * n + gx];
                        }
                        for (int i = threadIdx.x; i < CT * CT; i += blockDim.x) {
                            const int gx = tx0 + i % CT, gy = ty0 + i / CT;
                            sx[i] = gx < n && gy < n ? a.x[fo + (ll)gy * n + gx] : 0.0f;
                        }
                        __syncthreads();
                        int cur = 0;
                        for (int j = 0; j < sf; ++j) {
                            const int lo_ = j + 1, hi_ = CR - 1 - j;  // output region of this step
                            const float *din = sd[cur];
                            float *dout = sd[cur ^ 1];
                            for (int i = threadIdx.x; i < CR * CR; i += blockDim.x) {
                                const int lx = i % CR, ly = i / CR;
                                if (lx < lo_ || lx >= hi_ || ly < lo_ || ly >= hi_) continue;
                                float hi, lo;
                                stencil_s<P1>(din, i, hi, lo);
                                const float dv = din[i];
                                const int ix = lx - CH, iy = ly - CH;
                                if (ix >= 0 && ix < CT && iy >= 0 && iy < CT) sx[iy * CT + ix] += dv;
                                const float rv = sr[i] - fmaf(c, hi, c * lo);
                                sr[i] = rv;
                                dout[i] = fmaf(c1s[j], dv, c2s[j] * rv);
                            }
                            __syncthreads();
                            cur ^= 1;
                        }
                        for (int i = threadIdx.x; i < CT * CT; i += blockDim.x) {
                            const int ix = i % CT, iy = i / CT, gx = tx0 + ix, gy = ty0 + iy;
                            if (gx >= n || gy >= n) continue;
                            const int li = (iy + CH) * CR + ix + CH;
                            const ll o = fo + (ll)gy * n + gx;
                            a.x[o] = sx[i];
                            rn[o] = sr[li];
                            dn[o] = sd[cur][li];
                        }
                        __syncthreads();
                    }
                }
                float *t = dc;
                dc = dn;
                dn = t;
                t = rc;
                rc = rn;
                rn = t;
                if (!grid_sync(a.bar, a.status)) return;
            }
            steps_done += K;
            for (int f = 0; f < F; ++f) steps_f[f] += Kf[f];
            continue;
        }
        for (int k = 0; k < K; ++k) {
            const double rho1 = 1.0 / (2.0 * sigma - rho);
            const float c1 = (float)(rho1 * rho), c2 = (float)(2.0 * rho1 / delta);
            for (int f = 0; f < F; ++f) {
                if (k >= Kf[f]) continue;
                const float *df = dc + (ll)f * nn;
                for (ll i = tid; i < nn; i += nth) {
                    float hi, lo;
                    stencil<DIM, P1>(df, n, i, hi, lo);
                    const ll o = (ll)f * nn + i;
                    const float dv = df[i];
                    a.x[o] += dv;
                    const float rv = a.r[o] - fmaf(c, hi, c * lo);
                    a.r[o] = rv;
                    dn[o] = fmaf(c1, dv, c2 * rv);
                }
            }
            rho = rho1;
            float *t = dc;
            dc = dn;
            dn = t;
            if (!grid_sync(a.bar, a.status)) return;
        }
        steps_done += K;
        for (int f = 0; f < F; ++f) steps_f[f] += Kf[f];
    }
}

// ---------------------------------------------------------------------------
// 2D solve on quads of 4 consecutive nodes of a row (n % 4 == 0): the same
// algorithm and the same per-node arithmetic as k_cg<2>, with 16-byte loads
// and stores so that enough bytes are in flight to stream the vectors at HBM
// speed from a persistent grid.
// ---------------------------------------------------------------------------
struct Q4 {
    float v[4];
};

__device__ __forceinline__ Q4 ld4(const float *p) {
    const float4 t = *(const float4 *)p;
    return Q4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void st4(float *p, const Q4 &q) { *(float4 *)p = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]); }

// Compensated stencil sums (hi, lo) of the 4 nodes starting at flat index i0
// (i0 % 4 == 0), in the same addition order as stencil<2, P1>.
template <int P1>
__device__ __forceinline__ void stencil4(const float *__restrict__ xf, int n, ll i0, float hi[4], float lo[4],
                                         float ctr[4]) {
    const int ix = (int)(i0 % n), iy = (int)(i0 / n);
    const int ym = iy == 0 ? n - 1 : iy - 1, yp = iy + 1 == n ? 0 : iy + 1;
    const int xl = ix == 0 ? n - 1 : ix - 1, xr = ix + 4 == n ? 0 : ix + 4;
    const float *R0 = xf + (ll)ym * n, *R1 = xf + (ll)iy * n, *R2 = xf + (ll)yp * n;
    const Q4 a = ld4(R0 + ix), b = ld4(R1 + ix), c = ld4(R2 + ix);
    const float a_l = R0[xl], a_r = R0[xr], b_l = R1[xl], b_r = R1[xr], c_l = R2[xl], c_r = R2[xr];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float am = j == 0 ? a_l : a.v[j - 1], ap = j == 3 ? a_r : a.v[j + 1];
        const float bm = j == 0 ? b_l : b.v[j - 1], bp = j == 3 ? b_r : b.v[j + 1];
        const float cm = j == 0 ? c_l : c.v[j - 1], cp = j == 3 ? c_r : c.v[j + 1];
        Dot2 acc;
        if (P1) {
            acc.add(6.0f * b.v[j]);
            acc.add(bm);
            acc.add(bp);
            acc.add(a.v[j]);
            acc.add(c.v[j]);
            acc.add(am);
            acc.add(cp);
        } else {
            acc.add(16.0f * b.v[j]);
            acc.add(4.0f * bm);
            acc.add(4.0f * bp);
            acc.add(4.0f * a.v[j]);
            acc.add(4.0f * c.v[j]);
            acc.add(am);
            acc.add(ap);
            acc.add(cm);
            acc.add(cp);
        }
        hi[j] = acc.hi;
        lo[j] = acc.lo;
        ctr[j] = b.v[j];
    }
}

template <int P1>
__global__ void __launch_bounds__(256) k_cg2v(CG a) {
    // Reduction slot groups alternate (3 (k & 1) for the k-th reduction), so a
    // block that runs ahead never overwrites partials another block is summing.
    int rk = 0, rg = 0;
    const Geo g = a.g;
    const int F = a.F, n = g.n;
    const ll nn = g.ncell, nq = nn / 4;
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    const float c = P1 ? g.h * g.h / 12.0f : g.h * g.h / 36.0f;
    const double hd = (double)g.h * g.h;
    double v[PM_MAXF], w[PM_MAXF];
    double bb[PM_MAXF], rr[PM_MAXF], alpha[PM_MAXF], beta[PM_MAXF];
    bool act[PM_MAXF];
    int it_f[PM_MAXF];
    float *__restrict__ X = a.x;
    float *__restrict__ R = a.r;
    float *__restrict__ P = a.p;
    float *__restrict__ Qv = a.q;
    float *__restrict__ B = a.b;
    // --- phase 0: right-hand side as float, its sum and norm, sum of start
    for (int f = 0; f < F; ++f) {
        Dot2 sb, sa, sx;
        const float hd32 = g.h * g.h;
        const int E = a.bfix ? fixed_point_exp(__uint_as_float(a.maxabs[f]), hd32) : 0;
        for (ll qd = tid; qd < nq; qd += nth) {
            const ll o = (ll)f * nn + qd * 4;
            Q4 bv;
            if (a.bfix) {
                const longlong2 u = *(const longlong2 *)(a.bfix + o), w2 = *(const longlong2 *)(a.bfix + o + 2);
                bv.v[0] = ldexpf((float)u.x, -E);
                bv.v[1] = ldexpf((float)u.y, -E);
                bv.v[2] = ldexpf((float)w2.x, -E);
                bv.v[3] = ldexpf((float)w2.y, -E);
            } else {
                bv = ld4(a.bsrc + o);
            }
            st4(B + o, bv);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                sb.add(bv.v[j]);
                sa.add(fabsf(bv.v[j]));
            }
            if (a.has_start) {
                const Q4 xv = ld4(X + o);
#pragma unroll
                for (int j = 0; j < 4; ++j) sx.add(xv.v[j]);
            }
        }
        v[f] = (double)sb.hi + (double)sb.lo;
        w[f] = (double)sa.hi + (double)sa.lo;
        alpha[f] = (double)sx.hi + (double)sx.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(v, F, a.red, rg);
    block_partial(w, F, a.red, rg + 1);
    block_partial(alpha, F, a.red, rg + 2);
    if (!grid_sync(a.bar, a.status)) return;
    double sumb[PM_MAXF], sumx[PM_MAXF], suma[PM_MAXF];
    grid_total(a.red, F, rg, sumb);
    grid_total(a.red, F, rg + 1, suma);
    grid_total(a.red, F, rg + 2, sumx);
    // solve for S b (S a power of two, as in k_cg), exact mean mode, |S b|^2
    float S[PM_MAXF];
    for (int f = 0; f < F; ++f) {
        S[f] = solve_scale(suma[f] / (double)nn);
        const double shift = (double)S[f] * (sumb[f] / ((double)nn * hd) - (a.has_start ? sumx[f] / (double)nn : 0.0));
        const float sh = (float)shift;
        Dot2 s2;
        for (ll qd = tid; qd < nq; qd += nth) {
            const ll o = (ll)f * nn + qd * 4;
            Q4 xv = a.has_start ? ld4(X + o) : Q4{{0.0f, 0.0f, 0.0f, 0.0f}};
            Q4 bv = ld4(B + o);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                xv.v[j] = fmaf(xv.v[j], S[f], sh);
                bv.v[j] *= S[f];
                s2.fma_acc(bv.v[j], bv.v[j]);
            }
            st4(X + o, xv);
            st4(B + o, bv);
        }
        w[f] = (double)s2.hi + (double)s2.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(w, F, a.red, rg);
    if (!grid_sync(a.bar, a.status)) return;
    grid_total(a.red, F, rg, bb);
    // --- r = b - M x, p = r
    for (int f = 0; f < F; ++f) {
        Dot2 s;
        const float *xf = X + (ll)f * nn;
        for (ll qd = tid; qd < nq; qd += nth) {
            const ll o = (ll)f * nn + qd * 4;
            float hi[4], lo[4], ct[4];
            stencil4<P1>(xf, n, qd * 4, hi, lo, ct);
            const Q4 bv = ld4(B + o);
            Q4 rv;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                rv.v[j] = fmaf(-c, hi[j], bv.v[j]) - c * lo[j];
                s.fma_acc(rv.v[j], rv.v[j]);
            }
            st4(R + o, rv);
            st4(P + o, rv);
        }
        v[f] = (double)s.hi + (double)s.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(v, F, a.red, rg);
    if (!grid_sync(a.bar, a.status)) return;
    grid_total(a.red, F, rg, rr);
    const double tol2 = a.rtol * a.rtol;
    for (int f = 0; f < F; ++f) {
        act[f] = rr[f] > tol2 * bb[f] && bb[f] > 0.0;
        it_f[f] = 0;
        if (blockIdx.x == 0 && threadIdx.x == 0)
            a.scal[f * 16 + S_INIT] = bb[f] > 0.0 ? sqrt(rr[f] / bb[f]) : 0.0;
    }
    // squared true residual of field f (and optionally restart r = p = it)
    auto true_resid = [&](int f, bool restart) {
        Dot2 s;
        const float *xf = X + (ll)f * nn;
        for (ll qd = tid; qd < nq; qd += nth) {
            const ll o = (ll)f * nn + qd * 4;
            float hi[4], lo[4], ct[4];
            stencil4<P1>(xf, n, qd * 4, hi, lo, ct);
            const Q4 bv = ld4(B + o);
            Q4 rv;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                rv.v[j] = fmaf(-c, hi[j], bv.v[j]) - c * lo[j];
                s.fma_acc(rv.v[j], rv.v[j]);
            }
            if (restart) {
                st4(R + o, rv);
                st4(P + o, rv);
            }
        }
        return (double)s.hi + (double)s.lo;
    };
    int restarts = 0;
    for (int it = 0; it < a.max_iter; ++it) {
        bool any = false;
        for (int f = 0; f < F; ++f) any |= act[f];
        if (!any) {
            // recursive residuals converged: check the true residual once
            for (int f = 0; f < F; ++f) v[f] = true_resid(f, false);
            rg = 3 * (rk++ & 1);
            block_partial(v, F, a.red, rg);
            if (!grid_sync(a.bar, a.status)) return;
            double tr[PM_MAXF];
            grid_total(a.red, F, rg, tr);
            bool again = false;
            for (int f = 0; f < F; ++f)
                if (bb[f] > 0.0 && tr[f] > tol2 * bb[f]) { act[f] = true; again = true; }
            if (!again || restarts >= 3) break;
            ++restarts;
            // restart the drifted fields from their true residual
            for (int f = 0; f < F; ++f) v[f] = act[f] ? true_resid(f, true) : 0.0;
            rg = 3 * (rk++ & 1);
            block_partial(v, F, a.red, rg);
            if (!grid_sync(a.bar, a.status)) return;
            grid_total(a.red, F, rg, w);
            for (int f = 0; f < F; ++f)
                if (act[f]) rr[f] = w[f];
        }
        // q = M p, (p, q)
        for (int f = 0; f < F; ++f) {
            v[f] = 0.0;
            if (!act[f]) continue;
            Dot2 s;
            const float *pf = P + (ll)f * nn;
            for (ll qd = tid; qd < nq; qd += nth) {
                float hi[4], lo[4], ct[4];
                stencil4<P1>(pf, n, qd * 4, hi, lo, ct);
                Q4 qv;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    qv.v[j] = fmaf(c, hi[j], c * lo[j]);
                    s.fma_acc(ct[j], qv.v[j]);
                }
                st4(Qv + (ll)f * nn + qd * 4, qv);
            }
            v[f] = (double)s.hi + (double)s.lo;
        }
        rg = 3 * (rk++ & 1);
        block_partial(v, F, a.red, rg);
        if (!grid_sync(a.bar, a.status)) return;
        grid_total(a.red, F, rg, w);
        // x += alpha p, r -= alpha q, (r, r)
        for (int f = 0; f < F; ++f) {
            v[f] = 0.0;
            if (!act[f]) continue;
            alpha[f] = rr[f] / w[f];
            const float al = (float)alpha[f];
            Dot2 s;
            for (ll qd = tid; qd < nq; qd += nth) {
                const ll o = (ll)f * nn + qd * 4;
                Q4 xv = ld4(X + o), pv = ld4(P + o), qv = ld4(Qv + o), rv = ld4(R + o);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    xv.v[j] = fmaf(al, pv.v[j], xv.v[j]);
                    rv.v[j] = fmaf(-al, qv.v[j], rv.v[j]);
                    s.fma_acc(rv.v[j], rv.v[j]);
                }
                st4(X + o, xv);
                st4(R + o, rv);
            }
            v[f] = (double)s.hi + (double)s.lo;
        }
        rg = 3 * (rk++ & 1);
        block_partial(v, F, a.red, rg);
        if (!grid_sync(a.bar, a.status)) return;
        grid_total(a.red, F, rg, w);
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
            for (ll qd = tid; qd < nq; qd += nth) {
                const ll o = (ll)f * nn + qd * 4;
                Q4 pv = ld4(P + o);
                const Q4 rv = ld4(R + o);
#pragma unroll
                for (int j = 0; j < 4; ++j) pv.v[j] = fmaf(be, pv.v[j], rv.v[j]);
                st4(P + o, pv);
            }
        }
        if (!grid_sync(a.bar, a.status)) return;
    }
    // --- report: true residual and sum of the mesh field
    for (int f = 0; f < F; ++f) {
        Dot2 s, sx;
        const float *xf = X + (ll)f * nn;
        for (ll qd = tid; qd < nq; qd += nth) {
            const ll o = (ll)f * nn + qd * 4;
            float hi[4], lo[4], ct[4];
            stencil4<P1>(xf, n, qd * 4, hi, lo, ct);
            const Q4 bv = ld4(B + o);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float rv = fmaf(-c, hi[j], bv.v[j]) - c * lo[j];
                s.fma_acc(rv, rv);
                sx.add(ct[j]);
            }
        }
        v[f] = (double)s.hi + (double)s.lo;
        w[f] = (double)sx.hi + (double)sx.lo;
    }
    rg = 3 * (rk++ & 1);
    block_partial(v, F, a.red, rg);
    block_partial(w, F, a.red, rg + 1);
    if (!grid_sync(a.bar, a.status)) return;
    double tr[PM_MAXF], sx[PM_MAXF];
    grid_total(a.red, F, rg, tr);
    grid_total(a.red, F, rg + 1, sx);
    double ps1[PM_MAXF], ps2[PM_MAXF];
    if (blockIdx.x == 0 && a.psum) particle_sums(a.psum, a.nblk_psum, F, ps1, ps2);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool bad = false;
        for (int f = 0; f < F; ++f) {
            double res = bb[f] > 0.0 ? sqrt(tr[f] / bb[f]) : 0.0;
            a.scal[f * 16 + S_ITERS] = it_f[f];
            a.scal[f * 16 + S_RESID] = res;
            a.scal[f * 16 + S_SUMMESH] = sx[f] * hd / (double)S[f];
            if (a.psum) {
                a.scal[f * 16 + S_SUMPART] = ps1[f];
                a.scal[f * 16 + S_SUMABS] = ps2[f];
            } else {
                a.scal[f * 16 + S_SUMPART] = sumb[f];
                a.scal[f * 16 + S_SUMABS] = 0.0;
            }
            if (res > a.rtol) bad = true;
        }
        if (bad) atomicOr(a.status, ST_NOTCONV);
    }
    for (int f = 0; f < F; ++f) {
        const float inv = 1.0f / S[f];  // a power of two: exact
        for (ll qd = tid; qd < nq; qd += nth) {
            const ll o = (ll)f * nn + qd * 4;
            Q4 xv = ld4(X + o);
#pragma unroll
            for (int j = 0; j < 4; ++j) xv.v[j] *= inv;
            st4(X + o, xv);
        }
    }
}

template <int DIM, int P1>
__global__ void k_mass_apply(Geo g, const float *__restrict__ x, int F, float *__restrict__ y) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const float c = DIM == 1 ? g.h / 6.0f : (P1 ? g.h * g.h / 12.0f : g.h * g.h / 36.0f);
    for (int f = 0; f < F; ++f) {
        float hi, lo;
        stencil<DIM, P1>(x + (ll)f * g.ncell, g.n, i, hi, lo);
        y[(ll)f * g.ncell + i] = fmaf(c, hi, c * lo);
    }
}

// ---------------------------------------------------------------------------
// Full-mass mesh -> particle projection (Eq. proj2): solve M_p x = c with
// (M_p)_{mu nu} = int psi_mu psi_nu, applied matrix-free from the Delaunay
// stars (2D: diagonal v/2 and, for neighbour q_k, the coefficient
// (|T_k| + |T_k+1|)/12 of the two star triangles sharing the edge; 1D: gaps g
// give g/6 (x_left + 2 x_p) and g/6 (2 x_p + x_right)). Conjugate gradients
// with the Jacobi preconditioner D (diagonal v/2 in 2D, 2v/3 in 1D), from the
// lumped start c/v, in one persistent cooperative kernel with fixed-order
// FP64 reductions. The vectors are interleaved per particle, [np][FF] with
// FF = 2, 4 or 8 >= F, so that one row of M_p gathers each neighbour's fields
// with one wide load; fields past F stay 0, and a converged field is frozen
// by zero step lengths.
//
// Two passes and two grid barriers per iteration. The kernel keeps the
// preconditioned residual z = D^-1 r instead of r (r = D z where the norms
// need it). The pass that applies M_p forms the new search direction
// p = z + beta p_prev at the row and at each neighbour it gathers (the same
// FMA at every use, so every copy has the same bits), writes p into the
// other of two direction buffers, and applies the previous iteration's
// x += alpha p_prev at its own row. The second pass updates z. The last
// x += alpha p is folded into the closing residual pass, which writes the
// solution to q.
// ---------------------------------------------------------------------------
struct PCG {
    Geo g;
    int F;
    ll np;
    const float *c, *vol;  // c: [F][np] (fields apart), vol: [np]
    const uint2 *pos;
    const int *nbr;
    const unsigned char *deg;
    const float *coef;      // [PM_MAXDEG][np] off-diagonal row coefficients (2D)
    float *x, *z, *q;       // [np][FF]: iterate, D^-1 r, M_p p (the solution at exit)
    float *p[2];            // [np][FF]: search directions of even and odd iterations
    double *red, *scal;
    unsigned *bar;
    int *status;
    double rtol;
    int max_iter;
    float unit;  // L / 2^32: torus units -> length
};

template <int FF>
struct VF {
    float v[FF];
};

template <int FF>
__device__ __forceinline__ VF<FF> ldv(const float *p) {
    VF<FF> o;
    if (FF == 2) {
        const float2 t = *(const float2 *)p;
        o.v[0] = t.x;
        o.v[1] = t.y;
    } else {
#pragma unroll
        for (int i = 0; i < FF / 4; ++i) {
            const float4 t = ((const float4 *)p)[i];
            o.v[4 * i] = t.x;
            o.v[4 * i + 1] = t.y;
            o.v[4 * i + 2] = t.z;
            o.v[4 * i + 3] = t.w;
        }
    }
    return o;
}

template <int FF>
__device__ __forceinline__ void stv(float *p, const VF<FF> &o) {
    if (FF == 2) {
        *(float2 *)p = make_float2(o.v[0], o.v[1]);
    } else {
#pragma unroll
        for (int i = 0; i < FF / 4; ++i)
            ((float4 *)p)[i] = make_float4(o.v[4 * i], o.v[4 * i + 1], o.v[4 * i + 2], o.v[4 * i + 3]);
    }
}

// Row s of M_p applied to the vector whose value at particle i is val(i),
// all FF fields at once; xs = val(s), already at hand. In 2D the star is
// walked two entries at a time, with the next pair's entries loaded while the
// current pair's neighbours are gathered; the first pair is loaded together
// with the degree (every row has PM_MAXDEG allocated slots, so these loads
// stay in bounds; entries past the degree are never used). The sums keep the
// order diagonal, slot 0, 1, ...
template <int DIM, int FF, class Val>
__device__ __forceinline__ VF<FF> pmass_row(const PCG &a, ll s, const VF<FF> &xs, Val val) {
    const ll np = a.np;
    KSum acc[FF];
    if (DIM == 1) {
        const uint32_t X = a.pos[s].x;
        const ll sl = s == 0 ? np - 1 : s - 1, sr = s + 1 == np ? 0 : s + 1;
        const float u = a.unit * (1.0f / 6.0f);
        const float gl = (float)(uint32_t)(X - a.pos[sl].x) * u, gr = (float)(uint32_t)(a.pos[sr].x - X) * u;
        const VF<FF> xl = val(sl), xr = val(sr);
#pragma unroll
        for (int f = 0; f < FF; ++f) {
            acc[f].add(gl * xl.v[f]);
            acc[f].add(2.0f * (gl + gr) * xs.v[f]);
            acc[f].add(gr * xr.v[f]);
        }
    } else {
        int e0 = a.nbr[s], e1 = a.nbr[np + s];
        float w0 = a.coef[s], w1 = a.coef[np + s];
        const int m = a.deg[s];
        const float d = 0.5f * a.vol[s];
#pragma unroll
        for (int f = 0; f < FF; ++f) acc[f].add(d * xs.v[f]);
        for (int k = 0; k < m; k += 2) {
            int n0 = 0, n1 = 0;
            float u0 = 0.0f, u1 = 0.0f;
            if (k + 2 < m) {
                n0 = a.nbr[(ll)(k + 2) * np + s];
                u0 = a.coef[(ll)(k + 2) * np + s];
            }
            if (k + 3 < m) {
                n1 = a.nbr[(ll)(k + 3) * np + s];
                u1 = a.coef[(ll)(k + 3) * np + s];
            }
            int i0 = e0 & 0x0fffffff;
            PM_CHK(i0 < np, 402, i0 = (int)s)
            const VF<FF> x0 = val(i0);
            if (k + 1 < m) {
                int i1 = e1 & 0x0fffffff;
                PM_CHK(i1 < np, 402, i1 = (int)s)
                const VF<FF> x1 = val(i1);
#pragma unroll
                for (int f = 0; f < FF; ++f) {
                    acc[f].add(w0 * x0.v[f]);
                    acc[f].add(w1 * x1.v[f]);
                }
            } else {
#pragma unroll
                for (int f = 0; f < FF; ++f) acc[f].add(w0 * x0.v[f]);
            }
            e0 = n0;
            e1 = n1;
            w0 = u0;
            w1 = u1;
        }
    }
    VF<FF> o;
#pragma unroll
    for (int f = 0; f < FF; ++f) o.v[f] = acc[f].get();
    return o;
}

// Coefficients of the particle mass matrix rows from the stars: slot k of
// particle p gets (|T_k| + |T_k+1|) / 12, T_k = (p, q_k-1, q_k), areas from
// exact 64-bit cross products of the torus coordinates.
__global__ void k_star_coef(ll np, const uint2 *__restrict__ pos, const int *__restrict__ nbr,
                            const unsigned char *__restrict__ deg, float unit, float *__restrict__ coef) {
    const ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const int m = deg[s];
    if (m < 3) return;
    const uint2 Xp = pos[s];
    const float k12 = unit * unit * (1.0f / 24.0f);  // |T|/12 = area2 unit^2 / 24
    auto rel = [&](int e, ll &rx, ll &ry) {
        const int id = e & 0x0fffffff, cd = (unsigned)e >> 28;
        rx = (ll)pos[id].x + (ll)(cd / 3 - 1) * 4294967296LL - (ll)Xp.x;
        ry = (ll)pos[id].y + (ll)(cd % 3 - 1) * 4294967296LL - (ll)Xp.y;
    };
    ll ax, ay, bx, by;
    rel(nbr[(ll)(m - 1) * np + s], ax, ay);
    float wprev = 0.0f, wfirst = 0.0f;
    for (int k = 0; k < m; ++k) {
        rel(nbr[(ll)k * np + s], bx, by);
        const float w = (float)(ax * by - ay * bx) * k12;  // triangle k = (p, q_k-1, q_k)
        if (k == 0) wfirst = w;
        else coef[(ll)(k - 1) * np + s] = wprev + w;      // edge (p, q_k-1): triangles k-1 and k
        wprev = w;
        ax = bx;
        ay = by;
    }
    coef[(ll)(m - 1) * np + s] = wprev + wfirst;           // edge (p, q_m-1): triangles m-1 and 0
}


// Block reduction of FF per-thread doubles (fields f < F) into
// red[slot*F + f][block]; the same tree and order as block_partial.
template <int FF>
__device__ __forceinline__ void block_partial_v(const double (&v)[FF], int F, double *red, int slot) {
    __shared__ double sh[FF][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < FF; ++f) {
        if (f >= F) break;
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

// grid_total into a shared array: out[f] = sum over blocks of the partials
// of (slot, f), the same order on every block. Ends with a block barrier.
__device__ __forceinline__ void grid_total_sh(const double *red, int F, int slot, double *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < F) {
        const double *src = red + (ll)(slot * F + wid) * gridDim.x;
        double s = 0;
        for (unsigned i = lane; i < gridDim.x; i += 32) s += src[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[wid] = s;
    }
    __syncthreads();
}

// Per-field solver scalars, identical on every block (each block computes
// them from the same totals); shared so that the row loops stay small.
struct PcgState {
    double cc[PM_MAXF], rz[PM_MAXF], sumc[PM_MAXF], sumabs[PM_MAXF], t0[PM_MAXF], t1[PM_MAXF];
    float al[PM_MAXF], be[PM_MAXF];
    int act[PM_MAXF], its[PM_MAXF];
};

// Compensated partials of the FF fields as doubles (fields past F give 0).
template <int FF>
__device__ __forceinline__ void dot_out(const Dot2 (&s)[FF], int F, double (&v)[FF]) {
#pragma unroll
    for (int f = 0; f < FF; ++f) v[f] = f < F ? (double)s[f].hi + (double)s[f].lo : 0.0;
}

// Reductions use slot groups {0,1,2}, {3,4}, then alternate {0} and {1,2}
// inside the loop and {5,0} at the end: no two consecutive reductions share a
// slot, so a block that runs ahead to the next reduction never overwrites a
// partial that a slower block is still summing.
template <int DIM, int FF>
__global__ void __launch_bounds__(256, FF == 8 ? 2 : 4) k_pcg(PCG a) {
    __shared__ PcgState S;
    const int F = a.F;
    const ll np = a.np;
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    const float dfac = DIM == 2 ? 0.5f : 2.0f / 3.0f;  // Jacobi diagonal = dfac v
    // --- lumped start x = c / v; (c, c), sum c, sum |c|
    {
        Dot2 s2[FF], s1[FF], sa[FF];
        for (ll s = tid; s < np; s += nth) {
            const float vv = a.vol[s];
            VF<FF> cv, xv;
#pragma unroll
            for (int f = 0; f < FF; ++f) {
                cv.v[f] = f < F ? a.c[(ll)f * np + s] : 0.0f;
                xv.v[f] = vv > 0.0f ? cv.v[f] / vv : 0.0f;
                s2[f].fma_acc(cv.v[f], cv.v[f]);
                s1[f].add(cv.v[f]);
                sa[f].add(fabsf(cv.v[f]));
            }
            stv<FF>(a.x + s * FF, xv);
        }
        double v[FF];
        dot_out<FF>(s2, F, v);
        block_partial_v<FF>(v, F, a.red, 0);
        dot_out<FF>(s1, F, v);
        block_partial_v<FF>(v, F, a.red, 1);
        dot_out<FF>(sa, F, v);
        block_partial_v<FF>(v, F, a.red, 2);
    }
    if (!grid_sync(a.bar, a.status)) return;
    grid_total_sh(a.red, F, 0, S.cc);
    grid_total_sh(a.red, F, 1, S.sumc);
    grid_total_sh(a.red, F, 2, S.sumabs);
    // --- r = c - M x, z = r / d; (r, r), (r, z)
    {
        Dot2 s2[FF], sz[FF];
        for (ll s = tid; s < np; s += nth) {
            const VF<FF> xs = ldv<FF>(a.x + s * FF);
            const VF<FF> mx = pmass_row<DIM, FF>(a, s, xs, [&](ll i) { return ldv<FF>(a.x + i * FF); });
            const float d = dfac * a.vol[s];
            VF<FF> zv;
#pragma unroll
            for (int f = 0; f < FF; ++f) {
                const float rv = (f < F ? a.c[(ll)f * np + s] : 0.0f) - mx.v[f];
                zv.v[f] = d > 0.0f ? rv / d : 0.0f;
                s2[f].fma_acc(rv, rv);
                sz[f].fma_acc(rv, zv.v[f]);
            }
            stv<FF>(a.z + s * FF, zv);
        }
        double v[FF];
        dot_out<FF>(s2, F, v);
        block_partial_v<FF>(v, F, a.red, 3);
        dot_out<FF>(sz, F, v);
        block_partial_v<FF>(v, F, a.red, 4);
    }
    if (!grid_sync(a.bar, a.status)) return;
    grid_total_sh(a.red, F, 3, S.t0);
    grid_total_sh(a.red, F, 4, S.rz);
    // The iteration stops on its recurrence for (r, r), which in FP32 drifts
    // from the true residual by a few roundings (observed: under 1 %); it
    // stops at 0.9 rtol so that the true residual, recomputed at exit, meets
    // rtol.
    const double tol2 = 0.81 * a.rtol * a.rtol;
    if (threadIdx.x == 0)
        for (int f = 0; f < F; ++f) {
            S.act[f] = S.cc[f] > 0.0 && S.t0[f] > tol2 * S.cc[f];
            S.its[f] = 0;
            S.al[f] = 0.0f;
            S.be[f] = 0.0f;
            if (blockIdx.x == 0) a.scal[f * 16 + S_INIT] = S.cc[f] > 0.0 ? sqrt(S.t0[f] / S.cc[f]) : 0.0;
        }
    __syncthreads();
    int last = -1;  // the last iteration run: its alpha p is still to be added to x
    for (int it = 0; it < a.max_iter; ++it) {
        bool any = false;
        for (int f = 0; f < F; ++f) any |= S.act[f] != 0;
        if (!any) break;
        // p = z + beta p_prev (at the row and at each neighbour), q = M p,
        // (p, q); x += alpha_prev p_prev at the row
        const float *pin = a.p[(it + 1) & 1];
        float *pout = a.p[it & 1];
        float be[FF], ap[FF];
#pragma unroll
        for (int f = 0; f < FF; ++f) {
            be[f] = f < F ? S.be[f] : 0.0f;
            ap[f] = f < F ? S.al[f] : 0.0f;
        }
        const bool first = it == 0;
        {
            auto pval = [&](ll i) {
                VF<FF> zv = ldv<FF>(a.z + i * FF);
                if (!first) {
                    const VF<FF> pv = ldv<FF>(pin + i * FF);
#pragma unroll
                    for (int f = 0; f < FF; ++f) zv.v[f] = fmaf(be[f], pv.v[f], zv.v[f]);
                }
                return zv;
            };
            Dot2 sq[FF];
            for (ll s = tid; s < np; s += nth) {
                VF<FF> ps = ldv<FF>(a.z + s * FF);
                if (!first) {
                    const VF<FF> pv = ldv<FF>(pin + s * FF);
                    VF<FF> xv = ldv<FF>(a.x + s * FF);
#pragma unroll
                    for (int f = 0; f < FF; ++f) {
                        ps.v[f] = fmaf(be[f], pv.v[f], ps.v[f]);
                        xv.v[f] = fmaf(ap[f], pv.v[f], xv.v[f]);
                    }
                    stv<FF>(a.x + s * FF, xv);
                }
                const VF<FF> qv = pmass_row<DIM, FF>(a, s, ps, pval);
                stv<FF>(pout + s * FF, ps);
                stv<FF>(a.q + s * FF, qv);
#pragma unroll
                for (int f = 0; f < FF; ++f) sq[f].fma_acc(ps.v[f], qv.v[f]);
            }
            double v[FF];
            dot_out<FF>(sq, F, v);
            block_partial_v<FF>(v, F, a.red, 0);
        }
        if (!grid_sync(a.bar, a.status)) return;
        grid_total_sh(a.red, F, 0, S.t0);
        if (threadIdx.x == 0)
            for (int f = 0; f < F; ++f) S.al[f] = S.act[f] ? (float)(S.rz[f] / S.t0[f]) : 0.0f;
        __syncthreads();
        last = it;
        // z -= alpha q / d; (r, r) and (r, z) with r = d z
        {
            float al[FF];
#pragma unroll
            for (int f = 0; f < FF; ++f) al[f] = f < F ? S.al[f] : 0.0f;
            Dot2 s2[FF], sz[FF];
            for (ll s = tid; s < np; s += nth) {
                VF<FF> zv = ldv<FF>(a.z + s * FF);
                const VF<FF> qv = ldv<FF>(a.q + s * FF);
                const float d = dfac * a.vol[s];
#pragma unroll
                for (int f = 0; f < FF; ++f) {
                    zv.v[f] = d > 0.0f ? fmaf(-al[f], qv.v[f] / d, zv.v[f]) : 0.0f;
                    const float rv = d * zv.v[f];
                    s2[f].fma_acc(rv, rv);
                    sz[f].fma_acc(rv, zv.v[f]);
                }
                stv<FF>(a.z + s * FF, zv);
            }
            double v[FF];
            dot_out<FF>(s2, F, v);
            block_partial_v<FF>(v, F, a.red, 1);
            dot_out<FF>(sz, F, v);
            block_partial_v<FF>(v, F, a.red, 2);
        }
        if (!grid_sync(a.bar, a.status)) return;
        grid_total_sh(a.red, F, 1, S.t0);
        grid_total_sh(a.red, F, 2, S.t1);
        if (threadIdx.x == 0)
            for (int f = 0; f < F; ++f) {
                S.be[f] = 0.0f;
                if (!S.act[f]) continue;
                S.be[f] = (float)(S.t1[f] / S.rz[f]);
                S.rz[f] = S.t1[f];
                ++S.its[f];
                if (S.t0[f] <= tol2 * S.cc[f]) S.act[f] = 0;
            }
        __syncthreads();
    }
    // --- report: x += alpha p of the last iteration (at the row and at each
    // neighbour), true residual c - M x, sum v x (= sum c for the exact
    // solution); the solution goes to q
    {
        float ap[FF];
#pragma unroll
        for (int f = 0; f < FF; ++f) ap[f] = (f < F && last >= 0) ? S.al[f] : 0.0f;
        const float *pl = a.p[(last >= 0 ? last : 0) & 1];
        const bool pend = last >= 0;
        auto xval = [&](ll i) {
            VF<FF> xv = ldv<FF>(a.x + i * FF);
            if (pend) {
                const VF<FF> pv = ldv<FF>(pl + i * FF);
#pragma unroll
                for (int f = 0; f < FF; ++f) xv.v[f] = fmaf(ap[f], pv.v[f], xv.v[f]);
            }
            return xv;
        };
        Dot2 s2[FF], sv[FF];
        for (ll s = tid; s < np; s += nth) {
            const VF<FF> xs = xval(s);
            const VF<FF> mx = pmass_row<DIM, FF>(a, s, xs, xval);
            const float vv = a.vol[s];
#pragma unroll
            for (int f = 0; f < FF; ++f) {
                const float rv = (f < F ? a.c[(ll)f * np + s] : 0.0f) - mx.v[f];
                s2[f].fma_acc(rv, rv);
                sv[f].fma_acc(vv, xs.v[f]);
            }
            stv<FF>(a.q + s * FF, xs);
        }
        double v[FF];
        dot_out<FF>(s2, F, v);
        block_partial_v<FF>(v, F, a.red, 5);
        dot_out<FF>(sv, F, v);
        block_partial_v<FF>(v, F, a.red, 0);
    }
    if (!grid_sync(a.bar, a.status)) return;
    grid_total_sh(a.red, F, 5, S.t0);
    grid_total_sh(a.red, F, 0, S.t1);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool bad = false;
        for (int f = 0; f < F; ++f) {
            const double res = S.cc[f] > 0.0 ? sqrt(S.t0[f] / S.cc[f]) : 0.0;
            a.scal[f * 16 + S_ITERS] = S.its[f];
            a.scal[f * 16 + S_RESID] = res;
            a.scal[f * 16 + S_SUMMESH] = S.sumc[f];   // int Ab = sum_mu c_mu
            a.scal[f * 16 + S_SUMPART] = S.t1[f];     // sum_mu v_mu Abb_mu
            a.scal[f * 16 + S_SUMABS] = S.sumabs[f];  // sum_mu |c_mu|: scale of the conservation error
            if (res > a.rtol) bad = true;
        }
        if (bad) atomicOr(a.status, ST_NOTCONV);
    }
}

// Interleaved solution [np][FF] -> caller order [F][np], one field per grid
// row: the rows run one after another, so the scattered writes of a row stay
// within one field's array, which the L2 holds and merges before writing back.
__global__ void k_unsort_aos(ll np, int FF, const int *__restrict__ perm, const float *__restrict__ x,
                             float *__restrict__ out) {
    const ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const int f = blockIdx.y;
    out[(ll)f * np + perm[s]] = x[s * FF + f];
}

// Resident blocks of a persistent kernel: SMs x min(occupancy, cap), looked
// up once per (device, kernel variant) and cached. The cache is keyed by the
// current device and guarded, so threads driving different devices each get
// their own device's figure.
#define PM_GRID_MAXDEV 64
std::mutex g_grid_mu;
int g_grid_cache[PM_GRID_MAXDEV][16];

int persistent_grid(int variant, const void *kern, int cap) {
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < PM_GRID_MAXDEV;
    if (cached) {
        std::lock_guard<std::mutex> lk(g_grid_mu);
        if (g_grid_cache[dev][variant]) return g_grid_cache[dev][variant];
    }
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0);
    if (per < 1) per = 1;
    if (per > cap) per = cap;
    const int grid = sms * per;
    if (cached) {
        std::lock_guard<std::mutex> lk(g_grid_mu);
        g_grid_cache[dev][variant] = grid;
    }
    return grid;
}

// The reduction partials hold w.red_blocks blocks per slot: never launch more.
int clamp_grid(int grid, ll need, const Work &w) {
    if (need < grid) grid = (int)(need < 1 ? 1 : need);
    if (w.red_blocks > 0 && grid > w.red_blocks) grid = w.red_blocks;
    return grid;
}

}  // namespace

void launch_mass_apply(const Geo &g, const float *x, int F, float *y, cudaStream_t st) {
    if (g.dim == 1)
        k_mass_apply<1, 0><<<div_up(g.ncell, 256), 256, 0, st>>>(g, x, F, y);
    else
        if (g.p1)
            k_mass_apply<2, 1><<<div_up(g.ncell, 256), 256, 0, st>>>(g, x, F, y);
        else
            k_mass_apply<2, 0><<<div_up(g.ncell, 256), 256, 0, st>>>(g, x, F, y);
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
    // 2D meshes with n % 4 == 0 take the quad kernel (16-byte accesses)
    const bool quad = g.dim == 2 && g.n % 4 == 0, p1 = g.dim == 2 && g.p1;
    const int di = (quad ? 2 : g.dim - 1) + (p1 ? 3 : 0);
    void (*kern)(CG) = quad ? (p1 ? k_cg2v<1> : k_cg2v<0>)
                            : (g.dim == 1 ? k_cg<1, 0> : (p1 ? k_cg<2, 1> : k_cg<2, 0>));
    const ll need = ((quad ? g.ncell / 4 : g.ncell) + 255) / 256;
    const int grid = clamp_grid(persistent_grid(di, (const void *)kern, quad ? 4 : 2), need, w);
    cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st);
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(256), args, 0, st);
    count_launches(1);
    return (int)e;
}

// Chebyshev solve: same arguments, workspace and report as launch_cg.

int launch_cheb(const Geo &g, Work &w, int F, const float *b_float, bool b_from_fix, float *x, bool x_has_start,
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
    a.r2 = w.r2;
    a.red = w.red;
    a.scal = w.scal;
    a.bar = w.bar;
    a.status = w.status;
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.has_start = x_has_start ? 1 : 0;
    a.psum = b_from_fix ? w.psum : nullptr;
    a.nblk_psum = w.nblk_psum;
    const bool p1 = g.dim == 2 && g.p1;
    const int di = g.dim == 1 ? 0 : (p1 ? 2 : 1);
    if (g.dim == 2 && !w.r2) return (int)cudaErrorInvalidValue;
    void (*kern)(CG) = g.dim == 1 ? k_cheb<1, 0> : (p1 ? k_cheb<2, 1> : k_cheb<2, 0>);
    const ll need = (g.ncell + 255) / 256;
    const int grid = clamp_grid(persistent_grid(6 + di, (const void *)kern, 4), need, w);
    cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st);
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(256), args, 0, st);
    count_launches(1);
    return (int)e;
}

int pcg_width(int F) { return F <= 2 ? 2 : (F <= 4 ? 4 : PM_MAXF); }

int launch_pcg(const Geo &g, Work &w, ll np, int F, const float *c, float *out, double rtol, int max_iter,
               cudaStream_t st) {
    const int FF = pcg_width(F);
    PCG a;
    a.g = g;
    a.F = F;
    a.np = np;
    a.c = c;
    a.vol = w.vol;
    a.pos = w.pos;
    a.nbr = w.nbr;
    a.deg = w.deg;
    a.coef = w.pcoef;
    a.x = w.px;
    a.z = w.prp;
    a.p[0] = w.prp + (ll)pcg_width(w.F_max) * w.np_max;
    a.p[1] = w.pp2;
    a.q = w.pq;
    a.red = w.red;
    a.scal = w.scal;
    a.bar = w.bar;
    a.status = w.status;
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.unit = (float)(g.L / 4294967296.0);
    const int fi = FF == 2 ? 0 : (FF == 4 ? 1 : 2);
    const int di = (g.dim - 1) * 3 + fi;
    void (*const kerns[6])(PCG) = {k_pcg<1, 2>, k_pcg<1, 4>, k_pcg<1, PM_MAXF>,
                                   k_pcg<2, 2>, k_pcg<2, 4>, k_pcg<2, PM_MAXF>};
    void (*kern)(PCG) = kerns[di];
    const ll need = (np + 255) / 256;
    const int grid = clamp_grid(persistent_grid(9 + di, (const void *)kern, 4), need, w);
    if (g.dim == 2 && np > 0) {
        k_star_coef<<<div_up(np, 256), 256, 0, st>>>(np, w.pos, w.nbr, w.deg, a.unit, w.pcoef);
        count_launches(1);
    }
    cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st);
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(256), args, 0, st);
    count_launches(1);
    if (e != cudaSuccess) return (int)e;
    if (np > 0) {
        k_unsort_aos<<<dim3((unsigned)div_up(np, 256), F), 256, 0, st>>>(np, FF, w.perm, w.pq, out);
        count_launches(1);
    }
    return 0;
}
