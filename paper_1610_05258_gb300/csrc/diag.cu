// Stability diagnostics of a transfer (Sec. 2.1, Eq. stab, read in integral
// form): the integral of the squared field on each side,
//
//   mesh:      int Ab^2 = Ab^T M Ab,      m_ij = int psi_i psi_j   (Sec. 2.4)
//   particles: int A^2  = A^T M_p A,      (M_p)_{mu nu} = int psi_mu psi_nu
//
// The L2 projections (mass assignment, full-mass interpolation) are
// contractions, so the side they produce never holds more of this integral
// than the side they start from.
//
// Particle side: P1 functions on the periodic Delaunay triangulation (2D),
// where int_T A^2 = |T| / 6 (a^2 + b^2 + c^2 + ab + bc + ca) for a triangle T
// with vertex values a, b, c; hats on the ordered particles (1D), where an
// interval of length l with end values a, b gives l / 3 (a^2 + ab + b^2).
// Each triangle is counted once, by its lowest sorted vertex (the delta
// assignment's ownership rule). Per-thread sums are compensated FP32,
// block and grid totals FP64 in a fixed order.
#include "internal.cuh"

namespace {

constexpr int kBlocks = 4 * 152;
constexpr int kThreads = 256;

// Block partial of one double per field into part[slot][blockIdx.x].
__device__ void block_partials(double v[PM_MAXF], int F, double *part, int nblk) {
    __shared__ double sh[PM_MAXF][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int f = 0; f < F; ++f) {
        double s = v[f];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh[f][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < F) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[threadIdx.x][w];
        part[(ll)threadIdx.x * nblk + blockIdx.x] = s;
    }
}

// Ab^T M Ab without the stencil's constant factor.
template <int DIM, int P1>
__global__ void __launch_bounds__(kThreads) k_energy_mesh(Geo g, int F, const float *__restrict__ x,
                                                         double *__restrict__ part) {
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    double v[PM_MAXF];
    for (int f = 0; f < F; ++f) {
        const float *xf = x + (ll)f * g.ncell;
        Dot2 acc;
        for (ll i = tid; i < g.ncell; i += nth) {
            float hi, lo;
            stencil<DIM, P1>(xf, g.n, i, hi, lo);
            acc.fma_acc(xf[i], hi);
            acc.fma_acc(xf[i], lo);
        }
        v[f] = (double)acc.hi + (double)acc.lo;
    }
    block_partials(v, F, part, gridDim.x);
}

// A^T M_p A over the owned triangles of every sorted particle, in units of
// the torus coordinate squared (the caller scales by (L / 2^32)^2 / 12).
// Value of field f at sorted particle s: vals[f * fs + s * ss].
__global__ void __launch_bounds__(kThreads) k_energy_tris(ll np, const uint2 *__restrict__ pos,
                                                         const int *__restrict__ nbr,
                                                         const unsigned char *__restrict__ deg,
                                                         const float *__restrict__ vals, ll fs, ll ss, int F,
                                                         double *__restrict__ part) {
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    Dot2 acc[PM_MAXF];
    for (ll pl = tid; pl < np; pl += nth) {
        const int p = (int)pl, m = deg[p];
        if (m < 3) continue;
        const uint2 Xp = pos[p];
        auto rel = [&](int e, int &id, ll &rx, ll &ry) {
            id = e & 0x0fffffff;
            const int c = (unsigned)e >> 28, ox = c / 3 - 1, oy = c % 3 - 1;
            const uint2 Xq = pos[id];
            rx = (ll)Xq.x + (ll)ox * 4294967296LL - (ll)Xp.x;
            ry = (ll)Xq.y + (ll)oy * 4294967296LL - (ll)Xp.y;
        };
        int ida;
        ll ax, ay;
        rel(nbr[(ll)(m - 1) * np + p], ida, ax, ay);
        for (int k = 0; k < m; ++k) {
            int idb;
            ll bx, by;
            rel(nbr[(ll)k * np + p], idb, bx, by);
            if (ida > p && idb > p) {
                // twice the area in torus units^2 (exact: |.| < 2^61), scaled by 2^-64
                const float w2 = (float)(ax * by - ay * bx) * 5.421010862427522e-20f;
                for (int f = 0; f < F; ++f) {
                    const float a = vals[f * fs + (ll)p * ss], b = vals[f * fs + (ll)ida * ss],
                                c = vals[f * fs + (ll)idb * ss];
                    const float q = a * a + b * b + c * c + a * b + b * c + c * a;
                    acc[f].fma_acc(w2, q);
                }
            }
            ida = idb;
            ax = bx;
            ay = by;
        }
    }
    double v[PM_MAXF];
    for (int f = 0; f < F; ++f) v[f] = (double)acc[f].hi + (double)acc[f].lo;
    block_partials(v, F, part, gridDim.x);
}

// 1D: interval from sorted particle s to the next one around the circle, in
// torus units scaled by 2^-32 (the caller scales by L / 3).
__global__ void __launch_bounds__(kThreads) k_energy_1d(ll np, const uint2 *__restrict__ pos,
                                                       const float *__restrict__ vals, ll fs, ll ss, int F,
                                                       double *__restrict__ part) {
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    Dot2 acc[PM_MAXF];
    for (ll s = tid; s < np; s += nth) {
        const ll s1 = s + 1 < np ? s + 1 : 0;
        const uint32_t d = pos[s1].x - pos[s].x;  // modulo 2^32: the gap around the circle
        const float l = np == 1 ? 1.0f : (float)d * 2.3283064365386963e-10f;
        for (int f = 0; f < F; ++f) {
            const float a = vals[f * fs + s * ss], b = vals[f * fs + s1 * ss];
            acc[f].fma_acc(l, a * a + a * b + b * b);
        }
    }
    double v[PM_MAXF];
    for (int f = 0; f < F; ++f) v[f] = (double)acc[f].hi + (double)acc[f].lo;
    block_partials(v, F, part, gridDim.x);
}

// Totals in a fixed order (warp k sums row k), scaled, into the report slots.
__global__ void k_energy_final(int F, const double *__restrict__ part, int nblk, double cm, double cp, int has_part,
                               double *__restrict__ scal) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = wid; k < 2 * F; k += (int)(blockDim.x >> 5)) {
        const bool mesh_row = k < F;
        double s = 0.0;
        if (mesh_row || has_part) {
            const double *src = part + (ll)k * nblk;
            for (int i = lane; i < nblk; i += 32) s += src[i];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (lane == 0) {
            if (mesh_row)
                scal[16 * k + 6] = s * cm;
            else
                scal[16 * (k - F) + 7] = has_part ? s * cp : 0.0;
        }
    }
}

}  // namespace

int energy_blocks() { return kBlocks; }

void launch_energies(const Geo &g, Work &w, int F, const float *mesh, ll np, const float *pvals, ll fs, ll ss,
                     cudaStream_t st) {
    double *part = w.epart;
    const double h = g.L / g.n;
    double cm;
    if (g.dim == 1) {
        cm = h / 6.0;
        k_energy_mesh<1, 0><<<kBlocks, kThreads, 0, st>>>(g, F, mesh, part);
    } else if (g.p1) {
        cm = h * h / 12.0;
        k_energy_mesh<2, 1><<<kBlocks, kThreads, 0, st>>>(g, F, mesh, part);
    } else {
        cm = h * h / 36.0;
        k_energy_mesh<2, 0><<<kBlocks, kThreads, 0, st>>>(g, F, mesh, part);
    }
    int k = 1;
    const bool has_part = pvals != nullptr && np > 0;
    double cp = 0.0;
    if (has_part) {
        if (g.dim == 1) {
            cp = g.L / 3.0;
            k_energy_1d<<<kBlocks, kThreads, 0, st>>>(np, w.pos, pvals, fs, ss, F, part + (ll)F * kBlocks);
        } else {
            cp = g.L * g.L / 12.0;  // (2 |T| / L^2) 2^-64 scaled back: |T| / 6 = (2|T|) / 12
            k_energy_tris<<<kBlocks, kThreads, 0, st>>>(np, w.pos, w.nbr, w.deg, pvals, fs, ss, F,
                                                       part + (ll)F * kBlocks);
        }
        ++k;
    }
    k_energy_final<<<1, 512, 0, st>>>(F, part, kBlocks, cm, cp, has_part ? 1 : 0, w.scal);
    count_launches(k + 1);
}
