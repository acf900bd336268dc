// Direct solve of the mesh mass system M Ab = b (Sec. 2.4, Eq. phi_def) on
// the uniform periodic mesh. The 1D mass matrix is M1 = (h/6) circ(1, 4, 1)
// and the bilinear 2D one is M1 (x) M1, so M^-1 = M1^-1 (x) M1^-1 applies as
// two separable convolutions. The inverse of circ(1, 4, 1) on n points is the
// circulant with entries f(j) = (r^j + r^(n-j)) / ((1 - r^n) sqrt 12),
// j = 0..n-1, r = sqrt 3 - 2 (the root of r^2 + 4 r + 1 = 0 inside the unit
// circle): f solves f(j-1) + 4 f(j) + f(j+1) = delta_j0 with periodic ends.
// |r| < 0.268, so offsets beyond 16 weigh below 2e-10 and are dropped on
// meshes with n > 33; smaller meshes take every offset. Each pass stages a
// tile with its halo in shared memory. Every tap is carried as a float pair
// (hi + lo = the double weight to ~2^-48) and the sum is compensated (Dot2):
// with single float taps the rounding of the weights perturbs the operator's
// low-frequency symbol by ~1e-7 in one direction, a bias that a long chain of
// assignments (a 256-step transport) accumulates step after step.
#include <math.h>
#include <string.h>

#include "internal.cuh"

namespace {

#define DT 32      // tile side (outputs)
#define DK 16      // largest offset kept
#define DMAXT 40   // tap capacity (n <= 33 uses n taps)

struct Taps {
    int nt;             // number of taps
    int off[DMAXT];     // offsets along the direction (distinct mod n)
    float w[DMAXT];     // weights f(offset mod n) times the scale (rounded)
    float wl[DMAXT];    // the weights' rounding remainders
    int halo;           // largest |offset|
};

// One pass along x (DIR 0) or y (DIR 1) of one field over the tile at
// (x0, y0): d = taps * s (s, d the field's n x n arrays).
template <int DIR>
__device__ __forceinline__ void circ_tile(int n, const float *__restrict__ s, float *__restrict__ d, const Taps &t,
                                          int x0, int y0) {
    __shared__ float tile[DT + 2 * DK][DT + 1];  // halo <= DK on every mesh
    const int H = t.halo;
    // stage: along the pass direction the tile is DT + 2H long
    for (int i = threadIdx.x; i < (DT + 2 * H) * DT; i += blockDim.x) {
        const int a = i / DT, b = i % DT;  // a along the pass direction, b across
        int x, y;
        if (DIR == 0) { x = x0 + a - H; y = y0 + b; }
        else { x = x0 + b; y = y0 + a - H; }
        x = ((x % n) + n) % n;
        y = ((y % n) + n) % n;
        tile[a][b] = __ldg(s + (ll)y * n + x);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < DT * DT; i += blockDim.x) {
        const int a = i / DT, b = i % DT;
        int x, y;
        if (DIR == 0) { x = x0 + a; y = y0 + b; }
        else { x = x0 + b; y = y0 + a; }
        if (x >= n || y >= n) continue;
        Dot2 acc;
        float lo = 0.0f;
        for (int k = 0; k < t.nt; ++k) {
            const float v = tile[a + H + t.off[k]][b];
            acc.fma_acc(t.w[k], v);
            lo = fmaf(t.wl[k], v, lo);
        }
        d[(ll)y * n + x] = acc.hi + (acc.lo + lo);
    }
}

template <int DIR>
__global__ void __launch_bounds__(256) k_circ(int n, int F, const float *__restrict__ src, float *__restrict__ dst,
                                              Taps t) {
    const int tiles = (n + DT - 1) / DT;
    const ll nn = (ll)n * n;
    const int f = blockIdx.y;
    circ_tile<DIR>(n, src + (ll)f * nn, dst + (ll)f * nn, t, (blockIdx.x % tiles) * DT, (blockIdx.x / tiles) * DT);
}

// Batched: block b is tile b - tile_start[k] of instance k (taps[k] staged in
// shared memory); fields are [F][NC] packed arrays.
template <int DIR>
__global__ void __launch_bounds__(256) k_circ_b(BTab bt, const Taps *__restrict__ taps, const int *__restrict__ tile_start,
                                                const float *__restrict__ src, float *__restrict__ dst) {
    __shared__ Taps st;
    const int k = find_slot(tile_start, bt.ninst, (int)blockIdx.x);
    for (int i = threadIdx.x; i < (int)(sizeof(Taps) / 4); i += blockDim.x)
        ((int *)&st)[i] = ((const int *)(taps + k))[i];
    __syncthreads();
    const int n = bt.inst[k].n, tiles = (n + DT - 1) / DT, tl = (int)blockIdx.x - __ldg(tile_start + k);
    const ll off = (ll)blockIdx.y * bt.NC + __ldg(bt.coff + k);
    circ_tile<DIR>(n, src + off, dst + off, st, (tl % tiles) * DT, (tl / tiles) * DT);
}

__global__ void __launch_bounds__(256) k_circ1(int n, int F, const float *__restrict__ src, float *__restrict__ dst,
                                               Taps t) {
    const ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (ll)n * F) return;
    const int f = (int)(i / n), x = (int)(i % n);
    Dot2 acc;
    float lo = 0.0f;
    for (int k = 0; k < t.nt; ++k) {
        const float v = __ldg(src + (ll)f * n + (((x + t.off[k]) % n) + n) % n);
        acc.fma_acc(t.w[k], v);
        lo = fmaf(t.wl[k], v, lo);
    }
    dst[i] = acc.hi + (acc.lo + lo);
}

Taps make_taps(int n, double scale) {
    Taps t;
    const double r = sqrt(3.0) - 2.0, rn = pow(r, n), c = 1.0 / ((1.0 - rn) * sqrt(12.0));
    auto f = [&](int j) { return (pow(r, j) + pow(r, n - j)) * c; };
    t.nt = 0;
    if (n > 2 * DK + 1) {
        for (int j = -DK; j <= DK; ++j) {
            const double wd = scale * f(j < 0 ? -j : j);
            t.off[t.nt] = j;
            t.w[t.nt] = (float)wd;
            t.wl[t.nt] = (float)(wd - (double)t.w[t.nt]);
            ++t.nt;
        }
        t.halo = DK;
    } else {
        // every residue once, offsets in (-n/2, n/2]
        for (int j = -((n - 1) / 2); j <= n / 2; ++j) {
            const double wd = scale * f(((j % n) + n) % n);
            t.off[t.nt] = j;
            t.w[t.nt] = (float)wd;
            t.wl[t.nt] = (float)(wd - (double)t.w[t.nt]);
            ++t.nt;
        }
        t.halo = n / 2;
    }
    return t;
}

}  // namespace

size_t direct_taps_bytes() { return sizeof(Taps); }
void make_direct_taps(int n, double L, void *out) {
    const Taps t = make_taps(n, 6.0 / (L / n));
    memcpy(out, &t, sizeof(Taps));
}
int direct_tile_count(int n) {
    const int tiles = (n + DT - 1) / DT;
    return tiles * tiles;
}

void launch_mass_direct_batched(const BTab &t, const void *taps, const int *tile_start, int ntiles, const float *b,
                                int F, float *x, float *tmp, cudaStream_t st) {
    dim3 grid(ntiles, F);
    k_circ_b<0><<<grid, 256, 0, st>>>(t, (const Taps *)taps, tile_start, b, tmp);
    k_circ_b<1><<<grid, 256, 0, st>>>(t, (const Taps *)taps, tile_start, tmp, x);
    count_launches(2);
}

// x = M^-1 b for F fields (b, x device [F][n^dim]; tmp [F][n^dim] scratch).
void launch_mass_direct(const Geo &g, const float *b, int F, float *x, float *tmp, cudaStream_t st) {
    const int n = g.n;
    if (g.dim == 1) {
        const Taps t = make_taps(n, 6.0 / ((double)g.L / n));
        k_circ1<<<div_up((ll)n * F, 256), 256, 0, st>>>(n, F, b, x, t);
        count_launches(1);
        return;
    }
    const double h = (double)g.L / n;
    const Taps tx = make_taps(n, 6.0 / h), ty = make_taps(n, 6.0 / h);
    const int tiles = (n + DT - 1) / DT;
    dim3 grid(tiles * tiles, F);
    k_circ<0><<<grid, 256, 0, st>>>(n, F, b, tmp, tx);
    k_circ<1><<<grid, 256, 0, st>>>(n, F, tmp, x, ty);
    count_launches(2);
}
