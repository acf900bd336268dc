// Mesh -> particle interpolation, Sec. 2.2 Eq. delta2:
//   Abb_mu = sum_i Ab_i psi_i(r_mu),
// psi_i linear (1D) / bilinear or P1 on split cells (2D). Only the 2^dim nodes of the particle's
// cell contribute. One thread per particle in caller order: positions and
// outputs stream coalesced; the mesh (a few MB to tens of MB per field) is
// read through L1/L2, where the four corner loads of neighbouring particles
// hit the same lines.
#include "internal.cuh"

namespace {

template <int DIM>
__global__ void __launch_bounds__(256) k_g2p(Geo g, const float *__restrict__ mesh, int F,
                                             const float *__restrict__ px, const float *__restrict__ py, ll np,
                                             float *__restrict__ out, int *__restrict__ status) {
    ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    float x = px[k];
    float y = DIM == 2 ? py[k] : 0.0f;
    if (!isfinite(x) || !isfinite(y)) {
        atomicOr(status, ST_NONFINITE);
        x = 0.0f;
        y = 0.0f;
    }
    const int n = g.n;
    uint32_t X = torus_coord(x, g.invL);
    int cx = cell_of(X, n);
    float s = frac_f(X, n);
    int x1 = cx + 1 == n ? 0 : cx + 1;
    if (DIM == 1) {
        for (int f = 0; f < F; ++f) {
            const float *m = mesh + (ll)f * n;
            out[(ll)f * np + k] = fmaf(s, __ldg(m + x1), (1.0f - s) * __ldg(m + cx));
        }
        return;
    }
    uint32_t Y = torus_coord(y, g.invL);
    int cy = cell_of(Y, n);
    float t = frac_f(Y, n);
    int y1 = cy + 1 == n ? 0 : cy + 1;
    const ll i00 = (ll)cy * n + cx, i10 = (ll)cy * n + x1, i01 = (ll)y1 * n + cx, i11 = (ll)y1 * n + x1;
    float w00, w10, w01, w11;
    cell_weights(g.p1 != 0, s, t, w00, w10, w01, w11);
    const ll nn = g.ncell;
    for (int f = 0; f < F; ++f) {
        const float *m = mesh + (ll)f * nn;
        float v = w00 * __ldg(m + i00);
        v = fmaf(w10, __ldg(m + i10), v);
        v = fmaf(w01, __ldg(m + i01), v);
        v = fmaf(w11, __ldg(m + i11), v);
        out[(ll)f * np + k] = v;
    }
}

__global__ void k_unsort(ll np, const int *__restrict__ perm, const float *__restrict__ src, float *__restrict__ dst) {
    ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < np) dst[perm[s]] = src[s];
}

}  // namespace

void launch_g2p(const Geo &g, const float *mesh, int F, const float *px, const float *py, ll np, float *out,
                int *status, cudaStream_t st) {
    if (np <= 0) return;
    if (g.dim == 1)
        k_g2p<1><<<div_up(np, 256), 256, 0, st>>>(g, mesh, F, px, py, np, out, status);
    else
        k_g2p<2><<<div_up(np, 256), 256, 0, st>>>(g, mesh, F, px, py, np, out, status);
    count_launches(1);
}

void launch_scatter_sorted(ll np, const int *perm, const float *src, float *dst, cudaStream_t st) {
    if (np > 0) {
        k_unsort<<<div_up(np, 256), 256, 0, st>>>(np, perm, src, dst);
        count_launches(1);
    }
}
