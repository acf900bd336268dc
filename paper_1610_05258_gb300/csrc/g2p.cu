// Mesh -> particle interpolation, Sec. 2.2 Eq. delta2:
//   Abb_mu = sum_i Ab_i psi_i(r_mu),
// psi_i linear (1D) / bilinear or P1 on split cells (2D). Only the 2^dim
// nodes of the particle's cell contribute.
//
// Particles come in the caller's order, which is arbitrary, so the mesh is
// read by gathers. The mesh of a benchmark-sized problem (2048^2 nodes x 4
// fields = 67 MB) fits in the 129 MB L2, so the design keeps it there and
// makes every gather cheap:
//  * the F fields are first interleaved per node ([n^dim][W] with W = 1, 2, 4
//    or 8 >= F, one coalesced pass), so the two corners of a cell row are one
//    contiguous 2W-float read instead of F separate ones;
//  * positions are loaded and results stored with streaming (evict-first)
//    accesses, so the particle streams do not push the mesh out of L2.
// One thread per particle; the arithmetic (weights, FMA order) is the same
// for every layout.
#include "internal.cuh"

namespace {

template <int W>
struct NodeVec {
    float v[W];
};

template <int W>
__device__ __forceinline__ NodeVec<W> load_node(const float *__restrict__ il, ll i) {
    NodeVec<W> r;
    const float *p = il + i * W;
    if (W == 1) {
        r.v[0] = __ldg(p);
    } else if (W == 2) {
        const float2 a = __ldg((const float2 *)p);
        r.v[0] = a.x;
        r.v[1] = a.y;
    } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q) {
            const float4 a = __ldg((const float4 *)p + q);
            r.v[4 * q] = a.x;
            r.v[4 * q + 1] = a.y;
            r.v[4 * q + 2] = a.z;
            r.v[4 * q + 3] = a.w;
        }
    }
    return r;
}

// mesh [F][nn] -> il [nn][W] (fields beyond F padded with zeros).
template <int W>
__global__ void __launch_bounds__(256) k_interleave(ll nn, int F, const float *__restrict__ mesh,
                                                   float *__restrict__ il) {
    const ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    float v[W];
#pragma unroll
    for (int f = 0; f < W; ++f) v[f] = f < F ? __ldcs(mesh + (ll)f * nn + i) : 0.0f;
    if (W == 2) {
        ((float2 *)il)[i] = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
            ((float4 *)il)[i * (W / 4) + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

// il: the mesh fields interleaved per node, [nn][W] (W = 1: the caller's
// single field as it is).
template <int DIM, int W>
__global__ void __launch_bounds__(256) k_g2p(Geo g, const float *__restrict__ il, int F,
                                             const float *__restrict__ px, const float *__restrict__ py, ll np,
                                             float *__restrict__ out, int *__restrict__ status) {
    ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    float x = __ldcs(px + k);
    float y = DIM == 2 ? __ldcs(py + k) : 0.0f;
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
        const NodeVec<W> m0 = load_node<W>(il, cx), m1 = load_node<W>(il, x1);
#pragma unroll
        for (int f = 0; f < W; ++f)
            if (f < F) __stcs(out + (ll)f * np + k, fmaf(s, m1.v[f], (1.0f - s) * m0.v[f]));
        return;
    }
    uint32_t Y = torus_coord(y, g.invL);
    int cy = cell_of(Y, n);
    float t = frac_f(Y, n);
    int y1 = cy + 1 == n ? 0 : cy + 1;
    const ll i00 = (ll)cy * n + cx, i10 = (ll)cy * n + x1, i01 = (ll)y1 * n + cx, i11 = (ll)y1 * n + x1;
    float w00, w10, w01, w11;
    cell_weights(g.p1 != 0, s, t, w00, w10, w01, w11);
    const NodeVec<W> m00 = load_node<W>(il, i00), m10 = load_node<W>(il, i10), m01 = load_node<W>(il, i01),
                     m11 = load_node<W>(il, i11);
#pragma unroll
    for (int f = 0; f < W; ++f) {
        if (f < F) {
            float v = w00 * m00.v[f];
            v = fmaf(w10, m10.v[f], v);
            v = fmaf(w01, m01.v[f], v);
            v = fmaf(w11, m11.v[f], v);
            __stcs(out + (ll)f * np + k, v);
        }
    }
}

// The same interpolation at the particles of the context's sort, in sorted
// order: slot s reads its torus coordinates from pos[s] (those of caller
// particle perm[s], so the weights and the result are the same bits as
// k_g2p's for that particle) and writes out[f][s]. Consecutive threads hold
// particles of the same or neighbouring cells, so a warp's corner loads fall
// on a few lines and mostly hit L1. The fields stay interleaved per node:
// four 16-byte corner loads beat 4F 4-byte ones here too (0.128 against
// 0.182 ms on 16.8M particles, F = 4).
template <int DIM, int W>
__global__ void __launch_bounds__(256) k_g2p_sorted(Geo g, const float *__restrict__ il, int F,
                                                    const uint2 *__restrict__ pos, ll np, float *__restrict__ out) {
    const ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const int n = g.n;
    const uint2 P = __ldcs(pos + k);
    const int cx = cell_of(P.x, n);
    const float s = frac_f(P.x, n);
    const int x1 = cx + 1 == n ? 0 : cx + 1;
    if (DIM == 1) {
        const NodeVec<W> m0 = load_node<W>(il, cx), m1 = load_node<W>(il, x1);
#pragma unroll
        for (int f = 0; f < W; ++f)
            if (f < F) __stcs(out + (ll)f * np + k, fmaf(s, m1.v[f], (1.0f - s) * m0.v[f]));
        return;
    }
    const int cy = cell_of(P.y, n);
    const float t = frac_f(P.y, n);
    const int y1 = cy + 1 == n ? 0 : cy + 1;
    const ll i00 = (ll)cy * n + cx, i10 = (ll)cy * n + x1, i01 = (ll)y1 * n + cx, i11 = (ll)y1 * n + x1;
    float w00, w10, w01, w11;
    cell_weights(g.p1 != 0, s, t, w00, w10, w01, w11);
    const NodeVec<W> m00 = load_node<W>(il, i00), m10 = load_node<W>(il, i10), m01 = load_node<W>(il, i01),
                     m11 = load_node<W>(il, i11);
#pragma unroll
    for (int f = 0; f < W; ++f) {
        if (f < F) {
            float v = w00 * m00.v[f];
            v = fmaf(w10, m10.v[f], v);
            v = fmaf(w01, m01.v[f], v);
            v = fmaf(w11, m11.v[f], v);
            __stcs(out + (ll)f * np + k, v);
        }
    }
}

template <int DIM>
void g2p_sorted_run(const Geo &g, const float *mesh, int F, const uint2 *pos, ll np, float *out, float *il,
                    cudaStream_t st) {
    const int nb = div_up(np, 256), nbm = div_up(g.ncell, 256);
    if (F == 1) {
        k_g2p_sorted<DIM, 1><<<nb, 256, 0, st>>>(g, mesh, F, pos, np, out);
        count_launches(1);
        return;
    }
    if (F == 2) {
        k_interleave<2><<<nbm, 256, 0, st>>>(g.ncell, F, mesh, il);
        k_g2p_sorted<DIM, 2><<<nb, 256, 0, st>>>(g, il, F, pos, np, out);
    } else if (F <= 4) {
        k_interleave<4><<<nbm, 256, 0, st>>>(g.ncell, F, mesh, il);
        k_g2p_sorted<DIM, 4><<<nb, 256, 0, st>>>(g, il, F, pos, np, out);
    } else {
        k_interleave<8><<<nbm, 256, 0, st>>>(g.ncell, F, mesh, il);
        k_g2p_sorted<DIM, 8><<<nb, 256, 0, st>>>(g, il, F, pos, np, out);
    }
    count_launches(2);
}

template <int DIM>
void g2p_run(const Geo &g, const float *mesh, int F, const float *px, const float *py, ll np, float *out,
               float *il, int *status, cudaStream_t st) {
    const int nb = div_up(np, 256), nbm = div_up(g.ncell, 256);
    if (F == 1) {
        k_g2p<DIM, 1><<<nb, 256, 0, st>>>(g, mesh, F, px, py, np, out, status);
        count_launches(1);
        return;
    }
    if (F == 2) {
        k_interleave<2><<<nbm, 256, 0, st>>>(g.ncell, F, mesh, il);
        k_g2p<DIM, 2><<<nb, 256, 0, st>>>(g, il, F, px, py, np, out, status);
    } else if (F <= 4) {
        k_interleave<4><<<nbm, 256, 0, st>>>(g.ncell, F, mesh, il);
        k_g2p<DIM, 4><<<nb, 256, 0, st>>>(g, il, F, px, py, np, out, status);
    } else {
        k_interleave<8><<<nbm, 256, 0, st>>>(g.ncell, F, mesh, il);
        k_g2p<DIM, 8><<<nb, 256, 0, st>>>(g, il, F, px, py, np, out, status);
    }
    count_launches(2);
}

__global__ void k_unsort(ll np, const int *__restrict__ perm, const float *__restrict__ src, float *__restrict__ dst) {
    ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < np) dst[perm[s]] = src[s];
}

}  // namespace

int g2p_width(int F) { return F == 1 ? 1 : (F == 2 ? 2 : (F <= 4 ? 4 : 8)); }

void launch_g2p(const Geo &g, const float *mesh, int F, const float *px, const float *py, ll np, float *out,
                float *il, int *status, cudaStream_t st) {
    if (np <= 0) return;
    if (g.dim == 1)
        g2p_run<1>(g, mesh, F, px, py, np, out, il, status, st);
    else
        g2p_run<2>(g, mesh, F, px, py, np, out, il, status, st);
}

void launch_g2p_sorted(const Geo &g, const float *mesh, int F, const uint2 *pos, ll np, float *out, float *il,
                       cudaStream_t st) {
    if (np <= 0) return;
    if (g.dim == 1)
        g2p_sorted_run<1>(g, mesh, F, pos, np, out, il, st);
    else
        g2p_sorted_run<2>(g, mesh, F, pos, np, out, il, st);
}

void launch_scatter_sorted(ll np, const int *perm, const float *src, float *dst, cudaStream_t st) {
    if (np > 0) {
        k_unsort<<<div_up(np, 256), 256, 0, st>>>(np, perm, src, dst);
        count_launches(1);
    }
}
