// Particle -> mesh assignments (Sec. 2.2 - 2.4).
//
//  delta  (Eq. delta):   Ab_i = A(r_i), the particle interpolant at the node.
//  FLIP   (Eqs. PIC, FLIP_vol): Ab_i = sum v A psi_i(r) / sum v psi_i(r).
//  mass right-hand side (Eq. proj with phi_def): b_j = int A psi_j.
//
// Determinism: delta writes every node exactly once (no reduction); FLIP sums
// per cell in a fixed order with compensated FP32 and then per node over the
// four adjacent cells in a fixed order; the right-hand side accumulates exact
// 64-bit fixed-point integers (2^E scaled, E from max |A| per field), whose
// sum does not depend on the order of the atomic additions.
#include "internal.cuh"

#define PM_VIRT_LIMIT 0x0ffffff0

PM_DEBUG_DECL(transfer)

namespace {

__device__ __forceinline__ void decode(int e, int &id, int &ox, int &oy) {
    id = e & 0x0fffffff;
    int c = (unsigned)e >> 28;
    ox = c / 3 - 1;
    oy = c % 3 - 1;
}

// Relative torus coordinates of the star neighbour encoded as e (|.| <= 2^30).
__device__ __forceinline__ void rel_of(int e, uint2 Xp, const uint2 *__restrict__ pos, int &id, ll &rx, ll &ry) {
    int ox, oy;
    decode(e, id, ox, oy);
    PM_CHK(id >= 0 && id < PM_VIRT_LIMIT, 301, id = 0)
    uint2 Xq = pos[id];
    rx = (ll)Xq.x + (ll)ox * 4294967296LL - (ll)Xp.x;
    ry = (ll)Xq.y + (ll)oy * 4294967296LL - (ll)Xp.y;
}

// Fixed-point exponent of field f (fixed_point_exp of its max|A|).
__device__ __forceinline__ int fix_exp(const unsigned *maxabs, int f, float hd) {
    return fixed_point_exp(__uint_as_float(maxabs[f]), hd);
}

// Sign of orient(U, V, Q) with Q perturbed by (eps, eps^2) (ties never zero).
__device__ __noinline__ int orient_pert_exact(ll ux, ll uy, ll vx, ll vy, ll qx, ll qy) {
    i128 o = (i128)(vx - ux) * (qy - uy) - (i128)(vy - uy) * (qx - ux);
    if (o != 0) return o > 0 ? 1 : -1;
    if (vy != uy) return vy > uy ? -1 : 1;
    return vx > ux ? 1 : -1;
}

// The same sign, decided in float when the float value clears a rigorous
// bound: with d1..d4 the exact integer differences, each converted with
// relative error <= u = 2^-24, the products carry <= 3.01u and the
// subtraction u, so |o_f - o| <= 4.1u (|t1| + |t2|); 8u is used. Otherwise
// (in particular for exact ties) the 128-bit evaluation decides.
__device__ __forceinline__ int orient_pert(ll ux, ll uy, ll vx, ll vy, ll qx, ll qy) {
    const float t1 = (float)(vx - ux) * (float)(qy - uy);
    const float t2 = (float)(vy - uy) * (float)(qx - ux);
    const float o = t1 - t2, bound = 4.77e-7f * (fabsf(t1) + fabsf(t2));
    if (o > bound) return 1;
    if (o < -bound) return -1;
    return orient_pert_exact(ux, uy, vx, vy, qx, qy);
}

// ---------------------------------------------------------------------------
// delta assignment
// ---------------------------------------------------------------------------
// Nodes inside the triangle (p, a, b) (relative torus coordinates of a and b
// given; p at Xp) get the linear interpolant of the particle values, Eq.
// delta. A node is inside when all three orientations are non-negative with
// the node perturbed by (eps, eps^2), so that every node belongs to exactly
// one triangle.
__device__ __forceinline__ void delta_tri(const Geo &g, ll np, int p, int ida, int idb, uint2 Xp, ll ax, ll ay,
                                          ll bx, ll by, const float *__restrict__ vals, int F,
                                          float *__restrict__ mesh) {
    const int n = g.n;
    const ll Xn = (ll)Xp.x * n, Yn = (ll)Xp.y * n;
    const float sc = (float)n * 2.3283064365386963e-10f;  // torus units -> cell units
    const ll Ax = ax * n, Ay = ay * n, Bx = bx * n, By = by * n;
    ll xlo = min(0LL, min(Ax, Bx)) + Xn, xhi = max(0LL, max(Ax, Bx)) + Xn;
    ll ylo = min(0LL, min(Ay, By)) + Yn, yhi = max(0LL, max(Ay, By)) + Yn;
    ll i0 = -((-xlo) >> 32), i1 = xhi >> 32, j0 = -((-ylo) >> 32), j1 = yhi >> 32;
    if (i0 > i1 || j0 > j1) return;
    const float fax = (float)ax * sc, fay = (float)ay * sc, fbx = (float)bx * sc, fby = (float)by * sc;
    const float D = fax * fby - fay * fbx;
    for (ll j = j0; j <= j1; ++j)
        for (ll i = i0; i <= i1; ++i) {
            const ll qx = i * 4294967296LL - Xn, qy = j * 4294967296LL - Yn;
            if (orient_pert(Ax, Ay, Bx, By, qx, qy) < 0) continue;
            if (orient_pert(Bx, By, 0, 0, qx, qy) < 0) continue;
            if (orient_pert(0, 0, Ax, Ay, qx, qy) < 0) continue;
            const float fqx = (float)qx * 2.3283064365386963e-10f, fqy = (float)qy * 2.3283064365386963e-10f;
            float la = (fqx * fby - fqy * fbx) / D;  // weight of a
            float lb = (fax * fqy - fay * fqx) / D;  // weight of b
            float lp = 1.0f - la - lb;
            const ll node = (ll)wrapi((int)(j % n), n) * n + wrapi((int)(i % n), n);
            PM_CHK(node >= 0 && node < g.ncell && ida < np && idb < np, 302, continue)
            const ll fs = field_stride(g);
            for (int f = 0; f < F; ++f) {
                const float *v = vals + (ll)f * np;
                mesh[(ll)f * fs + node] = lp * v[p] + la * v[ida] + lb * v[idb];
            }
        }
}

__device__ __forceinline__ void delta_particle(const Geo &g, ll np, int p, const uint2 *__restrict__ pos,
                                               const int *__restrict__ nbr, const unsigned char *__restrict__ deg,
                                               const float *__restrict__ vals, int F, float *__restrict__ mesh) {
    const int m = deg[p];
    if (m < 3) return;
    const uint2 Xp = pos[p];
    int ida;
    ll ax, ay;
    rel_of(nbr[(ll)(m - 1) * np + p], Xp, pos, ida, ax, ay);
    for (int k = 0; k < m; ++k) {
        int idb;
        ll bx, by;
        rel_of(nbr[(ll)k * np + p], Xp, pos, idb, bx, by);
        // triangle (p, a, b) with a = q_{k-1}, b = q_k; owned by its lowest sorted index
        if (ida > p && idb > p) delta_tri(g, np, p, ida, idb, Xp, ax, ay, bx, by, vals, F, mesh);
        ida = idb;
        ax = bx;
        ay = by;
    }
}

__global__ void __launch_bounds__(128, 8) k_delta2d(Geo g, ll np, const uint2 *__restrict__ pos,
                                                 const int *__restrict__ nbr, const unsigned char *__restrict__ deg,
                                                 const float *__restrict__ vals, int F, float *__restrict__ mesh) {
    const ll pl = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl < np) delta_particle(g, np, (int)pl, pos, nbr, deg, vals, F, mesh);
}

// Batched: the particle's instance writes its nodes of the packed [F][NC] mesh.
__global__ void __launch_bounds__(128, 8) k_delta2d_b(BTab t, const uint2 *__restrict__ pos,
                                                   const int *__restrict__ nbr, const unsigned char *__restrict__ deg,
                                                   const float *__restrict__ vals, int F, float *__restrict__ mesh) {
    const ll pl = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= t.NP) return;
    const int k = find_slot(t.poff, t.ninst, pl);
    delta_particle(batch_geo(t, k), t.NP, (int)pl, pos, nbr, deg, vals, F, mesh + __ldg(t.coff + k));
}

// 1D: node i lies between the last particle at or left of it and the next one.
// The nodes are those of the mesh refined r times (r n nodes at spacing h/r);
// node i lies in mesh cell i / r.
__global__ void k_delta1d(Geo g, ll np, const uint2 *__restrict__ pos, const int *__restrict__ cell_start,
                          const float *__restrict__ vals, int F, float *__restrict__ mesh, int r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = g.n * r;
    if (i >= n) return;
    const ull node = (ull)i << 32;  // node position times r n
    // last sorted particle with X r n <= i 2^32
    ll s = -1;
    int c = i / r, steps = 0;
    {
        int e = cell_start[c + 1];
        for (int t = cell_start[c]; t < e; ++t)
            if ((ull)pos[t].x * (ull)n <= node) s = t;
    }
    while (s < 0 && steps < g.n) {
        c = c == 0 ? g.n - 1 : c - 1;
        ++steps;
        if (cell_start[c + 1] > cell_start[c]) s = cell_start[c + 1] - 1;
    }
    if (s < 0) return;
    ll s1 = s + 1 < np ? s + 1 : 0;
    double xa = (double)((ull)pos[s].x * (ull)n), xb = (double)((ull)pos[s1].x * (ull)n);
    double xn = (double)node;
    if (xa > xn) xa -= 4294967296.0 * n;  // wrapped from the previous period
    if (xb <= xa) xb += 4294967296.0 * n;
    float w = (float)((xn - xa) / (xb - xa));
    for (int f = 0; f < F; ++f) {
        const float *v = vals + (ll)f * np;
        mesh[(ll)f * n + i] = (1.0f - w) * v[s] + w * v[s1];
    }
}

// ---------------------------------------------------------------------------
// FLIP
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(128) k_flip_cells(Geo g, ll np, const int *__restrict__ cell_start,
                                                    const uint2 *__restrict__ pos, const float *__restrict__ vals,
                                                    const float *__restrict__ vol, int F, float *__restrict__ part) {
    ll c = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    constexpr int NC = DIM == 2 ? 4 : 2;
    KSum acc[NC][PM_MAXF + 1];
    const int s0 = cell_start[c], s1 = cell_start[c + 1];
    for (int s = s0; s < s1; ++s) {
        uint2 X = pos[s];
        float sx = frac_f(X.x, g.n);
        float w[NC];
        if (DIM == 2) {
            float ty = frac_f(X.y, g.n);
            cell_weights(g.p1 != 0, sx, ty, w[0], w[1], w[NC - 2], w[NC - 1]);
        } else {
            w[0] = 1.0f - sx;
            w[1] = sx;
        }
        const float v = vol[s];
        for (int k = 0; k < NC; ++k) {
            const float vw = v * w[k];
            acc[k][F].add(vw);
            for (int f = 0; f < F; ++f) acc[k][f].add(vw * vals[(ll)f * np + s]);
        }
    }
    for (int k = 0; k < NC; ++k)
        for (int f = 0; f <= F; ++f) part[(ll)(k * (F + 1) + f) * g.ncell + c] = acc[k][f].get();
}

// Per node: v_i^FLIP = sum over its cells of the volume partials, and
// Ab_i = (sum of the value partials) / v_i (FLIP, pic_vol = 0) or / pic_vol
// (PIC with the mesh volume pic_vol = int psi_i = h^dim, Eq. PIC with
// Eq. mesh_v).
template <int DIM>
__global__ void k_flip_nodes(Geo g, int F, const float *__restrict__ part, float *__restrict__ mesh,
                             float *__restrict__ node_vol, int *__restrict__ empty, float pic_vol) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    int e = 0;
    if (i < g.ncell) {
        const int n = g.n;
        ll cells[4];
        int nc;
        if (DIM == 2) {
            int ix = (int)(i % n), iy = (int)(i / n);
            int xm = ix == 0 ? n - 1 : ix - 1, ym = iy == 0 ? n - 1 : iy - 1;
            cells[0] = (ll)iy * n + ix;   // node is corner 0 (lower left) of this cell
            cells[1] = (ll)iy * n + xm;   // corner 1
            cells[2] = (ll)ym * n + ix;   // corner 2
            cells[3] = (ll)ym * n + xm;   // corner 3
            nc = 4;
        } else {
            cells[0] = i;
            cells[1] = i == 0 ? n - 1 : i - 1;
            nc = 2;
        }
        KSum den;
        for (int k = 0; k < nc; ++k) den.add(part[(ll)(k * (F + 1) + F) * g.ncell + cells[k]]);
        float d = den.get();
        if (node_vol) node_vol[i] = d;
        if (d == 0.0f) e = 1;
        for (int f = 0; f < F; ++f) {
            KSum num;
            for (int k = 0; k < nc; ++k) num.add(part[(ll)(k * (F + 1) + f) * g.ncell + cells[k]]);
            if (pic_vol > 0.0f)
                mesh[(ll)f * g.ncell + i] = num.get() / pic_vol;
            else
                mesh[(ll)f * g.ncell + i] = d != 0.0f ? num.get() / d : 0.0f;
        }
    }
    e = __syncthreads_count(e);
    if (threadIdx.x == 0 && e) atomicAdd(empty, e);
}

// ---------------------------------------------------------------------------
// mass right-hand side, exact
// ---------------------------------------------------------------------------

// Green's-theorem edge sums of the directed segment (x0,y0) -> (x1,y1) for the
// moments  int s^a t^b  (a + b <= 3, without s^3 and t^3); scaled at the end.
struct Mom {
    float a0 = 0, a10 = 0, a01 = 0, a20 = 0, a11 = 0, a02 = 0, a21 = 0, a12 = 0;
    __device__ __forceinline__ void seg(float x0, float y0, float x1, float y1) {
        const float c = x0 * y1 - x1 * y0;
        a0 += c;
        a10 += c * (x0 + x1);
        a01 += c * (y0 + y1);
        a20 += c * (x0 * x0 + x0 * x1 + x1 * x1);
        a02 += c * (y0 * y0 + y0 * y1 + y1 * y1);
        a11 += c * (x0 * y1 + 2.0f * x0 * y0 + 2.0f * x1 * y1 + x1 * y0);
        a21 += c * (3.0f * x1 * x1 * y1 + 2.0f * x0 * x1 * y1 + x0 * x0 * y1 + x1 * x1 * y0 + 2.0f * x0 * x1 * y0 +
                    3.0f * x0 * x0 * y0);
        a12 += c * (3.0f * y1 * y1 * x1 + 2.0f * y0 * y1 * x1 + y0 * y0 * x1 + y1 * y1 * x0 + 2.0f * y0 * y1 * x0 +
                    3.0f * y0 * y0 * x0);
    }
};

// Liang-Barsky step for the constraint p t <= q on t in [t0, t1], with
// rinv = 1/p given (every p here is a component of a triangle edge, so each
// piece needs only six reciprocals).
__device__ __forceinline__ bool lb(float p, float q, float rinv, float &t0, float &t1) {
    if (p == 0.0f) return q >= 0.0f;
    const float r = q * rinv;
    if (p < 0.0f) t0 = fmaxf(t0, r);
    else t1 = fminf(t1, r);
    return true;
}

// Moments of (triangle T) intersected with the unit cell [0,1]^2, in
// coordinates relative to the origin (ox, oy). T counter-clockwise, given in
// cell coordinates. The boundary of the intersection is the part of T's
// edges inside the cell plus the part of the cell's edges inside T.
__device__ __forceinline__ Mom tri_cell_moments(const float tx[3], const float ty[3], float ox, float oy) {
    Mom M;
    float ex[3], ey[3], rx[3], ry[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1;
        ex[k] = tx[k1] - tx[k];
        ey[k] = ty[k1] - ty[k];
        rx[k] = __frcp_rn(ex[k]);
        ry[k] = __frcp_rn(ey[k]);
    }
    for (int k = 0; k < 3; ++k) {
        const float px = tx[k], py = ty[k], dx = ex[k], dy = ey[k];
        // an edge lying exactly on a cell line is accounted for by the cell edge
        if ((dx == 0.0f && (px == 0.0f || px == 1.0f)) || (dy == 0.0f && (py == 0.0f || py == 1.0f))) continue;
        float t0 = 0.0f, t1 = 1.0f;
        if (!lb(-dx, px, -rx[k], t0, t1) || !lb(dx, 1.0f - px, rx[k], t0, t1) || !lb(-dy, py, -ry[k], t0, t1) ||
            !lb(dy, 1.0f - py, ry[k], t0, t1))
            continue;
        if (!(t0 < t1)) continue;
        M.seg(px + t0 * dx - ox, py + t0 * dy - oy, px + t1 * dx - ox, py + t1 * dy - oy);
    }
    const float cxs[5] = {0.0f, 1.0f, 1.0f, 0.0f, 0.0f}, cys[5] = {0.0f, 0.0f, 1.0f, 1.0f, 0.0f};
    for (int e = 0; e < 4; ++e) {
        const float ux = cxs[e], uy = cys[e], vx = cxs[e + 1], vy = cys[e + 1];
        float t0 = 0.0f, t1 = 1.0f;
        bool ok = true;
        for (int k = 0; k < 3 && ok; ++k) {
            const float q0 = ex[k] * (uy - ty[k]) - ey[k] * (ux - tx[k]);
            // cell edge directions (1,0), (0,1), (-1,0), (0,-1): dq = -ey, ex, ey, -ex
            const float dq = e == 0 ? -ey[k] : (e == 1 ? ex[k] : (e == 2 ? ey[k] : -ex[k]));
            const float rdq = e == 0 ? -ry[k] : (e == 1 ? rx[k] : (e == 2 ? ry[k] : -rx[k]));
            ok = lb(-dq, q0, -rdq, t0, t1);
        }
        if (!ok || !(t0 < t1)) continue;
        M.seg(ux + t0 * (vx - ux) - ox, uy + t0 * (vy - uy) - oy, ux + t1 * (vx - ux) - ox, uy + t1 * (vy - uy) - oy);
    }
    return M;
}

// Moments of (triangle T) intersected with the lower half of the unit cell
// (s >= t: the triangle (0,0), (1,0), (1,1) of the P1 split), relative to
// (ox, oy); T counter-clockwise in cell coordinates. As for the cell: T's
// edges inside the half plus the half's edges inside T. An edge of T on a
// line of the half's boundary is left to the half's edge; when T lies on the
// far side of the diagonal with an edge on it, the intersection is a segment
// and the moments are zero.
__device__ __forceinline__ Mom tri_lower_moments(const float tx[3], const float ty[3], float ox, float oy) {
    Mom M;
    float ex[3], ey[3], rx[3], ry[3], rd[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1;
        ex[k] = tx[k1] - tx[k];
        ey[k] = ty[k1] - ty[k];
        rx[k] = __frcp_rn(ex[k]);
        ry[k] = __frcp_rn(ey[k]);
        rd[k] = __frcp_rn(ex[k] - ey[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
        if (tx[k] == ty[k] && tx[k1] == ty[k1] && tx[k2] < ty[k2]) return M;
    }
    for (int k = 0; k < 3; ++k) {
        const float px = tx[k], py = ty[k], dx = ex[k], dy = ey[k];
        if ((dy == 0.0f && py == 0.0f) || (dx == 0.0f && px == 1.0f) || (dx == dy && px == py)) continue;
        float t0 = 0.0f, t1 = 1.0f;
        // y >= 0, x <= 1, x - y >= 0
        if (!lb(-dy, py, -ry[k], t0, t1) || !lb(dx, 1.0f - px, rx[k], t0, t1) ||
            !lb(dy - dx, px - py, -rd[k], t0, t1))
            continue;
        if (!(t0 < t1)) continue;
        M.seg(px + t0 * dx - ox, py + t0 * dy - oy, px + t1 * dx - ox, py + t1 * dy - oy);
    }
    // the half's edges (0,0)->(1,0), (1,0)->(1,1), (1,1)->(0,0)
    const float hxs[4] = {0.0f, 1.0f, 1.0f, 0.0f}, hys[4] = {0.0f, 0.0f, 1.0f, 0.0f};
    for (int e = 0; e < 3; ++e) {
        const float ux = hxs[e], uy = hys[e], vx = hxs[e + 1], vy = hys[e + 1];
        float t0 = 0.0f, t1 = 1.0f;
        bool ok = true;
        for (int k = 0; k < 3 && ok; ++k) {
            const float q0 = ex[k] * (uy - ty[k]) - ey[k] * (ux - tx[k]);
            // directions (1,0), (0,1), (-1,-1): dq = -ey, ex, ey - ex
            const float dq = e == 0 ? -ey[k] : (e == 1 ? ex[k] : ey[k] - ex[k]);
            const float rdq = e == 0 ? -ry[k] : (e == 1 ? rx[k] : -rd[k]);
            ok = lb(-dq, q0, -rdq, t0, t1);
        }
        if (!ok || !(t0 < t1)) continue;
        M.seg(ux + t0 * (vx - ux) - ox, uy + t0 * (vy - uy) - oy, ux + t1 * (vx - ux) - ox, uy + t1 * (vy - uy) - oy);
    }
    return M;
}

// Integrals K0 = int psi_c, K1 = int X psi_c, K2 = int Y psi_c of the four
// corner functions over one piece, in local coordinates X = s - ox,
// Y = t - oy. Bilinear: from the piece's moments up to degree 3. P1: on each
// half of the split cell the three non-zero hats are affine, P + Q X + R Y,
// so the moments up to degree 2 of the two halves suffice (the upper half's
// are the piece's minus the lower half's).
template <int P1>
__device__ __forceinline__ void corner_integrals(const Mom &Mm, const float tx[3], const float ty[3], float ox,
                                                 float oy, float K0[4], float K1[4], float K2[4]) {
    const float M00 = Mm.a0 * 0.5f, M10 = Mm.a10 * (1.0f / 6.0f), M01 = Mm.a01 * (1.0f / 6.0f);
    const float M20 = Mm.a20 * (1.0f / 12.0f), M11 = Mm.a11 * (1.0f / 24.0f);
    const float M02 = Mm.a02 * (1.0f / 12.0f);
    if (!P1) {
        const float M21 = Mm.a21 * (1.0f / 60.0f), M12 = Mm.a12 * (1.0f / 60.0f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float A1 = (c & 1) ? ox : 1.0f - ox, B1 = (c & 1) ? 1.0f : -1.0f;
            const float A2 = (c & 2) ? oy : 1.0f - oy, B2 = (c & 2) ? 1.0f : -1.0f;
            const float aa = A1 * A2, ab = A1 * B2, ba = B1 * A2, bb = B1 * B2;
            K0[c] = aa * M00 + ab * M01 + ba * M10 + bb * M11;
            K1[c] = aa * M10 + ab * M11 + ba * M20 + bb * M21;
            K2[c] = aa * M01 + ab * M02 + ba * M11 + bb * M12;
        }
        return;
    }
    const Mom Ml = tri_lower_moments(tx, ty, ox, oy);
    const float L00 = Ml.a0 * 0.5f, L10 = Ml.a10 * (1.0f / 6.0f), L01 = Ml.a01 * (1.0f / 6.0f);
    const float L20 = Ml.a20 * (1.0f / 12.0f), L11 = Ml.a11 * (1.0f / 24.0f), L02 = Ml.a02 * (1.0f / 12.0f);
    const float U00 = M00 - L00, U10 = M10 - L10, U01 = M01 - L01;
    const float U20 = M20 - L20, U11 = M11 - L11, U02 = M02 - L02;
    // lower half: (0,0): 1 - s; (1,0): s - t; (1,1): t
    // upper half: (0,0): 1 - t; (0,1): t - s; (1,1): s
    const float pl0 = 1.0f - ox, pl1 = ox - oy, pl3 = oy;
    const float pu0 = 1.0f - oy, pu2 = oy - ox, pu3 = ox;
    K0[0] = pl0 * L00 - L10 + pu0 * U00 - U01;
    K1[0] = pl0 * L10 - L20 + pu0 * U10 - U11;
    K2[0] = pl0 * L01 - L11 + pu0 * U01 - U02;
    K0[1] = pl1 * L00 + L10 - L01;
    K1[1] = pl1 * L10 + L20 - L11;
    K2[1] = pl1 * L01 + L11 - L02;
    K0[2] = pu2 * U00 - U10 + U01;
    K1[2] = pu2 * U10 - U20 + U11;
    K2[2] = pu2 * U01 - U11 + U02;
    K0[3] = pl3 * L00 + L01 + pu3 * U00 + U10;
    K1[3] = pl3 * L10 + L11 + pu3 * U10 + U20;
    K2[3] = pl3 * L01 + L02 + pu3 * U01 + U11;
}

#define RTS 16                      // cells per tile side
#define RHALO 2                     // window halo in cells
#define RWIN (RTS + 2 * RHALO + 1)  // window side in nodes

// Triangle k of particle p's star, (p, q_{k-1}, q_k), in cell units relative
// to p's cell corner, and its cell bounding box. Returns false when p does not
// own it (ownership: lowest sorted index).
struct Tri {
    float vx[3], vy[3];
    int a, b, i0, i1, j0, j1;
};
__device__ __forceinline__ bool owned_tri(int p, int m, int k, uint2 Xp, float up, float wp, float sc,
                                          const uint2 *__restrict__ pos, const int *__restrict__ nbr, ll np, Tri &T) {
    ll ax, ay, bx, by;
    rel_of(nbr[(ll)(k == 0 ? m - 1 : k - 1) * np + p], Xp, pos, T.a, ax, ay);
    rel_of(nbr[(ll)k * np + p], Xp, pos, T.b, bx, by);
    if (T.a <= p || T.b <= p) return false;
    // One explicit rounding (FMA) per coordinate: the piece counting and the
    // piece integration call this separately and must get the same bits, also
    // when a vertex lies exactly on a cell line (the bounding box below);
    // left to the compiler, the two inlined copies may round differently.
    T.vx[0] = up; T.vx[1] = __fmaf_rn((float)ax, sc, up); T.vx[2] = __fmaf_rn((float)bx, sc, up);
    T.vy[0] = wp; T.vy[1] = __fmaf_rn((float)ay, sc, wp); T.vy[2] = __fmaf_rn((float)by, sc, wp);
    T.i0 = (int)floorf(fminf(T.vx[0], fminf(T.vx[1], T.vx[2])));
    T.i1 = (int)floorf(fmaxf(T.vx[0], fmaxf(T.vx[1], T.vx[2])));
    T.j0 = (int)floorf(fminf(T.vy[0], fminf(T.vy[1], T.vy[2])));
    T.j1 = (int)floorf(fmaxf(T.vy[0], fmaxf(T.vy[1], T.vy[2])));
    return true;
}

// Exact 64-bit accumulation with native 32-bit shared-memory atomics: the
// low word returns its old value, the carry out of it goes into the high word
// together with the high half of the addend (sums modulo 2^64, any order).
__device__ __forceinline__ void add64_split(unsigned *lo, unsigned *hi, ull v) {
    const unsigned vl = (unsigned)v, vh = (unsigned)(v >> 32);
    const unsigned old = atomicAdd(lo, vl);
    const unsigned carry = (unsigned)(old + vl < old);
    if (vh + carry) atomicAdd(hi, vh + carry);
}

#define RTAB 24  // owned-triangle table entries per particle (>= PM_MAXDEG)

// One block per tile of RTS x RTS cells. The (triangle, cell) pieces of the
// triangles owned by the tile's particles are spread evenly over the lanes of
// each warp (prefix sum of per-particle piece counts, then every lane takes
// one piece per round), integrated exactly, and their four corner integrals
// go to a shared window of nodes (64-bit fixed point, order-free integer
// sums) or, outside the window, straight to global memory. While counting,
// every lane records its owned triangles (star slot, running piece count) so
// that a piece finds its triangle without walking the star again.
//
// MODE 1 runs the same pieces the other way (mesh -> particles): it integrates
// the bilinear mesh interpolant Ab against the three particle functions of
// the triangle, c_mu = int Ab psi_mu, and adds the results to the particles'
// 64-bit fixed-point sums cfix (global atomics; order-free integer sums).
// maxabs then holds max|Ab| per field, and the fixed-point scale keeps 10
// bits of headroom for particle volumes up to 1024 h^2.
template <int FF, int MODE, int P1>
__device__ __forceinline__ void rhs2d_tile(const Geo &g, ll np, const uint2 *__restrict__ pos,
                                           const int *__restrict__ cell_start, const int *__restrict__ nbr,
                                           const unsigned char *__restrict__ deg, const float *__restrict__ vals,
                                           int F, const unsigned *__restrict__ maxabs, ll *__restrict__ bfix,
                                           int tiles_x, const float *__restrict__ mesh, ll *__restrict__ cfix,
                                           int tile) {
    // dynamic shared memory: acc_lo, acc_hi [FF][RWIN^2], tab [RTAB][256]
    extern __shared__ unsigned rhs_smem[];
    unsigned(*acc_lo)[RWIN * RWIN] = (unsigned(*)[RWIN * RWIN])rhs_smem;
    unsigned(*acc_hi)[RWIN * RWIN] = (unsigned(*)[RWIN * RWIN])(rhs_smem + FF * RWIN * RWIN);
    unsigned(*tab)[256] = (unsigned(*)[256])(rhs_smem + 2 * FF * RWIN * RWIN);  // (star slot << 16) | pieces so far
    __shared__ int rowpre[RTS + 1];
    __shared__ int rowbeg[RTS];
    __shared__ int next_chunk;  // next 32-particle chunk of the tile (warps take chunks as they finish)
    const int n = g.n;
    const int tx0 = (tile % tiles_x) * RTS, ty0 = (tile / tiles_x) * RTS;
    const ll fs = field_stride(g);
    const int wx0 = tx0 - RHALO, wy0 = ty0 - RHALO;
    for (int i = threadIdx.x; i < FF * RWIN * RWIN; i += blockDim.x) {
        (&acc_lo[0][0])[i] = 0u;
        (&acc_hi[0][0])[i] = 0u;
    }
    if (threadIdx.x == 0) {
        int tot = 0;
        const int xe = min(tx0 + RTS, n);
        for (int r = 0; r < RTS; ++r) {
            rowpre[r] = tot;
            int y = ty0 + r;
            if (y < n) {
                rowbeg[r] = cell_start[(ll)y * n + tx0];
                tot += cell_start[(ll)y * n + xe] - rowbeg[r];
            } else {
                rowbeg[r] = 0;
            }
        }
        rowpre[RTS] = tot;
        next_chunk = 0;
    }
    __syncthreads();
    const float hd = g.h * g.h;
    const float sc = (float)n * 2.3283064365386963e-10f;
    int E[FF];
    for (int f = 0; f < FF; ++f) E[f] = f < F ? fix_exp(maxabs, f, hd) - (MODE == 1 ? 10 : 0) : 0;
    // h^dim 2^E as one float factor: scaling by a power of two is exact, so
    // round(x (h^dim 2^E)) equals round(x h^dim) 2^E
    float S[FF];
    for (int f = 0; f < FF; ++f) S[f] = ldexpf(hd, E[f]);
    const int total = rowpre[RTS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int tcol = threadIdx.x;
    (void)wid;
    (void)nw;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&next_chunk, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        // this lane's particle, its owned triangles and its number of pieces
        const int k = base + lane;
        int p = -1, cnt = 0;
        if (k < total) {
            int r = 0;
            while (rowpre[r + 1] <= k) ++r;
            p = rowbeg[r] + (k - rowpre[r]);
            PM_CHK(p >= 0 && p < np, 303, p = 0)
            const int m = deg[p];
            if (m >= 3) {
                const uint2 Xp = pos[p];
                const float up = frac_f(Xp.x, n), wp = frac_f(Xp.y, n);
                int nt = 0;
                for (int kk = 0; kk < m; ++kk) {
                    Tri T;
                    if (owned_tri(p, m, kk, Xp, up, wp, sc, pos, nbr, np, T)) {
                        cnt += (T.i1 - T.i0 + 1) * (T.j1 - T.j0 + 1);
                        PM_CHK(nt < RTAB, 307, break)
                        tab[nt][tcol] = ((unsigned)kk << 16) | (unsigned)cnt;
                        ++nt;
                    }
                }
            }
        }
        __syncwarp();
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = incl - cnt;
        const int T_all = __shfl_sync(0xffffffffu, incl, 31);
        for (int j0 = 0; j0 < T_all; j0 += 32) {
            const int j = j0 + lane;
            // owner lane of piece j: the first lane whose inclusive count exceeds j
            int lo = 0;
            for (int step = 16; step > 0; step >>= 1) {
                int v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                if (v <= j) lo += step;
            }
            const int src = lo;
            const int ps = __shfl_sync(0xffffffffu, p, src);
            const int jj = j - __shfl_sync(0xffffffffu, excl, src);
            if (j >= T_all) continue;
            // locate the piece: the owner's table gives the star slot
            PM_CHK(ps >= 0 && ps < np, 304, continue)
            const int scol = (tcol & ~31) + src;
            int e = 0, prev = 0;
            unsigned te = tab[0][scol];
            while ((int)(te & 0xffffu) <= jj) {
                prev = (int)(te & 0xffffu);
                ++e;
                PM_CHK(e < RTAB, 308, break)
                te = tab[e][scol];
            }
            const int kk = (int)(te >> 16), rem = jj - prev;
            const int m = deg[ps];
            const uint2 Xp = pos[ps];
            const int cxp = cell_of(Xp.x, n), cyp = cell_of(Xp.y, n);
            const float up = frac_f(Xp.x, n), wp = frac_f(Xp.y, n);
            Tri T;
            if (!owned_tri(ps, m, kk, Xp, up, wp, sc, pos, nbr, np, T)) continue;
            const int wdt = T.i1 - T.i0 + 1;
            const int ci = T.i0 + rem % wdt, cj = T.j0 + rem / wdt;
            PM_CHK(T.a >= 0 && T.a < np && T.b >= 0 && T.b < np, 305, continue)
            const float fci = (float)ci, fcj = (float)cj;
            const float xmin = fminf(T.vx[0], fminf(T.vx[1], T.vx[2])), xmax = fmaxf(T.vx[0], fmaxf(T.vx[1], T.vx[2]));
            const float ymin = fminf(T.vy[0], fminf(T.vy[1], T.vy[2])), ymax = fmaxf(T.vy[0], fmaxf(T.vy[1], T.vy[2]));
            const float tx[3] = {T.vx[0] - fci, T.vx[1] - fci, T.vx[2] - fci};
            const float ty[3] = {T.vy[0] - fcj, T.vy[1] - fcj, T.vy[2] - fcj};
            const float ox = 0.5f * (fmaxf(0.0f, xmin - fci) + fminf(1.0f, xmax - fci));
            const float oy = 0.5f * (fmaxf(0.0f, ymin - fcj) + fminf(1.0f, ymax - fcj));
            Mom Mm = tri_cell_moments(tx, ty, ox, oy);
            if (!(Mm.a0 > 0.0f)) continue;
            float K0[4], K1[4], K2[4];
            corner_integrals<P1>(Mm, tx, ty, ox, oy, K0, K1, K2);
            // A on the triangle: value at p plus gradient (cell units)
            const float e1x = T.vx[1] - T.vx[0], e1y = T.vy[1] - T.vy[0];
            const float e2x = T.vx[2] - T.vx[0], e2y = T.vy[2] - T.vy[0];
            const float idet = 1.0f / (e1x * e2y - e1y * e2x);
            const float dsx = ox + fci - up, dty = oy + fcj - wp;
            const int gcx = cxp + ci, gcy = cyp + cj;  // unwrapped cell
            if (MODE == 1) {
                // W_k[f] = sum over corners of Ab_c * (K0, K1, K2)_c
                float W0[FF], W1[FF], W2[FF];
#pragma unroll
                for (int f = 0; f < FF; ++f) W0[f] = W1[f] = W2[f] = 0.0f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int nx = gcx + (c & 1), ny = gcy + ((c >> 1) & 1);
                    const ll node = (ll)wrapi(ny, n) * n + wrapi(nx, n);
                    PM_CHK(node >= 0 && node < g.ncell, 309, continue)
#pragma unroll
                    for (int f = 0; f < FF; ++f) {
                        if (f >= F) break;
                        const float ab_c = __ldg(mesh + (ll)f * fs + node);
                        W0[f] = fmaf(ab_c, K0[c], W0[f]);
                        W1[f] = fmaf(ab_c, K1[c], W1[f]);
                        W2[f] = fmaf(ab_c, K2[c], W2[f]);
                    }
                }
                // barycentric functions about the local origin: lambda = l0 + lx X' + ly Y'
                const float l0a = (dsx * e2y - dty * e2x) * idet, lxa = e2y * idet, lya = -e2x * idet;
                const float l0b = (e1x * dty - e1y * dsx) * idet, lxb = -e1y * idet, lyb = e1x * idet;
                const float l0p = 1.0f - l0a - l0b, lxp = -(lxa + lxb), lyp = -(lya + lyb);
                const int who[3] = {ps, T.a, T.b};
                const float L0[3] = {l0p, l0a, l0b}, LX[3] = {lxp, lxa, lxb}, LY[3] = {lyp, lya, lyb};
#pragma unroll
                for (int v = 0; v < 3; ++v) {
#pragma unroll
                    for (int f = 0; f < FF; ++f) {
                        if (f >= F) break;
                        const ll iv = __float2ll_rn((L0[v] * W0[f] + LX[v] * W1[f] + LY[v] * W2[f]) * S[f]);
                        if (iv) atomicAdd((ull *)&cfix[(ll)f * np + who[v]], (ull)iv);
                    }
                }
                continue;
            }
            float al[FF], gx[FF], gy[FF];
#pragma unroll
            for (int f = 0; f < FF; ++f) {
                if (f < F) {
                    const float A0 = vals[(ll)f * np + ps];
                    const float da = vals[(ll)f * np + T.a] - A0, db = vals[(ll)f * np + T.b] - A0;
                    gx[f] = (da * e2y - db * e1y) * idet;
                    gy[f] = (db * e1x - da * e2x) * idet;
                    al[f] = A0 + gx[f] * dsx + gy[f] * dty;  // A at the local origin
                } else {
                    gx[f] = gy[f] = al[f] = 0.0f;
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int nx = gcx + (c & 1), ny = gcy + ((c >> 1) & 1);
                const int lx = nx - wx0, ly = ny - wy0;
                const bool inwin = lx >= 0 && lx < RWIN && ly >= 0 && ly < RWIN;
                const ll node = (ll)wrapi(ny, n) * n + wrapi(nx, n);
                PM_CHK(node >= 0 && node < g.ncell, 306, continue)
#pragma unroll
                for (int f = 0; f < FF; ++f) {
                    if (f >= F) break;
                    const ll iv = __float2ll_rn((al[f] * K0[c] + gx[f] * K1[c] + gy[f] * K2[c]) * S[f]);
                    if (!iv) continue;
                    if (inwin)
                        add64_split(&acc_lo[f][ly * RWIN + lx], &acc_hi[f][ly * RWIN + lx], (ull)iv);
                    else
                        atomicAdd((ull *)&bfix[(ll)f * fs + node], (ull)iv);
                }
            }
        }
        __syncwarp();
    }
    if (MODE == 1) return;
    __syncthreads();
    for (int i = threadIdx.x; i < RWIN * RWIN; i += blockDim.x) {
        const int lx = i % RWIN, ly = i / RWIN;
        const ll node = (ll)wrapi(wy0 + ly, n) * n + wrapi(wx0 + lx, n);
        for (int f = 0; f < F && f < FF; ++f) {
            const ull v = ((ull)acc_hi[f][i] << 32) | (ull)acc_lo[f][i];
            if (v) atomicAdd((ull *)&bfix[(ll)f * fs + node], v);
        }
    }
}

template <int FF, int MODE, int P1>
__global__ void __launch_bounds__(256, 4) k_rhs2d(Geo g, ll np, const uint2 *__restrict__ pos,
                                               const int *__restrict__ cell_start, const int *__restrict__ nbr,
                                               const unsigned char *__restrict__ deg, const float *__restrict__ vals,
                                               int F, const unsigned *__restrict__ maxabs, ll *__restrict__ bfix,
                                               int tiles_x, const float *__restrict__ mesh, ll *__restrict__ cfix) {
    rhs2d_tile<FF, MODE, P1>(g, np, pos, cell_start, nbr, deg, vals, F, maxabs, bfix, tiles_x, mesh, cfix,
                             (int)blockIdx.x);
}

// Batched: block b is tile b - tile_start[k] of instance k; the instance's
// cell ranges, max|A| and fixed-point sums are views of the packed arrays.
template <int FF>
__global__ void __launch_bounds__(256, 4) k_rhs2d_b(BTab t, const int *__restrict__ tile_start,
                                                 const uint2 *__restrict__ pos, const int *__restrict__ cell_start,
                                                 const int *__restrict__ nbr, const unsigned char *__restrict__ deg,
                                                 const float *__restrict__ vals, int F,
                                                 const unsigned *__restrict__ maxabs, ll *__restrict__ bfix) {
    const int k = find_slot(tile_start, t.ninst, (int)blockIdx.x);
    const Geo g = batch_geo(t, k);
    const ll co = __ldg(t.coff + k);
    rhs2d_tile<FF, 0, 0>(g, t.NP, pos, cell_start + co, nbr, deg, vals, F, maxabs + (ll)k * PM_MAXF, bfix + co,
                         (g.n + RTS - 1) / RTS, nullptr, nullptr, (int)blockIdx.x - __ldg(tile_start + k));
}

// 1D: interval between sorted particle s and the next one on the circle.
__global__ void k_rhs1d(Geo g, ll np, const uint2 *__restrict__ pos, const float *__restrict__ vals, int F,
                        const unsigned *__restrict__ maxabs, ll *__restrict__ bfix) {
    ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const int n = g.n;
    const ll s1 = s + 1 < np ? s + 1 : 0;
    const uint32_t xa = pos[s].x;
    const ull gap = s + 1 < np ? (ull)(pos[s1].x - xa) : 4294967296ull - (ull)(xa - pos[0].x);
    if (gap == 0) return;
    const float len = (float)(gap * (ull)n) * 2.3283064365386963e-10f;  // in cells
    const int c0 = cell_of(xa, n);
    const float u0 = frac_f(xa, n), u1 = u0 + len;
    for (int k = 0; (float)k < u1; ++k) {
        float lo = fmaxf(u0, (float)k), hi = fminf(u1, (float)(k + 1));
        if (!(hi > lo)) continue;
        const int na = wrapi(c0 + k, n), nb = na + 1 == n ? 0 : na + 1;
        const float t0 = lo - (float)k, t1 = hi - (float)k;
        // integrals of 1, t, t^2 over [t0, t1]
        const float m0 = t1 - t0, m1 = 0.5f * (t1 * t1 - t0 * t0), m2 = (t1 * t1 * t1 - t0 * t0 * t0) * (1.0f / 3.0f);
        for (int f = 0; f < F; ++f) {
            const float Aa = vals[(ll)f * np + s], Ab = vals[(ll)f * np + s1];
            const float be = (Ab - Aa) / len;                 // dA/du
            const float al = Aa + be * ((float)k - u0);       // A at t = 0 of this cell
            // int A (1 - t) dt and int A t dt, A = al + be t
            const float wl = al * (m0 - m1) + be * (m1 - m2);
            const float wr = al * m1 + be * m2;
            const int E = fix_exp(maxabs, f, g.h);
            ll il = __float2ll_rn(ldexpf(wl * g.h, E)), ir = __float2ll_rn(ldexpf(wr * g.h, E));
            if (il) atomicAdd((ull *)&bfix[(ll)f * n + na], (ull)il);
            if (ir) atomicAdd((ull *)&bfix[(ll)f * n + nb], (ull)ir);
        }
    }
}

// App. B quadrature right-hand side from A sampled on the mesh refined twice
// (A2 [F][(2n)^dim], the delta values at the nodes, edge midpoints and cell
// centres). On every element A is replaced by its (bi)quadratic interpolant
// through those samples and integrated exactly against the (bi)linear hats:
// per dimension the element weights of the left hat at the points 0, h/2, h
// are h (1/6, 1/3, 0) and of the right hat h (0, 1/3, 1/6), so over the two
// elements around node i the weights at its refined offsets -1, 0, +1 are all
// h/3 (and 0 at +-2). b_i is thus h^dim / 3^dim times the sum of A2 over the
// 3 (1D) or 3 x 3 (2D) refined points around node i. Written once per node in
// the fixed point of the exact right-hand side.
template <int DIM>
__global__ void k_appb_box(Geo g, int F, const float *__restrict__ A2, const unsigned *__restrict__ maxabs,
                           ll *__restrict__ bfix) {
    const ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const int n = g.n, n2 = 2 * n;
    const ll nn2 = DIM == 2 ? (ll)n2 * n2 : (ll)n2;
    const float hd = DIM == 2 ? g.h * g.h : g.h;
    const float w = DIM == 2 ? hd * (1.0f / 9.0f) : hd * (1.0f / 3.0f);
    const int ix = (int)(i % n), iy = DIM == 2 ? (int)(i / n) : 0;
    for (int f = 0; f < F; ++f) {
        const float *a = A2 + (ll)f * nn2;
        float sum = 0.0f;
        if (DIM == 2) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const ll row = (ll)wrapi(2 * iy + dy, n2) * n2;
                float rs = 0.0f;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) rs += a[row + wrapi(2 * ix + dx, n2)];
                sum += rs;
            }
        } else {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) sum += a[wrapi(2 * ix + dx, n2)];
        }
        bfix[(ll)f * g.ncell + i] = __float2ll_rn(ldexpf(sum * w, fix_exp(maxabs, f, hd)));
    }
}

// Batched: node j of the packed [F][NC] arrays belongs to instance k.
__global__ void k_fix_to_float_b(BTab t, int F, const ll *__restrict__ bfix, const unsigned *__restrict__ maxabs,
                                 float *__restrict__ out) {
    const ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t.NC * F) return;
    const int f = (int)(i / t.NC);
    const int k = find_slot(t.coff, t.ninst, i - (ll)f * t.NC);
    const float h = t.inst[k].h;
    out[i] = ldexpf((float)bfix[i], -fix_exp(maxabs + (ll)k * PM_MAXF, f, h * h));
}

__global__ void k_fix_to_float(Geo g, int F, const ll *__restrict__ bfix, const unsigned *__restrict__ maxabs,
                               float *__restrict__ out) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell * F) return;
    int f = (int)(i / g.ncell);
    float hd = g.dim == 2 ? g.h * g.h : g.h;
    out[i] = ldexpf((float)bfix[i], -fix_exp(maxabs, f, hd));
}

// Per-block sums of v_mu A_mu and v_mu |A_mu| (FP64 across threads). Each
// thread takes 4 consecutive particles per step (16-byte loads when the
// arrays allow it) so that enough loads are in flight.
__global__ void __launch_bounds__(256) k_psum(ll np, const float *__restrict__ vals, const float *__restrict__ vol,
                                              int F, double *__restrict__ out, int nblk) {
    __shared__ double sh[2 * PM_MAXF][8];
    const ll tid = (ll)blockIdx.x * blockDim.x + threadIdx.x, nth = (ll)gridDim.x * blockDim.x;
    const bool vec = (np & 3) == 0;
    for (int f = 0; f < F; ++f) {
        Dot2 a, b;
        const float *x = vals + (ll)f * np;
        if (vec) {
            for (ll q = tid; q < np / 4; q += nth) {
                const float4 v = ((const float4 *)vol)[q], y = ((const float4 *)x)[q];
                a.fma_acc(v.x, y.x);
                a.fma_acc(v.y, y.y);
                a.fma_acc(v.z, y.z);
                a.fma_acc(v.w, y.w);
                b.fma_acc(v.x, fabsf(y.x));
                b.fma_acc(v.y, fabsf(y.y));
                b.fma_acc(v.z, fabsf(y.z));
                b.fma_acc(v.w, fabsf(y.w));
            }
        } else {
            for (ll s = tid; s < np; s += nth) {
                const float v = vol[s], y = x[s];
                a.fma_acc(v, y);
                b.fma_acc(v, fabsf(y));
            }
        }
        double da = (double)a.hi + (double)a.lo, db = (double)b.hi + (double)b.lo;
        for (int o = 16; o > 0; o >>= 1) {
            da += __shfl_xor_sync(0xffffffffu, da, o);
            db += __shfl_xor_sync(0xffffffffu, db, o);
        }
        if ((threadIdx.x & 31) == 0) {
            sh[2 * f][threadIdx.x >> 5] = da;
            sh[2 * f + 1][threadIdx.x >> 5] = db;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * F) {
        double s = 0;
        for (int w = 0; w < 8; ++w) s += sh[threadIdx.x][w];
        out[(ll)threadIdx.x * nblk + blockIdx.x] = s;
    }
}

// Network input per field f: delta / max|A_f| and the residual of the delta
// start, r = b - M delta (b the exact right-hand side from its fixed point,
// M the bilinear mass stencil), as PM_NET_RSCALE r / (h^2 max|A_f|): the exact
// correction is M^-1 r, a fixed, fast-decaying linear operator of r.
__global__ void k_features(Geo g, int F, const float *__restrict__ delta, const ll *__restrict__ bfix,
                           const unsigned *__restrict__ maxabs, float *__restrict__ feat) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const int n = g.n, ix = (int)(i % n), iy = (int)(i / n);
    const int xm = ix == 0 ? n - 1 : ix - 1, xp = ix + 1 == n ? 0 : ix + 1;
    const int ym = iy == 0 ? n - 1 : iy - 1, yp = iy + 1 == n ? 0 : iy + 1;
    const float hd = g.h * g.h;
    for (int f = 0; f < F; ++f) {
        const float s = __uint_as_float(maxabs[f]);
        const float inv = s > 0.0f ? 1.0f / s : 0.0f;
        const float *d = delta + (ll)f * g.ncell;
        const float *r0 = d + (ll)ym * n, *r1 = d + (ll)iy * n, *r2 = d + (ll)yp * n;
        Dot2 acc;
        acc.add(16.0f * r1[ix]);
        acc.add(4.0f * r1[xm]);
        acc.add(4.0f * r1[xp]);
        acc.add(4.0f * r0[ix]);
        acc.add(4.0f * r2[ix]);
        acc.add(r0[xm]);
        acc.add(r0[xp]);
        acc.add(r2[xm]);
        acc.add(r2[xp]);
        const float b = ldexpf((float)bfix[(ll)f * g.ncell + i], -fix_exp(maxabs, f, hd));
        const float res = (b - hd * (1.0f / 36.0f) * acc.hi) - hd * (1.0f / 36.0f) * acc.lo;
        feat[((ll)f * 2 + 0) * g.ncell + i] = d[i] * inv;
        feat[((ll)f * 2 + 1) * g.ncell + i] = PM_NET_RSCALE * res * inv / hd;
    }
}

// Relative residual of the delta start per field, ||b - M delta|| / ||b||,
// from the network's input channels: channel 1 is PM_NET_RSCALE r / (h^2
// max|A|); b is read from its fixed point. FP64 block partials [2F][nblk]
// (sum r^2, sum b^2, both in units of (h^2 max|A|)^2), reduced by
// k_start_resid_final into out[f].
__global__ void __launch_bounds__(256) k_start_resid(Geo g, int F, const float *__restrict__ feat,
                                                      const ll *__restrict__ bfix, const unsigned *__restrict__ maxabs,
                                                      double *__restrict__ part) {
    __shared__ double sh[2 * PM_MAXF][8];
    const float hd = g.h * g.h;
    double acc[2 * PM_MAXF];
    for (int k = 0; k < 2 * F; ++k) acc[k] = 0.0;
    for (ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x; i < g.ncell; i += (ll)gridDim.x * blockDim.x) {
        for (int f = 0; f < F; ++f) {
            const float s = __uint_as_float(maxabs[f]);
            const float inv = s > 0.0f ? 1.0f / (s * hd) : 0.0f;
            const double r = (double)feat[((ll)f * 2 + 1) * g.ncell + i] * (1.0 / PM_NET_RSCALE);
            const double b = (double)(ldexpf((float)bfix[(ll)f * g.ncell + i], -fix_exp(maxabs, f, hd)) * inv);
            acc[2 * f] += r * r;
            acc[2 * f + 1] += b * b;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 2 * F; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * F) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += sh[threadIdx.x][w];
        part[(ll)threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_start_resid_final(int F, int nblk, const double *__restrict__ part, double *__restrict__ out) {
    const int f = threadIdx.x;
    if (f >= F) return;
    double rr = 0.0, bb = 0.0;
    for (int b = 0; b < nblk; ++b) {
        rr += part[(ll)(2 * f) * nblk + b];
        bb += part[(ll)(2 * f + 1) * nblk + b];
    }
    out[f] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
}

// Step length of the network's correction. With r0 = b - M delta (feature
// channel 1 times max|A| h^2 / PM_NET_RSCALE) and the correction
// c = (max|A| / PM_NET_RSCALE) corr, the start delta + alpha c has residual
// r0 - alpha M c, smallest in the 2-norm for
//   alpha = <r0, M c> / <M c, M c> = 36 <feat1, S corr> / <S corr, S corr>
// (M = h^2/36 S, S the 9-point stencil 1-4-1 x 1-4-1). alpha = 0 keeps the
// delta start, so the network can never make the start worse than delta in
// this norm. Per-block FP64 partials, then one fixed-order reduction.
#define ALPHA_BLOCKS 608
__global__ void __launch_bounds__(256) k_alpha_partial(Geo g, int F, const float *__restrict__ feat,
                                                        const float *__restrict__ corr, double *__restrict__ part) {
    __shared__ double sh[2 * PM_MAXF][8];
    const int n = g.n;
    double acc[2 * PM_MAXF];
    for (int k = 0; k < 2 * F; ++k) acc[k] = 0.0;
    for (ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x; i < g.ncell; i += (ll)gridDim.x * blockDim.x) {
        const int ix = (int)(i % n), iy = (int)(i / n);
        const int xm = ix == 0 ? n - 1 : ix - 1, xp = ix + 1 == n ? 0 : ix + 1;
        const int ym = iy == 0 ? n - 1 : iy - 1, yp = iy + 1 == n ? 0 : iy + 1;
        for (int f = 0; f < F; ++f) {
            const float *c = corr + (ll)f * g.ncell;
            const float *r0 = c + (ll)ym * n, *r1 = c + (ll)iy * n, *r2 = c + (ll)yp * n;
            const float z = 16.0f * r1[ix] + 4.0f * (r1[xm] + r1[xp] + r0[ix] + r2[ix]) +
                            (r0[xm] + r0[xp] + r2[xm] + r2[xp]);
            const float f1 = feat[((ll)f * 2 + 1) * g.ncell + i];
            acc[2 * f] += (double)f1 * (double)z;
            acc[2 * f + 1] += (double)z * (double)z;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 2 * F; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * F) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += sh[threadIdx.x][w];
        part[(ll)threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_alpha_final(int F, int nblk, const double *__restrict__ part, double *__restrict__ alpha) {
    const int f = threadIdx.x;
    if (f >= F) return;
    double num = 0.0, den = 0.0;
    for (int b = 0; b < nblk; ++b) {
        num += part[(ll)(2 * f) * nblk + b];
        den += part[(ll)(2 * f + 1) * nblk + b];
    }
    const double a = den > 0.0 ? 36.0 * num / den : 0.0;
    alpha[f] = isfinite(a) ? a : 0.0;
}

// Warm start: mesh = delta + alpha_f (max|A_f| / PM_NET_RSCALE) * network output.
__global__ void k_apply_corr(Geo g, int F, const float *__restrict__ corr, const unsigned *__restrict__ maxabs,
                             const double *__restrict__ alpha, float *__restrict__ mesh) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    for (int f = 0; f < F; ++f) {
        const float k = (float)alpha[f] * __uint_as_float(maxabs[f]) * (1.0f / PM_NET_RSCALE);
        mesh[(ll)f * g.ncell + i] += k * corr[(ll)f * g.ncell + i];
    }
}

// ---------------------------------------------------------------------------
// mesh -> particle integrals c_mu = int Ab psi_mu (Table 1, right column)
// ---------------------------------------------------------------------------
// max |Ab| of every field (non-negative float bits order like unsigned ints)
__global__ void k_mesh_max(ll nn, int F, const float *__restrict__ mesh, unsigned *__restrict__ out) {
    for (int f = 0; f < F; ++f) {
        float m = 0.0f;
        for (ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (ll)gridDim.x * blockDim.x)
            m = fmaxf(m, fabsf(__ldg(mesh + (ll)f * nn + i)));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(out + f, __float_as_uint(m));
    }
}

// fixed-point particle sums -> float (the scale of the mesh->particle mode)
__global__ void k_fixc_to_float(ll np, int F, const ll *__restrict__ cfix, const unsigned *__restrict__ meshmax,
                                float hd, float *__restrict__ c) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np * F) return;
    const int f = (int)(i / np);
    c[i] = ldexpf((float)cfix[i], -(fix_exp(meshmax, f, hd) - 10));
}

// 1D: particle s (sorted by position) gathers its own integral over the two
// intervals beside it, cut at the mesh nodes; Simpson's rule is exact on each
// piece (linear x linear). Coordinates in cell units relative to s's cell.
__device__ __forceinline__ float ab1(const float *__restrict__ m, int n, int cx, float u) {
    const float fe = floorf(u);
    const float t = u - fe;
    const int e = cx + (int)fe;
    return __ldg(m + wrapi(e, n)) * (1.0f - t) + __ldg(m + wrapi(e + 1, n)) * t;
}

__global__ void k_g2pint1d(Geo g, ll np, const uint2 *__restrict__ pos, const float *__restrict__ mesh, int F,
                           float *__restrict__ c) {
    ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const int n = g.n;
    const uint32_t X = pos[s].x;
    const uint32_t Xl = pos[s == 0 ? np - 1 : s - 1].x, Xr = pos[s + 1 == np ? 0 : s + 1].x;
    const float sc = (float)n * 2.3283064365386963e-10f;
    const float dl = np > 1 ? (float)(uint32_t)(X - Xl) * sc : (float)n, dr = np > 1 ? (float)(uint32_t)(Xr - X) * sc
                                                                                   : (float)n;
    const int cx = cell_of(X, n);
    const float fs = frac_f(X, n);
    for (int f = 0; f < F; ++f) {
        const float *m = mesh + (ll)f * n;
        KSum acc;
        // left interval [fs - dl, fs]: psi rises from 0 to 1
        for (int side = 0; side < 2; ++side) {
            const float a = side == 0 ? fs - dl : fs, b = side == 0 ? fs : fs + dr, len = side == 0 ? dl : dr;
            if (!(len > 0.0f)) continue;
            float cur = a;
            while (cur < b) {
                const float nxt = fminf(floorf(cur) + 1.0f, b);
                const float mid = 0.5f * (cur + nxt);
                const float pa = side == 0 ? (cur - a) / len : (b - cur) / len;
                const float pm = side == 0 ? (mid - a) / len : (b - mid) / len;
                const float pb = side == 0 ? (nxt - a) / len : (b - nxt) / len;
                const float q = (nxt - cur) * (1.0f / 6.0f) *
                                (ab1(m, n, cx, cur) * pa + 4.0f * ab1(m, n, cx, mid) * pm + ab1(m, n, cx, nxt) * pb);
                acc.add(q);
                cur = nxt;
            }
        }
        c[(ll)f * np + s] = acc.get() * g.h;
    }
}

}  // namespace

void launch_features(const Geo &g, Work &w, int F, const float *delta, cudaStream_t st) {
    k_features<<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, delta, w.bfix, w.maxabs, w.feat);
    count_launches(1);
}

void launch_start_resid(const Geo &g, Work &w, int F, double *out, cudaStream_t st) {
    double *part = w.red;  // the solver's reduction buffer (the solve has not started yet)
    k_start_resid<<<ALPHA_BLOCKS, 256, 0, st>>>(g, F, w.feat, w.bfix, w.maxabs, part);
    k_start_resid_final<<<1, 32, 0, st>>>(F, ALPHA_BLOCKS, part, out);
    count_launches(2);
}

void launch_apply_correction(const Geo &g, Work &w, int F, float *mesh, cudaStream_t st) {
    // scratch: the solver's reduction buffer (the solve has not started yet)
    double *part = w.red, *alpha = w.red + 2LL * PM_MAXF * ALPHA_BLOCKS;
    k_alpha_partial<<<ALPHA_BLOCKS, 256, 0, st>>>(g, F, w.feat, w.corr, part);
    k_alpha_final<<<1, 32, 0, st>>>(F, ALPHA_BLOCKS, part, alpha);
    k_apply_corr<<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, w.corr, w.maxabs, alpha, mesh);
    count_launches(3);
}

void launch_delta(const Geo &g, Work &w, ll np, int F, float *mesh_out, cudaStream_t st) {
    if (g.dim == 2)
        k_delta2d<<<div_up(np, 128), 128, 0, st>>>(g, np, w.pos, w.nbr, w.deg, w.vals, F, mesh_out);
    else
        k_delta1d<<<div_up(g.n, 128), 128, 0, st>>>(g, np, w.pos, w.cell_start, w.vals, F, mesh_out, 1);
    count_launches(1);
}

// App. B quadrature right-hand side into bfix: delta on the mesh refined
// twice (into the FLIP partials, free in a mass assignment), then the box sum.
void launch_rhs_appb(const Geo &g, Work &w, ll np, int F, cudaStream_t st) {
    float *A2 = w.part;  // [F][(2n)^dim] <= (2^dim)(F + 1) n^dim floats
    if (g.dim == 2) {
        Geo g2 = g;
        g2.n = 2 * g.n;
        g2.ncell = 4 * g.ncell;
        g2.h = 0.5f * g.h;
        cudaMemsetAsync(A2, 0, sizeof(float) * F * g2.ncell, st);
        if (np > 0) k_delta2d<<<div_up(np, 128), 128, 0, st>>>(g2, np, w.pos, w.nbr, w.deg, w.vals, F, A2);
        k_appb_box<2><<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, A2, w.maxabs, w.bfix);
    } else {
        cudaMemsetAsync(A2, 0, sizeof(float) * F * 2 * g.n, st);
        if (np > 0) k_delta1d<<<div_up(2 * g.n, 128), 128, 0, st>>>(g, np, w.pos, w.cell_start, w.vals, F, A2, 2);
        k_appb_box<1><<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, A2, w.maxabs, w.bfix);
    }
    count_launches(np > 0 ? 2 : 1);
}

void launch_flip(const Geo &g, Work &w, ll np, int F, float *mesh_out, float *node_vol, cudaStream_t st,
                 float pic_vol) {
    cudaMemsetAsync(w.empty, 0, sizeof(int), st);
    if (g.dim == 2) {
        k_flip_cells<2><<<div_up(g.ncell, 128), 128, 0, st>>>(g, np, w.cell_start, w.pos, w.vals, w.vol, F, w.part);
        k_flip_nodes<2><<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, w.part, mesh_out, node_vol, w.empty, pic_vol);
    } else {
        k_flip_cells<1><<<div_up(g.ncell, 128), 128, 0, st>>>(g, np, w.cell_start, w.pos, w.vals, w.vol, F, w.part);
        k_flip_nodes<1><<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, w.part, mesh_out, node_vol, w.empty, pic_vol);
    }
    count_launches(2);
}

template <int FF>
static size_t rhs2d_smem() {
    return sizeof(unsigned) * (2 * FF * RWIN * RWIN + RTAB * 256);
}

// Raise the dynamic shared-memory limit of the RHS kernels on the current
// device (called when a context is created, outside any stream capture).
template <int FF>
static void rhs_attr() {
    cudaFuncSetAttribute(k_rhs2d_b<FF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs2d_smem<FF>());
    cudaFuncSetAttribute(k_rhs2d<FF, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs2d_smem<FF>());
    cudaFuncSetAttribute(k_rhs2d<FF, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs2d_smem<FF>());
    cudaFuncSetAttribute(k_rhs2d<FF, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs2d_smem<FF>());
    cudaFuncSetAttribute(k_rhs2d<FF, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs2d_smem<FF>());
}

void rhs_prepare_device() {
    rhs_attr<2>();
    rhs_attr<4>();
    rhs_attr<PM_MAXF>();
}

template <int FF>
static void launch_rhs2d(const Geo &g, Work &w, ll np, int F, int nt, int tx, cudaStream_t st) {
    const size_t bytes = rhs2d_smem<FF>();
    if (g.p1)
        k_rhs2d<FF, 0, 1><<<nt, 256, bytes, st>>>(g, np, w.pos, w.cell_start, w.nbr, w.deg, w.vals, F, w.maxabs,
                                                  w.bfix, tx, nullptr, nullptr);
    else
        k_rhs2d<FF, 0, 0><<<nt, 256, bytes, st>>>(g, np, w.pos, w.cell_start, w.nbr, w.deg, w.vals, F, w.maxabs,
                                                  w.bfix, tx, nullptr, nullptr);
}

template <int FF>
static void launch_g2pint2d(const Geo &g, Work &w, ll np, int F, const float *mesh, int nt, int tx,
                            cudaStream_t st) {
    const size_t bytes = rhs2d_smem<FF>();
    if (g.p1)
        k_rhs2d<FF, 1, 1><<<nt, 256, bytes, st>>>(g, np, w.pos, w.cell_start, w.nbr, w.deg, nullptr, F, w.meshmax,
                                                  nullptr, tx, mesh, w.cfix);
    else
        k_rhs2d<FF, 1, 0><<<nt, 256, bytes, st>>>(g, np, w.pos, w.cell_start, w.nbr, w.deg, nullptr, F, w.meshmax,
                                                  nullptr, tx, mesh, w.cfix);
}

void launch_rhs(const Geo &g, Work &w, ll np, int F, cudaStream_t st) {
    cudaMemsetAsync(w.bfix, 0, sizeof(ll) * g.ncell * F, st);
    if (np <= 0) return;
    if (g.dim == 2) {
        const int tx = div_up(g.n, RTS), nt = tx * tx;
        if (F <= 2)
            launch_rhs2d<2>(g, w, np, F, nt, tx, st);
        else if (F <= 4)
            launch_rhs2d<4>(g, w, np, F, nt, tx, st);
        else
            launch_rhs2d<PM_MAXF>(g, w, np, F, nt, tx, st);
    } else
        k_rhs1d<<<div_up(np, 128), 128, 0, st>>>(g, np, w.pos, w.vals, F, w.maxabs, w.bfix);
    count_launches(1);
}

int rhs_tile_side() { return RTS; }

void launch_delta_batched(const BTab &t, Work &w, int F, float *mesh_out, cudaStream_t st) {
    if (t.NP <= 0) return;
    k_delta2d_b<<<div_up(t.NP, 128), 128, 0, st>>>(t, w.pos, w.nbr, w.deg, w.vals, F, mesh_out);
    count_launches(1);
}

void launch_rhs_batched(const BTab &t, Work &w, int F, const int *tile_start, int ntiles, cudaStream_t st) {
    cudaMemsetAsync(w.bfix, 0, sizeof(ll) * t.NC * F, st);
    if (t.NP <= 0 || ntiles <= 0) return;
    if (F <= 2)
        k_rhs2d_b<2><<<ntiles, 256, rhs2d_smem<2>(), st>>>(t, tile_start, w.pos, w.cell_start, w.nbr, w.deg, w.vals,
                                                            F, w.maxabs, w.bfix);
    else if (F <= 4)
        k_rhs2d_b<4><<<ntiles, 256, rhs2d_smem<4>(), st>>>(t, tile_start, w.pos, w.cell_start, w.nbr, w.deg, w.vals,
                                                            F, w.maxabs, w.bfix);
    else
        k_rhs2d_b<PM_MAXF><<<ntiles, 256, rhs2d_smem<PM_MAXF>(), st>>>(t, tile_start, w.pos, w.cell_start, w.nbr,
                                                                        w.deg, w.vals, F, w.maxabs, w.bfix);
    count_launches(1);
}

void launch_rhs_to_float_batched(const BTab &t, Work &w, int F, float *b_out, cudaStream_t st) {
    k_fix_to_float_b<<<div_up(t.NC * F, 256), 256, 0, st>>>(t, F, w.bfix, w.maxabs, b_out);
    count_launches(1);
}

void launch_rhs_to_float(const Geo &g, Work &w, int F, float *b_out, cudaStream_t st) {
    k_fix_to_float<<<div_up(g.ncell * F, 256), 256, 0, st>>>(g, F, w.bfix, w.maxabs, b_out);
    count_launches(1);
}

// c_mu = int Ab psi_mu for every (sorted) particle and field -> c [F][np].
void launch_g2p_integral(const Geo &g, Work &w, ll np, int F, const float *mesh, float *c, cudaStream_t st) {
    if (np <= 0) return;
    cudaMemsetAsync(w.meshmax, 0, sizeof(unsigned) * PM_MAXF, st);
    k_mesh_max<<<2 * 152, 256, 0, st>>>(g.ncell, F, mesh, w.meshmax);
    if (g.dim == 1) {
        k_g2pint1d<<<div_up(np, 256), 256, 0, st>>>(g, np, w.pos, mesh, F, c);
        count_launches(2);
        return;
    }
    cudaMemsetAsync(w.cfix, 0, sizeof(ll) * np * F, st);
    const int tx = div_up(g.n, RTS), nt = tx * tx;
    if (F <= 2)
        launch_g2pint2d<2>(g, w, np, F, mesh, nt, tx, st);
    else if (F <= 4)
        launch_g2pint2d<4>(g, w, np, F, mesh, nt, tx, st);
    else
        launch_g2pint2d<PM_MAXF>(g, w, np, F, mesh, nt, tx, st);
    k_fixc_to_float<<<div_up(np * F, 256), 256, 0, st>>>(np, F, w.cfix, w.meshmax, g.h * g.h, c);
    count_launches(3);
}

namespace {
// Lumped mesh -> particle values: c_mu / v_mu (in place, sorted order).
__global__ void k_div_vol(ll np, int F, const float *__restrict__ vol, float *__restrict__ c) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np * F) return;
    const float v = vol[i % np];
    c[i] = v > 0.0f ? c[i] / v : 0.0f;
}
}  // namespace

void launch_div_vol(ll np, int F, const float *vol, float *c, cudaStream_t st) {
    if (np <= 0) return;
    k_div_vol<<<div_up(np * F, 256), 256, 0, st>>>(np, F, vol, c);
    count_launches(1);
}

namespace {
// Lumped particle -> mesh values: b_i / h^dim (in place).
__global__ void k_scale(ll m, float s, float *__restrict__ x) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) x[i] *= s;
}
}  // namespace

void launch_scale(ll m, float s, float *x, cudaStream_t st) {
    if (m <= 0) return;
    k_scale<<<div_up(m, 256), 256, 0, st>>>(m, s, x);
    count_launches(1);
}

void launch_psum(const Geo &g, Work &w, ll np, int F, cudaStream_t st) {
    (void)g;
    k_psum<<<w.nblk_psum, 256, 0, st>>>(np, w.vals, w.vol, F, w.psum, w.nblk_psum);
    count_launches(1);
}
