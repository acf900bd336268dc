// Particle functions psi_mu (Sec. 3.2, App. A): linear finite elements on the
// periodic Delaunay triangulation of the particles (2D), hat functions over
// the periodically ordered particles (1D); and particle volumes
// v_mu = int psi_mu (Sec. 2.1, Eq. part_v).
//
// 2D: one thread per particle p computes its Voronoi cell by clipping with
// the bisectors of nearby particles, scanned ring by ring of mesh cells from
// the cell-sorted array. The cell is a cyclic list of neighbours q_k; its
// vertex k is the circumcentre of (p, q_k, q_k+1). A candidate s removes
// vertex k iff s lies strictly inside the circle through (p, q_k, q_k+1):
// the in-circle predicate, evaluated exactly on the 32-bit torus
// coordinates (float filter, 128-bit integer fallback), with exact ties
// broken by symbolic perturbation of the lifted coordinate |r|^2 + eps^rank,
// rank = caller index. After ring r the cell is final once every vertex v
// satisfies 2|v| < (distance from p to the unscanned cells). The neighbour
// cycle is p's Delaunay star. Because every decision is exact and the
// perturbation is a property of the point set, the stars of all particles
// agree: every triangle (p, a, b) appears in the stars of p, a and b.
#include "internal.cuh"

namespace {

__device__ __forceinline__ int sgn_ll(ll v) { return (v > 0) - (v < 0); }
__device__ __forceinline__ int sgn_i128(i128 v) { return (v > 0) - (v < 0); }

// Exact "s strictly inside circle(p = 0, a, b)" for counter-clockwise (p,a,b),
// coordinates relative to p with |.| <= 2^30 (every term below 2^124).
__device__ __noinline__ bool incircle_exact(int ax, int ay, int bx, int by, int sx, int sy, int pp, int pa, int pb,
                                            int ps) {
    ll al = (ll)ax * ax + (ll)ay * ay;
    ll bl = (ll)bx * bx + (ll)by * by;
    ll sl = (ll)sx * sx + (ll)sy * sy;
    i128 t1 = (i128)by * sl - (i128)sy * bl;
    i128 t2 = (i128)bx * sl - (i128)sx * bl;
    i128 t3 = (i128)((ll)bx * sy - (ll)by * sx);
    i128 det = (i128)ax * t1 - (i128)ay * t2 + (i128)al * t3;
    if (det != 0) return det < 0;
    // Symbolic perturbation: d/d(eps_k) of the lifted 4x4 determinant is a
    // signed orientation of the other three points.
    int sg[4], pr[4] = {pp, pa, pb, ps};
    i128 oabs = (i128)((ll)bx - ax) * ((ll)sy - ay) - (i128)((ll)by - ay) * ((ll)sx - ax);
    sg[0] = sgn_i128(oabs);
    sg[1] = -sgn_ll((ll)bx * sy - (ll)by * sx);
    sg[2] = sgn_ll((ll)ax * sy - (ll)ay * sx);
    sg[3] = -sgn_ll((ll)ax * by - (ll)ay * bx);
    for (int it = 0; it < 4; ++it) {
        int best = -1;
        for (int k = 0; k < 4; ++k)
            if (pr[k] >= 0 && (best < 0 || pr[k] < pr[best])) best = k;
        if (best < 0) break;
        if (sg[best] != 0) return sg[best] > 0;
        pr[best] = -1;
    }
    return false;
}

// Float filter of the same predicate: +1 inside, -1 outside, 0 undecided.
// |error| of the float evaluation is far below 1e-5 of the permanent.
__device__ __forceinline__ int incircle_filter(float ax, float ay, float bx, float by, float sx, float sy) {
    float al = ax * ax + ay * ay, bl = bx * bx + by * by, sl = sx * sx + sy * sy;
    float t1 = by * sl - sy * bl, t2 = bx * sl - sx * bl, t3 = bx * sy - by * sx;
    float det = ax * t1 - ay * t2 + al * t3;
    float pm = fabsf(ax) * (fabsf(by) * sl + fabsf(sy) * bl) + fabsf(ay) * (fabsf(bx) * sl + fabsf(sx) * bl) +
               al * (fabsf(bx * sy) + fabsf(by * sx));
    float eb = 1e-5f * pm;
    if (det < -eb) return 1;
    if (det > eb) return -1;
    return 0;
}

// Upper bound of |circumcentre(0, a, b)|^2 (infinite when ill-conditioned).
__device__ __forceinline__ float circ_bound2(float ax, float ay, float bx, float by) {
    float al = ax * ax + ay * ay, bl = bx * bx + by * by;
    float D = 2.0f * (ax * by - ay * bx);
    float eD = 2e-5f * (fabsf(ax * by) + fabsf(ay * bx));
    float Nx = by * al - ay * bl, Ny = ax * bl - bx * al;
    float eNx = 1e-5f * (fabsf(by * al) + fabsf(ay * bl));
    float eNy = 1e-5f * (fabsf(ax * bl) + fabsf(bx * al));
    float den = fabsf(D) - eD;
    if (!(den > 0.0f)) return INFINITY;
    float cx = (fabsf(Nx) + eNx) / den, cy = (fabsf(Ny) + eNy) / den;
    return cx * cx + cy * cy;
}

__device__ __forceinline__ int prio(int enc, const int *__restrict__ perm) {
    return enc >= 0 ? perm[enc & 0x0fffffff] : 0x7fffffff + enc;  // virtual points rank last
}

struct Poly {
    int x[2][PM_MAXW], y[2][PM_MAXW], e[2][PM_MAXW];
    float c[2][PM_MAXW];
};

__global__ void __launch_bounds__(128) k_delaunay(Geo g, ll np, const uint2 *__restrict__ pos,
                                                  const int *__restrict__ cell_start, const int *__restrict__ perm,
                                                  int *__restrict__ nbr, unsigned char *__restrict__ deg,
                                                  float *__restrict__ vol, float vol_scale, int *__restrict__ status) {
    ll pl = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= np) return;
    const int p = (int)pl;
    const int n = g.n;
    Poly P;
    int cur = 0, m = 4;
    const int B = 1 << 29;
    // initial cell: the square cut out by four virtual points at distance B
    const int ix[4] = {B, 0, -B, 0}, iy[4] = {0, B, 0, -B};
    for (int k = 0; k < 4; ++k) {
        P.x[0][k] = ix[k];
        P.y[0][k] = iy[k];
        P.e[0][k] = -1 - k;
        P.c[0][k] = 0.5f * (float)B * (float)B;
    }
    float maxc2 = 0.5f * (float)B * (float)B;
    const uint2 Xp = pos[p];
    const int cx = cell_of(Xp.x, n), cy = cell_of(Xp.y, n);
    const float cw = 4294967296.0f / (float)n;
    const float fxl = (float)cell_frac(Xp.x, n) / (float)n, fyl = (float)cell_frac(Xp.y, n) / (float)n;
    const float edge = fminf(fminf(fxl, cw - fxl), fminf(fyl, cw - fyl));
    int pp = -2;  // priority of p, loaded on first exact test
    int rmax = min(PM_RCAP, n / 4 - 1);
    if (rmax < 0) rmax = 0;
    bool done = false;
    int err = 0;
    for (int r = 0; r <= rmax && !done && !err; ++r) {
        int ncells = r == 0 ? 1 : 8 * r;
        for (int ci = 0; ci < ncells && !err; ++ci) {
            int dx, dy;
            if (r == 0) { dx = 0; dy = 0; }
            else if (ci < 2 * r + 1) { dx = ci - r; dy = -r; }
            else if (ci < 4 * r + 2) { dx = ci - (3 * r + 1); dy = r; }
            else if (ci < 6 * r + 1) { dx = -r; dy = ci - (5 * r + 1); }
            else { dx = r; dy = ci - (7 * r); }
            int ux = cx + dx, uy = cy + dy;
            int ox = ux < 0 ? -1 : (ux >= n ? 1 : 0), oy = uy < 0 ? -1 : (uy >= n ? 1 : 0);
            int c = (uy - oy * n) * n + (ux - ox * n);
            int s0 = cell_start[c], s1 = cell_start[c + 1];
            for (int s = s0; s < s1; ++s) {
                if (s == p) continue;
                uint2 Xs = pos[s];
                ll rx = (ll)Xs.x + (ll)ox * 4294967296LL - (ll)Xp.x;
                ll ry = (ll)Xs.y + (ll)oy * 4294967296LL - (ll)Xp.y;
                if (rx == 0 && ry == 0) { err |= ST_DUP; break; }
                if (rx > (1LL << 30) || rx < -(1LL << 30) || ry > (1LL << 30) || ry < -(1LL << 30)) continue;
                const int sx = (int)rx, sy = (int)ry;
                const float fsx = (float)sx, fsy = (float)sy;
                const float d2 = fsx * fsx + fsy * fsy;
                if (d2 > 4.0001f * maxc2) continue;
                // which vertices does s cut away?
                unsigned mask = 0;
                int ps = -2;
                for (int k = 0; k < m; ++k) {
                    if (d2 > 4.0001f * P.c[cur][k]) continue;
                    int k1 = k + 1 == m ? 0 : k + 1;
                    int ax = P.x[cur][k], ay = P.y[cur][k], bx = P.x[cur][k1], by = P.y[cur][k1];
                    int v = incircle_filter((float)ax, (float)ay, (float)bx, (float)by, fsx, fsy);
                    if (v == 0) {
                        if (pp == -2) pp = perm[p];
                        if (ps == -2) ps = perm[s];
                        v = incircle_exact(ax, ay, bx, by, sx, sy, pp, prio(P.e[cur][k], perm),
                                           prio(P.e[cur][k1], perm), ps)
                                ? 1
                                : -1;
                    }
                    if (v > 0) mask |= 1u << k;
                }
                if (mask == 0) continue;
                int cnt = __popc(mask);
                if (cnt >= m) { err |= ST_RANGE; break; }
                // first vertex of the (cyclic) run of removed vertices
                int i0 = 0;
                for (int k = 0; k < m; ++k) {
                    int km = k == 0 ? m - 1 : k - 1;
                    if ((mask >> k & 1u) && !(mask >> km & 1u)) { i0 = k; break; }
                }
                int j1 = i0 + cnt;  // index (mod m) of the first kept neighbour after the run
                int mm = m - cnt + 2;
                if (mm > PM_MAXW) { err |= ST_DEGREE; break; }
                const int nx = cur ^ 1;
                int t = 0;
                for (; t <= m - cnt; ++t) {
                    int k = (j1 + t) % m;
                    P.x[nx][t] = P.x[cur][k];
                    P.y[nx][t] = P.y[cur][k];
                    P.e[nx][t] = P.e[cur][k];
                    P.c[nx][t] = P.c[cur][k];
                }
                // kept q_i (last copied) now meets s, and s meets the first kept
                int qi = m - cnt;
                P.c[nx][qi] = circ_bound2((float)P.x[nx][qi], (float)P.y[nx][qi], fsx, fsy);
                P.x[nx][t] = sx;
                P.y[nx][t] = sy;
                P.e[nx][t] = s | (((ox + 1) * 3 + (oy + 1)) << 28);
                P.c[nx][t] = circ_bound2(fsx, fsy, (float)P.x[nx][0], (float)P.y[nx][0]);
                cur = nx;
                m = mm;
                maxc2 = 0.0f;
                for (int k = 0; k < m; ++k) maxc2 = fmaxf(maxc2, P.c[cur][k]);
            }
        }
        // certified when every vertex is closer than half the distance to
        // anything not yet scanned
        float dmin = edge + (float)r * cw;
        if (4.0001f * maxc2 < dmin * dmin) done = true;
    }
    if (!done && !err) err |= ST_SPARSE;
    if (m > PM_MAXDEG) err |= ST_DEGREE;
    if (err) {
        atomicOr(status, err);
        deg[p] = 0;
        vol[p] = 0.0f;
        return;
    }
    ll area2 = 0;
    for (int k = 0; k < m; ++k) {
        int k1 = k + 1 == m ? 0 : k + 1;
        area2 += (ll)P.x[cur][k] * P.y[cur][k1] - (ll)P.y[cur][k] * P.x[cur][k1];
        nbr[(ll)k * np + p] = P.e[cur][k];
    }
    deg[p] = (unsigned char)m;
    vol[p] = (float)area2 * vol_scale;
}

// 1D: v_mu = half the distance between the two neighbours on the circle.
__global__ void k_vol1d(ll np, const uint2 *__restrict__ pos, float *__restrict__ vol, float scale) {
    ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    uint32_t x = pos[s].x;
    ull gn = s + 1 < np ? (ull)(pos[s + 1].x - x) : 4294967296ull - (ull)(x - pos[0].x);
    ull gp = s > 0 ? (ull)(x - pos[s - 1].x) : 4294967296ull - (ull)(pos[np - 1].x - x);
    vol[s] = (float)(gn + gp) * scale;
}

__global__ void k_export(ll np, const uint2 *__restrict__ pos, const int *__restrict__ nbr,
                         const unsigned char *__restrict__ deg, const int *__restrict__ perm, int *__restrict__ tri,
                         int *__restrict__ off, ll max_tri, ll *__restrict__ counter) {
    ll pl = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= np) return;
    int p = (int)pl, m = deg[p];
    for (int k = 0; k < m; ++k) {
        int ea = nbr[(ll)k * np + p], eb = nbr[(ll)(k + 1 == m ? 0 : k + 1) * np + p];
        int a = ea & 0x0fffffff, b = eb & 0x0fffffff;
        if (a <= p || b <= p) continue;
        ll t = atomicAdd((ull *)counter, 1ull);
        if (t >= max_tri) continue;
        tri[3 * t] = perm[p];
        tri[3 * t + 1] = perm[a];
        tri[3 * t + 2] = perm[b];
        int ca = (unsigned)ea >> 28, cb = (unsigned)eb >> 28;
        off[4 * t] = ca / 3 - 1;
        off[4 * t + 1] = ca % 3 - 1;
        off[4 * t + 2] = cb / 3 - 1;
        off[4 * t + 3] = cb % 3 - 1;
    }
}

}  // namespace

void launch_triangulate(const Geo &g, Work &w, ll np, cudaStream_t st) {
    if (np <= 0) return;
    double u = g.L / 4294967296.0;
    float scale = (float)(u * u / 6.0);
    k_delaunay<<<div_up(np, 128), 128, 0, st>>>(g, np, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol, scale,
                                                 w.status);
    count_launches(1);
}

void launch_volumes_1d(const Geo &g, Work &w, ll np, cudaStream_t st) {
    if (np <= 0) return;
    float scale = (float)(0.5 * g.L / 4294967296.0);
    k_vol1d<<<div_up(np, 256), 256, 0, st>>>(np, w.pos, w.vol, scale);
    count_launches(1);
}

void launch_export_tris(const Geo &g, Work &w, ll np, int *tri, int *off, ll max_tri, cudaStream_t st) {
    cudaMemsetAsync(w.ntri, 0, sizeof(ll), st);
    if (np > 0) {
        k_export<<<div_up(np, 256), 256, 0, st>>>(np, w.pos, w.nbr, w.deg, w.perm, tri, off, max_tri, w.ntri);
        count_launches(1);
    }
}
