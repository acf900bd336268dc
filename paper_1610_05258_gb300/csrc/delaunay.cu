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
// the in-circle predicate, equivalently 2 c_k . s > |s|^2 for the
// circumcentre c_k. It is decided in float from c_k and a rigorous bound on
// its error, and exactly on the 32-bit torus coordinates (128-bit integers)
// when the float value falls inside the error margin; exact ties are broken
// by symbolic perturbation of the lifted coordinate |r|^2 + eps^rank, rank =
// caller index. After ring r the cell is final once every vertex v
// satisfies 2|v| < (distance from p to the unscanned cells). The neighbour
// cycle is p's Delaunay star. Because every decision is exact and the
// perturbation is a property of the point set, the stars of all particles
// agree: every triangle (p, a, b) appears in the stars of p, a and b.
#include "internal.cuh"

PM_DEBUG_DECL(delaunay)

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

// Star entries carry the sorted index in the low 28 bits and the image code
// in the high 4 (so real entries may be negative as ints); the four virtual
// points of the initial cell use the indices PM_VIRT..PM_VIRT+3 and rank last.
#define PM_VIRT 0x0ffffff0
__device__ __forceinline__ int prio(int enc, const int *__restrict__ perm) {
    const int id = enc & 0x0fffffff;
    return id >= PM_VIRT ? 0x7ffffff0 + (id - PM_VIRT) : __ldg(perm + id);
}

#define DBLK 64     // threads per block of the main triangulation pass
#define DCAP 9      // polygon capacity of the main pass (22 warps per SM)
#define R1BLK 32    // threads per block of the first retry pass
#define R1CAP 12    // polygon capacity of the first retry pass (17 warps per SM)
#define RBLK 32     // threads per block of the last retry pass
#define RCAP 24     // polygon capacity of the last retry pass (= PM_MAXDEG)
#define ST_OVERFLOW 0x40000000  // internal: the cell outgrew the main pass's capacity

// Float circumcentre c of (0, a, b) and a bound e on the error of each of its
// components (infinite when the triangle is too flat to bound). Inputs are
// exact integers below 2^30 in magnitude; every rounding, including the
// conversion of the inputs to float, is covered by the 8u factors.
__device__ __forceinline__ void circumcentre(float ax, float ay, float bx, float by, float &cx, float &cy, float &e) {
    const float u8 = 4.8e-7f;  // 8 units of roundoff
    float al = ax * ax + ay * ay, bl = bx * bx + by * by;
    float D = 2.0f * (ax * by - ay * bx);
    float eD = 2.0f * u8 * (fabsf(ax * by) + fabsf(ay * bx));
    float Nx = by * al - ay * bl, Ny = ax * bl - bx * al;
    float eN = u8 * fmaxf(fabsf(by * al) + fabsf(ay * bl), fabsf(ax * bl) + fabsf(bx * al));
    float den = fabsf(D) - eD;
    const float iD = __frcp_rn(D);
    cx = Nx * iD;
    cy = Ny * iD;
    if (!(den > 0.0f)) {
        e = INFINITY;
        return;
    }
    float cm = fmaxf(fabsf(cx), fabsf(cy));
    // per-component bound (the reciprocal and product roundings are inside
    // the u8 term), doubled to cover the vector norm (sqrt 2) with slack
    e = 2.0f * ((eN + cm * eD) * __frcp_ru(den) + u8 * cm);
    if (!(e < INFINITY) || !(cm < INFINITY)) e = INFINITY;
}

// Polygon state of one thread, one column per thread in shared memory:
// neighbour k, q[k] = (x, y, entry) with entry = sorted index | image code <<
// 28, and vertex k, v[k] = (c_k, w_k, rr_k): the circumcentre c_k of
// (p, q_k, q_k+1), the margin w_k = e_k + 8u |c_k| (the float test
// 2 c_k . s > |s|^2 is certain outside w_k |s| + 4u |s|^2), and rr_k, an
// upper bound of (|c_k| + w_k)^2 without square roots:
// (|c| + w)^2 <= |c|^2 + 2 sqrt2 max(|cx|,|cy|) w + w^2 (infinite when the
// vertex is unbounded).
template <int NB>
struct PolyS {
    int4 (*q)[NB];
    float4 (*v)[NB];
    int t;
};

template <int NB>
__device__ __forceinline__ float set_vertex(PolyS<NB> P, int k, float ax, float ay, float bx, float by) {
    float cx, cy, e;
    circumcentre(ax, ay, bx, by, cx, cy, e);
    const float cm = fmaxf(fabsf(cx), fabsf(cy));
    float w = e + 4.8e-7f * cm * 1.5f;
    w = w < INFINITY ? w : INFINITY;
    float rr = (cx * cx + cy * cy) * 1.000001f + 2.8285f * cm * w + w * w;
    rr = rr < INFINITY ? rr : INFINITY;
    P.v[k][P.t] = make_float4(cx, cy, w, rr);
    return rr;
}

// Work of one thread, counted by the counting instantiation of the kernel:
// candidates examined, candidates passing the distance test, vertex tests,
// clips, and the sum of the cell sizes after each clip.
// Work of the cells a pass completes (a pass that gives a cell up to a larger
// capacity drops what it counted for it), and the cells given up.
struct WorkCount {
    unsigned cand = 0, tested = 0, vtests = 0, clips = 0, msum = 0, over = 0, exact = 0;
};

// Clip the cell of p by the bisector of candidate s (relative position
// (sx, sy), sorted index sidx, image code). R2 = max_k rr_k is kept up to
// date: the vertices that survive a clip are those the candidate does not
// remove, plus the two new ones. Returns an error bit or 0.
template <int CAP, int NB, bool COUNT>
__device__ __forceinline__ int clip_by(PolyS<NB> P, int &m, float &R2, int sx, int sy, int sidx, int code, int p,
                                       int &pp, const int *__restrict__ perm, WorkCount &wc) {
    const float fsx = (float)sx, fsy = (float)sy;
    const float d2 = fsx * fsx + fsy * fsy;
    if (COUNT) wc.cand++;
    if (d2 > 4.0001f * R2) return 0;  // |s| > 2 max|c|: no vertex can be cut
    if (COUNT) {
        wc.tested++;
        wc.vtests += m;
    }
    // |s| <= sqrt2 max(|sx|, |sy|) stands in for the norm in the margin
    const float hs = 0.5f * d2, ns = 1.41422f * fmaxf(fabsf(fsx), fabsf(fsy)), mr = 2.4e-7f * d2;
    // float pass: certain inside -> mask, certain outside -> nothing, else
    // undecided (exact pass below, rare)
    // rkeep: the largest radius bound among the vertices not certainly
    // removed (an upper bound of the kept ones: undecided vertices that the
    // exact pass removes only make it larger, which is safe)
    unsigned mask = 0, undecided = 0;
    float rkeep = 0.0f;
    const int t = P.t;
    if (CAP <= 12) {
        // CAP predicated iterations on every lane: no loop exit that depends
        // on the lane's own cell size (lanes of a warp hold cells of
        // different sizes). Entries past m are stale but in bounds, and are
        // masked out.
#pragma unroll
        for (int k = 0; k < CAP; ++k) {
            const bool live = k < m;
            const float4 c = P.v[k][t];
            const float hk = c.x * fsx + c.y * fsy - hs;
            const float mg = c.z * ns + mr;
            const bool in = live && hk > mg, out = hk < -mg;  // NaN: neither
            mask |= (in ? 1u : 0u) << k;
            undecided |= (live && !in && !out ? 1u : 0u) << k;
            rkeep = (in || !live) ? rkeep : fmaxf(rkeep, c.w);
        }
    } else {
#pragma unroll 4
        for (int k = 0; k < m; ++k) {
            const float4 c = P.v[k][t];
            const float hk = c.x * fsx + c.y * fsy - hs;
            const float mg = c.z * ns + mr;
            const bool in = hk > mg, out = hk < -mg;  // both false also when hk or mg is NaN
            mask |= (in ? 1u : 0u) << k;
            undecided |= (!in && !out ? 1u : 0u) << k;
            rkeep = in ? rkeep : fmaxf(rkeep, c.w);
        }
    }
    if (undecided) {
        if (COUNT) wc.exact += __popc(undecided);
        const int ps = perm[sidx];
        if (pp == -2) pp = perm[p];
        for (unsigned u = undecided; u; u &= u - 1) {
            const int k = __ffs(u) - 1;
            const int4 A = P.q[k][t], Bq = P.q[k + 1 == m ? 0 : k + 1][t];
            if (incircle_exact(A.x, A.y, Bq.x, Bq.y, sx, sy, pp, prio(A.z, perm), prio(Bq.z, perm), ps))
                mask |= 1u << k;
        }
    }
    if (mask == 0) return 0;
    const unsigned full = (1u << m) - 1u;
    const int cnt = __popc(mask);
    const unsigned prevm = ((mask << 1) | (mask >> (m - 1))) & full;
    const unsigned starts = mask & ~prevm;
    if (cnt >= m || __popc(starts) != 1) return ST_RANGE;
    const int i0 = __ffs(starts) - 1;  // first removed vertex; q_i0 is kept
    const int nd = cnt - 1;            // neighbours q_{i0+1..i0+nd} are removed
    if (m - nd + 1 > CAP) return CAP < RCAP ? ST_OVERFLOW : ST_DEGREE;
    PM_CHK(m - nd + 1 <= CAP, 204, return ST_DEGREE)
    const int4 S = make_int4(sx, sy, sidx | (code << 28), 0);
    int ipos;
    if (i0 + nd < m) {
        if (nd == 0) {
            for (int k = m; k > i0 + 1; --k) {
                P.q[k][t] = P.q[k - 1][t];
                P.v[k][t] = P.v[k - 1][t];
            }
            m += 1;
        } else if (nd > 1) {
            for (int k = i0 + 2; k + nd - 1 < m; ++k) {
                P.q[k][t] = P.q[k + nd - 1][t];
                P.v[k][t] = P.v[k + nd - 1][t];
            }
            m -= nd - 1;
        }
        P.q[i0 + 1][t] = S;
        ipos = i0 + 1;
    } else {
        const int dbeg = nd - (m - 1 - i0);
        for (int k = 0; k <= i0 - dbeg; ++k) {
            P.q[k][t] = P.q[k + dbeg][t];
            P.v[k][t] = P.v[k + dbeg][t];
        }
        m = i0 - dbeg + 1;
        P.q[m][t] = S;
        ipos = m;
        m += 1;
    }
    const int iprev = ipos == 0 ? m - 1 : ipos - 1, inext = ipos + 1 == m ? 0 : ipos + 1;
    const int4 Q = P.q[iprev][t], Nq = P.q[inext][t];
    const float r1 = set_vertex(P, iprev, (float)Q.x, (float)Q.y, fsx, fsy);
    const float r2 = set_vertex(P, ipos, fsx, fsy, (float)Nq.x, (float)Nq.y);
    R2 = fmaxf(rkeep, fmaxf(r1, r2));
    if (COUNT) {
        wc.clips++;
        wc.msum += m;
    }
    return 0;
}

// Cell (dx, dy) of the neighbourhood of cell (cx, cy): wrapped index, image offsets.
__device__ __forceinline__ int nb_cell(int cx, int cy, int dx, int dy, int n, int &ox, int &oy) {
    int ux = cx + dx, uy = cy + dy;
    ox = ux < 0 ? -1 : (ux >= n ? 1 : 0);
    oy = uy < 0 ? -1 : (uy >= n ? 1 : 0);
    return (uy - oy * n) * n + (ux - ox * n);
}

// Squared distance from p (offset (fx, fy) inside its cell, torus units) to
// the cell (dx, dy) of its neighbourhood, rounded down a little so that a cell
// is skipped only when every point in it is certainly farther.
__device__ __forceinline__ float box_dist2(int dx, int dy, float fx, float fy, float cw) {
    const float gx = dx > 0 ? (float)dx * cw - fx : (dx < 0 ? fx - (float)(dx + 1) * cw : 0.0f);
    const float gy = dy > 0 ? (float)dy * cw - fy : (dy < 0 ? fy - (float)(dy + 1) * cw : 0.0f);
    return (gx * gx + gy * gy) * 0.99999f;
}

__device__ __forceinline__ void cswap(unsigned &a, unsigned &b) {
    const unsigned lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Ring-1 slot i (0..7) -> cell offset (dx, dy).
__device__ __forceinline__ void ring1(int i, int &dx, int &dy) {
    dx = i < 3 ? i - 1 : (i < 5 ? (i == 3 ? -1 : 1) : i - 6);
    dy = i < 3 ? -1 : (i < 5 ? 0 : 1);
}

// The Voronoi cell (star) of one particle p. Candidates are taken ring by
// ring of cells around p until the cell is certified. A neighbouring cell is
// skipped when its box is farther than 2 max|c_k| (none of its points can cut
// the cell: the same test as for a single candidate), and the eight cells of
// the first ring are visited nearest first, so that the cell shrinks early and
// later candidates fail the distance test. The visiting order does not change
// the result: the Voronoi cell is unique and every decision is exact.
// Returns 0, an error bit, or ST_OVERFLOW when the cell outgrew CAP.
template <int CAP, int NB, bool COUNT>
__device__ __forceinline__ int star_of(PolyS<NB> P, int p, const Geo &g, ll np, const uint2 *__restrict__ pos,
                                       const int *__restrict__ cell_start, const int *__restrict__ perm,
                                       int *__restrict__ nbr, unsigned char *__restrict__ deg,
                                       float *__restrict__ vol, float vol_scale, WorkCount &wc) {
    const int t = P.t;
    const int n = g.n;
    int m = 4;
    // Initial cell: the square cut out by four virtual points at distance
    // B = 2^30, the largest coordinate the exact predicates take. A vertex
    // involving a virtual point is at least 2^29 from p, which the scan
    // (< 2^30) can never certify, so a certified cell is bounded by real
    // particles only; a cell still touching a virtual point after the last
    // ring is reported as ST_SPARSE.
    const int B = 1 << 30;
    const float hb = 0.5f * (float)B;
    const float rb = 2.0f * hb * hb * 1.0001f;
    P.q[0][t] = make_int4(B, 0, PM_VIRT + 0, 0);
    P.q[1][t] = make_int4(0, B, PM_VIRT + 1, 0);
    P.q[2][t] = make_int4(-B, 0, PM_VIRT + 2, 0);
    P.q[3][t] = make_int4(0, -B, PM_VIRT + 3, 0);
    P.v[0][t] = make_float4(hb, hb, 0.0f, rb);
    P.v[1][t] = make_float4(-hb, hb, 0.0f, rb);
    P.v[2][t] = make_float4(-hb, -hb, 0.0f, rb);
    P.v[3][t] = make_float4(hb, -hb, 0.0f, rb);
    float R2 = rb;
    const uint2 Xp = pos[p];
    const int cx = cell_of(Xp.x, n), cy = cell_of(Xp.y, n);
    const float cw = 4294967296.0f / (float)n;
    const float fxl = (float)cell_frac(Xp.x, n) / (float)n, fyl = (float)cell_frac(Xp.y, n) / (float)n;
    const float edge = fminf(fminf(fxl, cw - fxl), fminf(fyl, cw - fyl));
    int pp = -2;  // priority of p, loaded on first exact test
    int rmax = min(PM_RCAP, n / 4 - 1);
    if (rmax < 0) rmax = 0;
    int err = 0;
    bool done = false;
    // Candidates of one neighbouring cell. Differences of torus coordinates
    // in 32-bit arithmetic are the minimal-image offsets (all |.| < 2^31).
    auto scan_cell = [&](int dx, int dy) {
        if (dx != 0 || dy != 0) {
            if (box_dist2(dx, dy, fxl, fyl, cw) > 4.0001f * R2) return;
        }
        int ox, oy, c = nb_cell(cx, cy, dx, dy, n, ox, oy);
        const int code = (ox + 1) * 3 + (oy + 1);
        PM_CHK(c >= 0 && c < g.ncell, 201, return)
        const int s0 = __ldg(cell_start + c), s1 = __ldg(cell_start + c + 1);
        PM_CHK(s0 >= 0 && s1 <= np && s0 <= s1, 202, return)
        for (int s = s0; s < s1; ++s) {
            if (s == p) continue;
            const uint2 Xs = __ldg(pos + s);
            const int rx = (int)(Xs.x - Xp.x), ry = (int)(Xs.y - Xp.y);
            if ((rx | ry) == 0) { err |= ST_DUP; break; }
            if (rx > (1 << 30) || rx < -(1 << 30) || ry > (1 << 30) || ry < -(1 << 30)) continue;
            err |= clip_by<CAP, NB, COUNT>(P, m, R2, rx, ry, s, code, p, pp, perm, wc);
            if (err) break;
        }
    };
    for (int r = 0; r <= rmax && !done && !err; ++r) {
        if (r == 0) {
            scan_cell(0, 0);
        } else if (r == 1) {
            // the eight cells of ring 1 ordered by box distance: keys hold the
            // distance's float bits with the cell's slot in the low 3 bits
            unsigned k[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                int dx, dy;
                ring1(i, dx, dy);
                k[i] = (__float_as_uint(box_dist2(dx, dy, fxl, fyl, cw)) & ~7u) | (unsigned)i;
            }
            // Batcher's odd-even merge sort network for 8 keys (19 exchanges)
            cswap(k[0], k[1]); cswap(k[2], k[3]); cswap(k[4], k[5]); cswap(k[6], k[7]);
            cswap(k[0], k[2]); cswap(k[1], k[3]); cswap(k[4], k[6]); cswap(k[5], k[7]);
            cswap(k[1], k[2]); cswap(k[5], k[6]);
            cswap(k[0], k[4]); cswap(k[1], k[5]); cswap(k[2], k[6]); cswap(k[3], k[7]);
            cswap(k[2], k[4]); cswap(k[3], k[5]);
            cswap(k[1], k[2]); cswap(k[3], k[4]); cswap(k[5], k[6]);
            unsigned order = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) order |= (k[i] & 7u) << (3 * i);
            for (int i = 0; i < 8 && !err; ++i) {
                int dx, dy;
                ring1((order >> (3 * i)) & 7, dx, dy);
                scan_cell(dx, dy);
            }
        } else {
            const int ncells = 8 * r;
            for (int ci = 0; ci < ncells && !err; ++ci) {
                int dx, dy;
                if (ci < 2 * r + 1) { dx = ci - r; dy = -r; }
                else if (ci < 4 * r + 2) { dx = ci - (3 * r + 1); dy = r; }
                else if (ci < 6 * r + 1) { dx = -r; dy = ci - (5 * r + 1); }
                else { dx = r; dy = ci - (7 * r); }
                scan_cell(dx, dy);
            }
        }
        const float dmin = edge + (float)r * cw;
        if (4.0001f * R2 < dmin * dmin) done = true;
    }
    if (err) return err;
    if (!done) return ST_SPARSE;
    for (int k = 0; k < m; ++k)
        if ((P.q[k][t].z & 0x0fffffff) >= PM_VIRT) return ST_SPARSE;
    if (m > PM_MAXDEG) return ST_DEGREE;
    PM_CHK(m >= 3 && m <= PM_MAXDEG, 203, return ST_DEGREE)
    ll area2 = 0;
    int4 A = P.q[0][t];
    for (int k = 0; k < m; ++k) {
        int4 Bq = P.q[k + 1 == m ? 0 : k + 1][t];
        area2 += (ll)A.x * Bq.y - (ll)A.y * Bq.x;
        nbr[(ll)k * np + p] = A.z;
        A = Bq;
    }
    deg[p] = (unsigned char)m;
    vol[p] = (float)area2 * vol_scale;
    return 0;
}

// Work counters 0..4 into wsum[0..4], the give-ups into wsum[over_slot], the
// vertex tests the float filter left to the exact predicate into wsum[7].
template <bool COUNT>
__device__ __forceinline__ void add_counts(const WorkCount &wc, ull *__restrict__ wsum, int over_slot) {
    if (!COUNT) return;
    // warp sums, one atomic per warp and counter
    unsigned v[7] = {wc.cand, wc.tested, wc.vtests, wc.clips, wc.msum, wc.over, wc.exact};
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        unsigned x = v[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(wsum + (i < 5 ? i : (i == 5 ? over_slot : 7)), (ull)x);
    }
}

// Main pass: one thread per particle, polygon capacity DCAP. A particle whose
// cell outgrows it is appended to the retry list (no output written).
// Counters: wsum[0..4] the work of completed cells, wsum[5] the cells given
// up by the main pass, wsum[6] those given up by the first retry pass.
template <bool COUNT>
__global__ void __launch_bounds__(DBLK, 11) k_delaunay(Geo g, ll np, const uint2 *__restrict__ pos,
                                                   const int *__restrict__ cell_start, const int *__restrict__ perm,
                                                   int *__restrict__ nbr, unsigned char *__restrict__ deg,
                                                   float *__restrict__ vol, float vol_scale, int *__restrict__ status,
                                                   int *__restrict__ retry, int *__restrict__ nretry,
                                                   ull *__restrict__ wsum) {
    __shared__ int4 sq[DCAP][DBLK];
    __shared__ float4 sv[DCAP][DBLK];
    const ll pl = (ll)blockIdx.x * DBLK + threadIdx.x;
    WorkCount wc;
    if (pl < np) {
        const int p = (int)pl;
        PolyS<DBLK> P{sq, sv, (int)threadIdx.x};
        const int err = star_of<DCAP, DBLK, COUNT>(P, p, g, np, pos, cell_start, perm, nbr, deg, vol, vol_scale, wc);
        if (err == ST_OVERFLOW) {
            if (COUNT) {
                wc = WorkCount{};
                wc.over = 1;
            }
            const int k = atomicAdd(nretry, 1);
            PM_CHK(k >= 0 && k < np, 205, k = -1)
            if (k >= 0) retry[k] = p;
        } else if (err) {
            atomicOr(status, err & ~ST_OVERFLOW);
            deg[p] = 0;
            vol[p] = 0.0f;
        }
    }
    add_counts<COUNT>(wc, wsum, 5);
}

// Retry passes over the listed particles (grid-stride). The first (capacity
// R1CAP, LAST false) marks a particle whose cell outgrows it by storing ~p in
// its list entry; the last (capacity RCAP, LAST true) takes only the marked
// entries.
template <int CAP, int NB, bool LAST, bool COUNT>
__global__ void __launch_bounds__(NB) k_delaunay_retry(Geo g, ll np, const uint2 *__restrict__ pos,
                                                       const int *__restrict__ cell_start,
                                                       const int *__restrict__ perm, int *__restrict__ nbr,
                                                       unsigned char *__restrict__ deg, float *__restrict__ vol,
                                                       float vol_scale, int *__restrict__ status,
                                                       int *__restrict__ retry, const int *__restrict__ nretry,
                                                       ull *__restrict__ wsum) {
    __shared__ int4 sq[CAP][NB];
    __shared__ float4 sv[CAP][NB];
    const int cnt = *nretry;
    WorkCount wc;
    PolyS<NB> P{sq, sv, (int)threadIdx.x};
    for (ll j = (ll)blockIdx.x * NB + threadIdx.x; j < cnt; j += (ll)gridDim.x * NB) {
        int p = retry[j];
        if (LAST) {
            if (p >= 0) continue;
            p = ~p;
        }
        PM_CHK(p >= 0 && p < np, 206, continue)
        const WorkCount before = wc;
        const int err = star_of<CAP, NB, COUNT>(P, p, g, np, pos, cell_start, perm, nbr, deg, vol, vol_scale, wc);
        if (!LAST && err == ST_OVERFLOW) {
            if (COUNT) {
                wc = before;
                wc.over++;
            }
            retry[j] = ~p;
        } else if (err) {
            atomicOr(status, (err & ~ST_OVERFLOW) | (err == ST_OVERFLOW ? ST_DEGREE : 0));
            deg[p] = 0;
            vol[p] = 0.0f;
        }
    }
    add_counts<COUNT>(wc, wsum, 6);  // the first retry pass's give-ups (none in the last)
}

// Batched passes: the particle's instance comes from the packed offsets; its
// mesh, cell ranges and volume scale from the instance table. Stars hold
// packed sorted indices (< 2^28 in total).
__global__ void __launch_bounds__(DBLK, 11) k_delaunay_b(BTab t, const uint2 *__restrict__ pos,
                                                     const int *__restrict__ cell_start, const int *__restrict__ perm,
                                                     int *__restrict__ nbr, unsigned char *__restrict__ deg,
                                                     float *__restrict__ vol, int *__restrict__ status,
                                                     int *__restrict__ retry, int *__restrict__ nretry) {
    __shared__ int4 sq[DCAP][DBLK];
    __shared__ float4 sv[DCAP][DBLK];
    const ll pl = (ll)blockIdx.x * DBLK + threadIdx.x;
    WorkCount wc;
    if (pl < t.NP) {
        const int p = (int)pl;
        const int k = find_slot(t.poff, t.ninst, pl);
        const Geo g = batch_geo(t, k);
        PolyS<DBLK> P{sq, sv, (int)threadIdx.x};
        const int err = star_of<DCAP, DBLK, false>(P, p, g, t.NP, pos, cell_start + __ldg(t.coff + k), perm, nbr, deg,
                                                   vol, t.inst[k].vol_scale, wc);
        if (err == ST_OVERFLOW) {
            const int j = atomicAdd(nretry, 1);
            PM_CHK(j >= 0 && j < t.NP, 207, j = -1)
            if (j >= 0) retry[j] = p;
        } else if (err) {
            atomicOr(status, err & ~ST_OVERFLOW);
            deg[p] = 0;
            vol[p] = 0.0f;
        }
    }
}

template <int CAP, int NB, bool LAST>
__global__ void __launch_bounds__(NB) k_delaunay_retry_b(BTab t, const uint2 *__restrict__ pos,
                                                         const int *__restrict__ cell_start,
                                                         const int *__restrict__ perm, int *__restrict__ nbr,
                                                         unsigned char *__restrict__ deg, float *__restrict__ vol,
                                                         int *__restrict__ status, int *__restrict__ retry,
                                                         const int *__restrict__ nretry) {
    __shared__ int4 sq[CAP][NB];
    __shared__ float4 sv[CAP][NB];
    const int cnt = *nretry;
    WorkCount wc;
    PolyS<NB> P{sq, sv, (int)threadIdx.x};
    for (ll j = (ll)blockIdx.x * NB + threadIdx.x; j < cnt; j += (ll)gridDim.x * NB) {
        int p = retry[j];
        if (LAST) {
            if (p >= 0) continue;
            p = ~p;
        }
        PM_CHK(p >= 0 && p < t.NP, 208, continue)
        const int k = find_slot(t.poff, t.ninst, (ll)p);
        const Geo g = batch_geo(t, k);
        const int err = star_of<CAP, NB, false>(P, p, g, t.NP, pos, cell_start + __ldg(t.coff + k), perm, nbr, deg,
                                                vol, t.inst[k].vol_scale, wc);
        if (!LAST && err == ST_OVERFLOW) {
            retry[j] = ~p;
        } else if (err) {
            atomicOr(status, (err & ~ST_OVERFLOW) | (err == ST_OVERFLOW ? ST_DEGREE : 0));
            deg[p] = 0;
            vol[p] = 0.0f;
        }
    }
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

void launch_triangulate(const Geo &g, Work &w, ll np, cudaStream_t st, bool count_work) {
    if (np <= 0) return;
    double u = g.L / 4294967296.0;
    float scale = (float)(u * u / 6.0);
    cudaMemsetAsync(w.nretry, 0, sizeof(int), st);
    // w.tmp (caller indices before the canonical cell order) is free after the sort
    // grid-stride passes over the retry list: the first with 17 resident
    // blocks per SM, the last (rare entries) with 8
    const int r1grid = 17 * 152, rgrid = 8 * 152;
    if (count_work) {
        k_delaunay<true><<<div_up(np, DBLK), DBLK, 0, st>>>(g, np, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol,
                                                             scale, w.status, w.tmp, w.nretry, w.wsum);
        k_delaunay_retry<R1CAP, R1BLK, false, true><<<r1grid, R1BLK, 0, st>>>(
            g, np, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol, scale, w.status, w.tmp, w.nretry, w.wsum);
        k_delaunay_retry<RCAP, RBLK, true, true><<<rgrid, RBLK, 0, st>>>(
            g, np, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol, scale, w.status, w.tmp, w.nretry, w.wsum);
    } else {
        k_delaunay<false><<<div_up(np, DBLK), DBLK, 0, st>>>(g, np, w.pos, w.cell_start, w.perm, w.nbr, w.deg,
                                                              w.vol, scale, w.status, w.tmp, w.nretry, nullptr);
        k_delaunay_retry<R1CAP, R1BLK, false, false><<<r1grid, R1BLK, 0, st>>>(
            g, np, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol, scale, w.status, w.tmp, w.nretry, nullptr);
        k_delaunay_retry<RCAP, RBLK, true, false><<<rgrid, RBLK, 0, st>>>(
            g, np, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol, scale, w.status, w.tmp, w.nretry, nullptr);
    }
    count_launches(3);
}

void launch_triangulate_batched(const BTab &t, Work &w, cudaStream_t st) {
    if (t.NP <= 0) return;
    cudaMemsetAsync(w.nretry, 0, sizeof(int), st);
    const int r1grid = 17 * 152, rgrid = 8 * 152;
    k_delaunay_b<<<div_up(t.NP, DBLK), DBLK, 0, st>>>(t, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol, w.status,
                                                       w.tmp, w.nretry);
    k_delaunay_retry_b<R1CAP, R1BLK, false><<<r1grid, R1BLK, 0, st>>>(t, w.pos, w.cell_start, w.perm, w.nbr, w.deg,
                                                                       w.vol, w.status, w.tmp, w.nretry);
    k_delaunay_retry_b<RCAP, RBLK, true><<<rgrid, RBLK, 0, st>>>(t, w.pos, w.cell_start, w.perm, w.nbr, w.deg, w.vol,
                                                                  w.status, w.tmp, w.nretry);
    count_launches(3);
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
