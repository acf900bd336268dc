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
    uint2 Xq = pos[id];
    rx = (ll)Xq.x + (ll)ox * 4294967296LL - (ll)Xp.x;
    ry = (ll)Xq.y + (ll)oy * 4294967296LL - (ll)Xp.y;
}

// Fixed-point exponent of field f: |b_j| <= max|A| h^dim < 2^(60 - E).
__device__ __forceinline__ int fix_exp(const unsigned *maxabs, int f, float hd) {
    float m = __uint_as_float(maxabs[f]) * hd;
    if (!(m > 0.0f)) return 0;
    int e;
    frexpf(m, &e);
    return 60 - e;
}

// Sign of orient(U, V, Q) with Q perturbed by (eps, eps^2) (ties never zero).
__device__ __forceinline__ int orient_pert(ll ux, ll uy, ll vx, ll vy, ll qx, ll qy) {
    i128 o = (i128)(vx - ux) * (qy - uy) - (i128)(vy - uy) * (qx - ux);
    if (o != 0) return o > 0 ? 1 : -1;
    if (vy != uy) return vy > uy ? -1 : 1;
    return vx > ux ? 1 : -1;
}

// ---------------------------------------------------------------------------
// delta assignment
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_delta2d(Geo g, ll np, const uint2 *__restrict__ pos,
                                                 const int *__restrict__ nbr, const unsigned char *__restrict__ deg,
                                                 const float *__restrict__ vals, int F, float *__restrict__ mesh) {
    ll pl = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= np) return;
    const int p = (int)pl, n = g.n, m = deg[p];
    if (m < 3) return;
    const uint2 Xp = pos[p];
    const ll Xn = (ll)Xp.x * n, Yn = (ll)Xp.y * n;
    const float sc = (float)n * 2.3283064365386963e-10f;  // torus units -> cell units
    int ida;
    ll ax, ay;
    rel_of(nbr[(ll)(m - 1) * np + p], Xp, pos, ida, ax, ay);
    for (int k = 0; k < m; ++k) {
        int idb;
        ll bx, by;
        rel_of(nbr[(ll)k * np + p], Xp, pos, idb, bx, by);
        // triangle (p, a, b) with a = q_{k-1}, b = q_k; owned by its lowest sorted index
        if (ida > p && idb > p) {
            const ll Ax = ax * n, Ay = ay * n, Bx = bx * n, By = by * n;
            ll xlo = min(0LL, min(Ax, Bx)) + Xn, xhi = max(0LL, max(Ax, Bx)) + Xn;
            ll ylo = min(0LL, min(Ay, By)) + Yn, yhi = max(0LL, max(Ay, By)) + Yn;
            ll i0 = -((-xlo) >> 32), i1 = xhi >> 32, j0 = -((-ylo) >> 32), j1 = yhi >> 32;
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
                    for (int f = 0; f < F; ++f) {
                        const float *v = vals + (ll)f * np;
                        mesh[(ll)f * g.ncell + node] = lp * v[p] + la * v[ida] + lb * v[idb];
                    }
                }
        }
        ida = idb;
        ax = bx;
        ay = by;
    }
}

// 1D: node i lies between the last particle at or left of it and the next one.
__global__ void k_delta1d(Geo g, ll np, const uint2 *__restrict__ pos, const int *__restrict__ cell_start,
                          const float *__restrict__ vals, int F, float *__restrict__ mesh) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = g.n;
    if (i >= n) return;
    const ull node = (ull)i << 32;  // node position times n
    // last sorted particle with X n <= i 2^32
    ll s = -1;
    int c = i, steps = 0;
    {
        int e = cell_start[c + 1];
        for (int t = cell_start[c]; t < e; ++t)
            if ((ull)pos[t].x * (ull)n <= node) s = t;
    }
    while (s < 0 && steps < n) {
        c = c == 0 ? n - 1 : c - 1;
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
            w[0] = (1.0f - sx) * (1.0f - ty);
            w[1] = sx * (1.0f - ty);
            w[NC - 2] = (1.0f - sx) * ty;
            w[NC - 1] = sx * ty;
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

template <int DIM>
__global__ void k_flip_nodes(Geo g, int F, const float *__restrict__ part, float *__restrict__ mesh,
                             float *__restrict__ node_vol, int *__restrict__ empty) {
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
            mesh[(ll)f * g.ncell + i] = d != 0.0f ? num.get() / d : 0.0f;
        }
    }
    e = __syncthreads_count(e);
    if (threadIdx.x == 0 && e) atomicAdd(empty, e);
}

// ---------------------------------------------------------------------------
// mass right-hand side, exact
// ---------------------------------------------------------------------------

// Sutherland-Hodgman clip of a convex polygon (in place into out) against
// the half plane  sgn * (coord) <= lim  (coord = x if ax == 0 else y).
__device__ __forceinline__ int clip_poly(const float *xi, const float *yi, int m, int axis, float sgn, float lim,
                                         float *xo, float *yo) {
    int k = 0;
    for (int a = 0; a < m; ++a) {
        int b = a + 1 == m ? 0 : a + 1;
        float da = sgn * (axis == 0 ? xi[a] : yi[a]) - lim;
        float db = sgn * (axis == 0 ? xi[b] : yi[b]) - lim;
        if (da <= 0.0f) { xo[k] = xi[a]; yo[k] = yi[a]; ++k; }
        if ((da < 0.0f && db > 0.0f) || (da > 0.0f && db < 0.0f)) {
            float t = da / (da - db);
            xo[k] = fmaf(t, xi[b] - xi[a], xi[a]);
            yo[k] = fmaf(t, yi[b] - yi[a], yi[a]);
            ++k;
        }
    }
    return k;
}

// Moments int s^a t^b over a counter-clockwise polygon by Green's theorem
// (edge sums of the cross term c_k times binomial vertex polynomials).
// M = {M00, M10, M01, M20, M11, M02, M21, M12}
__device__ __forceinline__ void poly_moments(const float *x, const float *y, int m, float M[8]) {
    float a0 = 0, a10 = 0, a01 = 0, a20 = 0, a11 = 0, a02 = 0, a21 = 0, a12 = 0;
    for (int k = 0; k < m; ++k) {
        int l = k + 1 == m ? 0 : k + 1;
        float x0 = x[k], y0 = y[k], x1 = x[l], y1 = y[l];
        float c = x0 * y1 - x1 * y0;
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
    M[0] = a0 * 0.5f;
    M[1] = a10 * (1.0f / 6.0f);
    M[2] = a01 * (1.0f / 6.0f);
    M[3] = a20 * (1.0f / 12.0f);
    M[4] = a11 * (1.0f / 24.0f);
    M[5] = a02 * (1.0f / 12.0f);
    M[6] = a21 * (1.0f / 60.0f);
    M[7] = a12 * (1.0f / 60.0f);
}

__global__ void __launch_bounds__(128) k_rhs2d(Geo g, ll np, const uint2 *__restrict__ pos,
                                               const int *__restrict__ nbr, const unsigned char *__restrict__ deg,
                                               const float *__restrict__ vals, int F,
                                               const unsigned *__restrict__ maxabs, ll *__restrict__ bfix) {
    ll pl = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= np) return;
    const int p = (int)pl, n = g.n, m = deg[p];
    if (m < 3) return;
    const float hd = g.h * g.h;
    int E[PM_MAXF];
    for (int f = 0; f < F; ++f) E[f] = fix_exp(maxabs, f, hd);
    const uint2 Xp = pos[p];
    const int cxp = cell_of(Xp.x, n), cyp = cell_of(Xp.y, n);
    const float up = frac_f(Xp.x, n), wp = frac_f(Xp.y, n);
    const float sc = (float)n * 2.3283064365386963e-10f;
    float Ap[PM_MAXF];
    for (int f = 0; f < F; ++f) Ap[f] = vals[(ll)f * np + p];
    int ida;
    ll ax, ay;
    rel_of(nbr[(ll)(m - 1) * np + p], Xp, pos, ida, ax, ay);
    for (int k = 0; k < m; ++k) {
        int idb;
        ll bx, by;
        rel_of(nbr[(ll)k * np + p], Xp, pos, idb, bx, by);
        if (ida > p && idb > p) {
            // triangle in cell units relative to p's cell corner
            float tx[3] = {up, up + (float)ax * sc, up + (float)bx * sc};
            float ty[3] = {wp, wp + (float)ay * sc, wp + (float)by * sc};
            float e1x = tx[1] - tx[0], e1y = ty[1] - ty[0], e2x = tx[2] - tx[0], e2y = ty[2] - ty[0];
            float det = e1x * e2y - e1y * e2x;
            float ga[PM_MAXF][2];
            for (int f = 0; f < F; ++f) {
                float da = vals[(ll)f * np + ida] - Ap[f], db = vals[(ll)f * np + idb] - Ap[f];
                ga[f][0] = (da * e2y - db * e1y) / det;
                ga[f][1] = (db * e1x - da * e2x) / det;
            }
            int i0 = (int)floorf(fminf(tx[0], fminf(tx[1], tx[2]))), i1 = (int)floorf(fmaxf(tx[0], fmaxf(tx[1], tx[2])));
            int j0 = (int)floorf(fminf(ty[0], fminf(ty[1], ty[2]))), j1 = (int)floorf(fmaxf(ty[0], fmaxf(ty[1], ty[2])));
            for (int cj = j0; cj <= j1; ++cj)
                for (int ci = i0; ci <= i1; ++ci) {
                    float xa[8], ya[8], xb[8], yb[8];
                    for (int v = 0; v < 3; ++v) { xa[v] = tx[v] - (float)ci; ya[v] = ty[v] - (float)cj; }
                    int mm = clip_poly(xa, ya, 3, 0, -1.0f, 0.0f, xb, yb);
                    mm = clip_poly(xb, yb, mm, 0, 1.0f, 1.0f, xa, ya);
                    mm = clip_poly(xa, ya, mm, 1, -1.0f, 0.0f, xb, yb);
                    mm = clip_poly(xb, yb, mm, 1, 1.0f, 1.0f, xa, ya);
                    if (mm < 3) continue;
                    const float s0 = xa[0], t0 = ya[0];
                    for (int v = 0; v < mm; ++v) { xb[v] = xa[v] - s0; yb[v] = ya[v] - t0; }
                    float M[8];
                    poly_moments(xb, yb, mm, M);
                    if (!(M[0] > 0.0f)) continue;
                    // corners (bx, by): psi = phi_bx(s) phi_by(t), phi_0 = 1 - s, phi_1 = s
                    float K[4][3];
                    for (int c = 0; c < 4; ++c) {
                        float A1 = (c & 1) ? s0 : 1.0f - s0, B1 = (c & 1) ? 1.0f : -1.0f;
                        float A2 = (c & 2) ? t0 : 1.0f - t0, B2 = (c & 2) ? 1.0f : -1.0f;
                        float aa = A1 * A2, ab = A1 * B2, ba = B1 * A2, bb = B1 * B2;
                        K[c][0] = aa * M[0] + ab * M[2] + ba * M[1] + bb * M[4];
                        K[c][1] = aa * M[1] + ab * M[4] + ba * M[3] + bb * M[6];
                        K[c][2] = aa * M[2] + ab * M[5] + ba * M[4] + bb * M[7];
                    }
                    const int gx0 = wrapi(cxp + ci, n), gy0 = wrapi(cyp + cj, n);
                    const int gx1 = gx0 + 1 == n ? 0 : gx0 + 1, gy1 = gy0 + 1 == n ? 0 : gy0 + 1;
                    const ll nodes[4] = {(ll)gy0 * n + gx0, (ll)gy0 * n + gx1, (ll)gy1 * n + gx0, (ll)gy1 * n + gx1};
                    const float dsx = s0 + (float)ci - up, dty = t0 + (float)cj - wp;
                    for (int f = 0; f < F; ++f) {
                        float al = Ap[f] + ga[f][0] * dsx + ga[f][1] * dty;  // A at the polygon's first vertex
                        for (int c = 0; c < 4; ++c) {
                            float val = (al * K[c][0] + ga[f][0] * K[c][1] + ga[f][1] * K[c][2]) * hd;
                            ll iv = __float2ll_rn(ldexpf(val, E[f]));
                            if (iv) atomicAdd((ull *)&bfix[(ll)f * g.ncell + nodes[c]], (ull)iv);
                        }
                    }
                }
        }
        ida = idb;
        ax = bx;
        ay = by;
    }
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

__global__ void k_fix_to_float(Geo g, int F, const ll *__restrict__ bfix, const unsigned *__restrict__ maxabs,
                               float *__restrict__ out) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell * F) return;
    int f = (int)(i / g.ncell);
    float hd = g.dim == 2 ? g.h * g.h : g.h;
    out[i] = ldexpf((float)bfix[i], -fix_exp(maxabs, f, hd));
}

// Per-block sums of v_mu A_mu and v_mu |A_mu| (FP64 across threads).
__global__ void __launch_bounds__(256) k_psum(ll np, const float *__restrict__ vals, const float *__restrict__ vol,
                                              int F, double *__restrict__ out, int nblk) {
    __shared__ double sh[2 * PM_MAXF][8];
    for (int f = 0; f < F; ++f) {
        Dot2 a, b;
        for (ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x; s < np; s += (ll)gridDim.x * blockDim.x) {
            float v = vol[s], x = vals[(ll)f * np + s];
            a.fma_acc(v, x);
            b.fma_acc(v, fabsf(x));
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

}  // namespace

void launch_delta(const Geo &g, Work &w, ll np, int F, float *mesh_out, cudaStream_t st) {
    if (g.dim == 2)
        k_delta2d<<<div_up(np, 128), 128, 0, st>>>(g, np, w.pos, w.nbr, w.deg, w.vals, F, mesh_out);
    else
        k_delta1d<<<div_up(g.n, 128), 128, 0, st>>>(g, np, w.pos, w.cell_start, w.vals, F, mesh_out);
    count_launches(1);
}

void launch_flip(const Geo &g, Work &w, ll np, int F, float *mesh_out, float *node_vol, cudaStream_t st) {
    cudaMemsetAsync(w.empty, 0, sizeof(int), st);
    if (g.dim == 2) {
        k_flip_cells<2><<<div_up(g.ncell, 128), 128, 0, st>>>(g, np, w.cell_start, w.pos, w.vals, w.vol, F, w.part);
        k_flip_nodes<2><<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, w.part, mesh_out, node_vol, w.empty);
    } else {
        k_flip_cells<1><<<div_up(g.ncell, 128), 128, 0, st>>>(g, np, w.cell_start, w.pos, w.vals, w.vol, F, w.part);
        k_flip_nodes<1><<<div_up(g.ncell, 256), 256, 0, st>>>(g, F, w.part, mesh_out, node_vol, w.empty);
    }
    count_launches(2);
}

void launch_rhs(const Geo &g, Work &w, ll np, int F, cudaStream_t st) {
    cudaMemsetAsync(w.bfix, 0, sizeof(ll) * g.ncell * F, st);
    if (np <= 0) return;
    if (g.dim == 2)
        k_rhs2d<<<div_up(np, 128), 128, 0, st>>>(g, np, w.pos, w.nbr, w.deg, w.vals, F, w.maxabs, w.bfix);
    else
        k_rhs1d<<<div_up(np, 128), 128, 0, st>>>(g, np, w.pos, w.vals, F, w.maxabs, w.bfix);
    count_launches(1);
}

void launch_rhs_to_float(const Geo &g, Work &w, int F, float *b_out, cudaStream_t st) {
    k_fix_to_float<<<div_up(g.ncell * F, 256), 256, 0, st>>>(g, F, w.bfix, w.maxabs, b_out);
    count_launches(1);
}

void launch_psum(const Geo &g, Work &w, ll np, int F, cudaStream_t st) {
    (void)g;
    k_psum<<<w.nblk_psum, 256, 0, st>>>(np, w.vals, w.vol, F, w.psum, w.nblk_psum);
    count_launches(1);
}
