/*
 * FP64 CPU oracle for particle<->mesh field transfer (Duque & Espanol,
 * "Assignment of fields from particles to mesh", arXiv 1610.05258).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no code with the CUDA path.
 *
 * Every routine is written from the paper's definitions, plainly and slowly,
 * in double precision:
 *   - particle interpolant  A(r)  = sum_mu A_mu psi_mu(r)          (Sec. 2, Eq. part_interp)
 *   - mesh interpolant      Ab(r) = sum_i Ab_i psi_i(r)            (Sec. 2, Eq. mesh_interp)
 *   - volumes v_mu = int psi_mu,  v_i = int psi_i                  (Sec. 2.1, Eqs. part_v, mesh_v)
 *   - delta assignment  Ab_i = A(r_i),  G2P  Abb_mu = Ab(r_mu)     (Sec. 2.2, Eqs. delta, delta2)
 *   - FLIP  Ab_i = sum A_mu v_mu psi_i(r_mu) / sum v_mu psi_i(r_mu) (Sec. 2.3, Eqs. PIC, FLIP_vol)
 *   - mass  Ab_i = sum_j m^-1_ij int A psi_j,  m_ij = int psi_i psi_j (Sec. 2.4, Eqs. proj, phi_def)
 * Linear finite elements are used for both particles and mesh (Sec. 3.1,
 * Sec. 3.2): hat functions on the periodically ordered particles in 1D, P1
 * functions on the periodic Delaunay triangulation of the particles in 2D
 * (Sec. 3.2, App. A), and linear (1D) / bilinear (2D) functions on the
 * uniform periodic mesh.
 *
 * Positions: a float coordinate x on a periodic box of length L is read as
 * the 32-bit fixed-point torus coordinate X ~ frac(x/L) * 2^32 (see
 * fixcoord); every geometric decision (cell, ordering, Delaunay predicates)
 * is taken on X, exactly, and the physical position is X * L / 2^32.
 *
 * Parity-unpinned parts are listed in the Python wrapper's docstring.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef long long ll;

#define TWO32 4294967296.0

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EDEGENERATE = 5 };

/* ------------------------------------------------------------------------ */
/* Positions                                                                  */
/* ------------------------------------------------------------------------ */

/* Canonical torus coordinate of a float position x on a box of length L:
 *   t = fl32(x * fl32(1/L))   (one correctly rounded single-precision product)
 *   X = floor((t - floor(t)) * 2^32) mod 2^32
 * t - floor(t) and the scaling by 2^32 are exact in single precision, so X is
 * fully determined by IEEE arithmetic and lies within one float ulp of the
 * exact frac(x/L) 2^32. */
static int fixcoord(float xf, double L, uint32_t *out) {
    if (!isfinite(xf)) return OR_EINVAL;
    volatile float invL = (float)(1.0 / L);
    volatile float t = xf * invL;
    float f = t - floorf(t);
    if (f >= 1.0f) f = 0.0f;
    *out = (uint32_t)(f * 4294967296.0f);
    return OR_OK;
}

int or_fixed_coords(const float *x, ll np, double L, uint32_t *X) {
    for (ll k = 0; k < np; ++k)
        if (fixcoord(x[k], L, &X[k])) return OR_EINVAL;
    return OR_OK;
}

/* cell index floor(X * n / 2^32) and the exact fraction inside the cell */
static int cell_of(uint32_t X, int n) { return (int)(((uint64_t)X * (uint64_t)n) >> 32); }
static double frac_of(uint32_t X, int n) {
    return (double)(((uint64_t)X * (uint64_t)n) & 0xffffffffull) / TWO32;
}

/* ------------------------------------------------------------------------ */
/* Stable ordering of particles by mesh cell (row-major cell, then index)    */
/* ------------------------------------------------------------------------ */

typedef struct { ll key; ll idx; } keyidx;
static int cmp_keyidx(const void *a, const void *b) {
    const keyidx *p = a, *q = b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

/* perm[k] = original index of the k-th particle in (cell, index) order;
 * cell_start[c] = first sorted slot of cell c, cell_start[n^dim] = np. */
int or_sort_by_cell(int dim, int n, double L, const float *px, const float *py, ll np,
                    ll *perm, ll *cell_start) {
    keyidx *k = malloc(sizeof(keyidx) * (np > 0 ? np : 1));
    if (!k) return OR_ENOMEM;
    ll ncell = dim == 1 ? n : (ll)n * n;
    for (ll c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (ll i = 0; i < np; ++i) {
        uint32_t X, Y = 0;
        if (fixcoord(px[i], L, &X) || (dim == 2 && fixcoord(py[i], L, &Y))) { free(k); return OR_EINVAL; }
        ll c = cell_of(X, n);
        if (dim == 2) c += (ll)cell_of(Y, n) * n;
        k[i].key = c; k[i].idx = i;
        cell_start[c + 1]++;
    }
    qsort(k, np, sizeof(keyidx), cmp_keyidx);
    for (ll i = 0; i < np; ++i) perm[i] = k[i].idx;
    for (ll c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    free(k);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Mesh functions, mass matrix and its solution                              */
/* ------------------------------------------------------------------------ */

static int wrapi(ll i, int n) { ll r = i % n; return (int)(r < 0 ? r + n : r); }

/* The four mesh functions that are non-zero on a 2D cell, at local
 * coordinates (s, t) in [0,1]^2, in the corner order (0,0), (1,0), (0,1),
 * (1,1).
 *   Q1 (p1 = 0): bilinear, (1-s)(1-t), s(1-t), (1-s)t, st.
 *   P1 (p1 = 1): the cell is split by its diagonal from (0,0) to (1,1) into
 *     the triangles {(0,0),(1,0),(1,1)} (s >= t) and {(0,0),(1,1),(0,1)}
 *     (s <= t); on each, the hats are the barycentric coordinates of its three
 *     corners and the fourth corner's hat is zero. */
static void cell_hats(int p1, double s, double t, double w[4]) {
    if (!p1) {
        w[0] = (1 - s) * (1 - t); w[1] = s * (1 - t); w[2] = (1 - s) * t; w[3] = s * t;
    } else if (s >= t) {
        w[0] = 1 - s; w[1] = s - t; w[2] = 0.0; w[3] = t;
    } else {
        w[0] = 1 - t; w[1] = 0.0; w[2] = t - s; w[3] = s;
    }
}

/* Linear (1D) / bilinear (2D) hat of node i evaluated at local coordinate s
 * in [0,1) of the cell whose left node is i (s) or i+1 (1-s). */

/* m_ij = int psi_i psi_j (Sec. 2.4), assembled element by element with a
 * Gauss-Legendre rule that is exact for the element products (degree 2 per
 * axis), then applied: y_i = sum_j m_ij x_j. 2D P1 (p1 = 1): each cell is two
 * triangles of area h^2/2 with the P1 element matrix (area/12)(1 + delta_ab). */
void or_mass_apply(int dim, int n, double L, const double *x, int F, double *y, int p1) {
    const double h = L / n;
    const double g[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)}; /* on [0,1], weights 1/2 */
    if (dim == 1) {
        double me[2][2] = {{0, 0}, {0, 0}};
        for (int q = 0; q < 2; ++q) {
            double sh[2] = {1.0 - g[q], g[q]};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) me[a][b] += 0.5 * h * sh[a] * sh[b];
        }
        for (int f = 0; f < F; ++f) {
            const double *xf = x + (ll)f * n;
            double *yf = y + (ll)f * n;
            for (int i = 0; i < n; ++i) yf[i] = 0.0;
            for (int e = 0; e < n; ++e) {
                int nd[2] = {e, wrapi(e + 1, n)};
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) yf[nd[a]] += me[a][b] * xf[nd[b]];
            }
        }
        return;
    }
    double me[4][4];
    memset(me, 0, sizeof(me));
    if (p1) {
        /* corners in cell order (0,0), (1,0), (0,1), (1,1); triangles
         * {0, 1, 3} and {0, 3, 2} */
        const int tv[2][3] = {{0, 1, 3}, {0, 3, 2}};
        for (int e = 0; e < 2; ++e)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) me[tv[e][a]][tv[e][b]] += (0.5 * h * h / 12.0) * (a == b ? 2.0 : 1.0);
    } else for (int qx = 0; qx < 2; ++qx)
        for (int qy = 0; qy < 2; ++qy) {
            double s = g[qx], t = g[qy];
            double sh[4] = {(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t};
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) me[a][b] += 0.25 * h * h * sh[a] * sh[b];
        }
    const ll nn = (ll)n * n;
    for (int f = 0; f < F; ++f) {
        const double *xf = x + f * nn;
        double *yf = y + f * nn;
        for (ll i = 0; i < nn; ++i) yf[i] = 0.0;
        for (int ey = 0; ey < n; ++ey)
            for (int ex = 0; ex < n; ++ex) {
                int x1 = wrapi(ex + 1, n), y1 = wrapi(ey + 1, n);
                ll nd[4] = {(ll)ey * n + ex, (ll)ey * n + x1, (ll)y1 * n + ex, (ll)y1 * n + x1};
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b) yf[nd[a]] += me[a][b] * xf[nd[b]];
            }
    }
}

/* Solve the periodic tridiagonal system  c*(u[i-1] + 4 u[i] + u[i+1]) = r[i]
 * (the 1D mesh mass matrix, c = h/6) by splitting off the two corner entries
 * as a rank-one update and applying the Sherman-Morrison formula around a
 * plain tridiagonal (Thomas) elimination. In-place on a strided vector. */
static void cyclic_mass_solve(int n, double c, double *r, ll stride, double *w) {
    /* A = T + u v^T with u = (gam, 0.., 0, 1), v = (1, 0.., 0, 1/gam), so that
     * T has diagonal 4 except T00 = 4 - gam, T_{n-1,n-1} = 4 - 1/gam. */
    const double gam = -4.0;
    double *diag = w, *z = w + n, *rhs = w + 2 * n, *cp = w + 3 * n;
    for (int i = 0; i < n; ++i) { diag[i] = 4.0; rhs[i] = r[(ll)i * stride] / c; z[i] = 0.0; }
    diag[0] -= gam;
    diag[n - 1] -= 1.0 / gam;
    z[0] = gam;
    z[n - 1] = 1.0;
    /* Thomas forward sweep on both right-hand sides (sub = super = 1). */
    cp[0] = 1.0 / diag[0];
    rhs[0] /= diag[0];
    z[0] /= diag[0];
    for (int i = 1; i < n; ++i) {
        double m = diag[i] - cp[i - 1];
        cp[i] = 1.0 / m;
        rhs[i] = (rhs[i] - rhs[i - 1]) / m;
        z[i] = (z[i] - z[i - 1]) / m;
    }
    for (int i = n - 2; i >= 0; --i) {
        rhs[i] -= cp[i] * rhs[i + 1];
        z[i] -= cp[i] * z[i + 1];
    }
    double vy = rhs[0] + rhs[n - 1] / gam, vz = z[0] + z[n - 1] / gam;
    double fac = vy / (1.0 + vz);
    for (int i = 0; i < n; ++i) r[(ll)i * stride] = rhs[i] - fac * z[i];
}

/* Direct solve of M x = b. In 1D M = (h/6) circ(1,4,1); in 2D the bilinear
 * mass matrix is the tensor product of two such 1D matrices, so the solve is
 * one 1D solve along every row followed by one along every column. */
int or_mass_solve_direct(int dim, int n, double L, const double *b, int F, double *x) {
    const double c = (L / n) / 6.0;
    double *w = malloc(sizeof(double) * 4 * n);
    if (!w) return OR_ENOMEM;
    ll nn = dim == 1 ? n : (ll)n * n;
    for (int f = 0; f < F; ++f) {
        double *xf = x + f * nn;
        memcpy(xf, b + f * nn, sizeof(double) * nn);
        if (dim == 1) {
            cyclic_mass_solve(n, c, xf, 1, w);
        } else {
            for (int j = 0; j < n; ++j) cyclic_mass_solve(n, c, xf + (ll)j * n, 1, w);
            for (int i = 0; i < n; ++i) cyclic_mass_solve(n, c, xf + i, n, w);
        }
    }
    free(w);
    return OR_OK;
}

/* Plain FP64 conjugate gradients on or_mass_apply; used to cross-check the
 * direct solve. Stops when ||b - M x|| <= rtol ||b||. */
int or_mass_solve_cg(int dim, int n, double L, const double *b, int F, double *x, const double *x0,
                     double rtol, int max_iter, int *iters, double *rel_resid, int p1) {
    ll nn = dim == 1 ? n : (ll)n * n;
    double *r = malloc(sizeof(double) * nn * 3);
    if (!r) return OR_ENOMEM;
    double *p = r + nn, *q = r + 2 * nn;
    for (int f = 0; f < F; ++f) {
        const double *bf = b + f * nn;
        double *xf = x + f * nn;
        for (ll i = 0; i < nn; ++i) xf[i] = x0 ? x0[f * nn + i] : 0.0;
        or_mass_apply(dim, n, L, xf, 1, q, p1);
        double bb = 0, rr = 0;
        for (ll i = 0; i < nn; ++i) { r[i] = bf[i] - q[i]; p[i] = r[i]; bb += bf[i] * bf[i]; rr += r[i] * r[i]; }
        int it = 0;
        if (bb == 0.0) { for (ll i = 0; i < nn; ++i) xf[i] = 0.0; rr = 0.0; bb = 1.0; }
        while (it < max_iter && sqrt(rr) > rtol * sqrt(bb)) {
            or_mass_apply(dim, n, L, p, 1, q, p1);
            double pq = 0;
            for (ll i = 0; i < nn; ++i) pq += p[i] * q[i];
            double alpha = rr / pq, rr2 = 0;
            for (ll i = 0; i < nn; ++i) { xf[i] += alpha * p[i]; r[i] -= alpha * q[i]; rr2 += r[i] * r[i]; }
            double beta = rr2 / rr;
            rr = rr2;
            for (ll i = 0; i < nn; ++i) p[i] = r[i] + beta * p[i];
            ++it;
        }
        or_mass_apply(dim, n, L, xf, 1, q, p1);
        double tr = 0;
        for (ll i = 0; i < nn; ++i) tr += (bf[i] - q[i]) * (bf[i] - q[i]);
        if (iters) iters[f] = it;
        if (rel_resid) rel_resid[f] = sqrt(tr) / sqrt(bb);
    }
    free(r);
    return OR_OK;
}

/* G2P (Sec. 2.2, Eq. delta2): Abb_mu = sum_i Ab_i psi_i(r_mu). Only the nodes
 * of the particle's cell have psi_i(r_mu) != 0. */
int or_interpolate(int dim, int n, double L, const double *mesh, int F, const float *px,
                   const float *py, ll np, double *out, int p1) {
    ll nn = dim == 1 ? n : (ll)n * n;
    for (ll k = 0; k < np; ++k) {
        uint32_t X, Y = 0;
        if (fixcoord(px[k], L, &X) || (dim == 2 && fixcoord(py[k], L, &Y))) return OR_EINVAL;
        int cx = cell_of(X, n);
        double s = frac_of(X, n);
        if (dim == 1) {
            for (int f = 0; f < F; ++f)
                out[f * np + k] = mesh[f * nn + cx] * (1 - s) + mesh[f * nn + wrapi(cx + 1, n)] * s;
        } else {
            int cy = cell_of(Y, n);
            double t = frac_of(Y, n);
            int x1 = wrapi(cx + 1, n), y1 = wrapi(cy + 1, n);
            double w[4];
            cell_hats(p1, s, t, w);
            for (int f = 0; f < F; ++f) {
                const double *m = mesh + f * nn;
                out[f * np + k] = m[(ll)cy * n + cx] * w[0] + m[(ll)cy * n + x1] * w[1] +
                                  m[(ll)y1 * n + cx] * w[2] + m[(ll)y1 * n + x1] * w[3];
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 1D particle functions: hats on the periodically ordered particles         */
/* (Sec. 3.1: linear FE, "area weighting").                                   */
/* ------------------------------------------------------------------------ */

typedef struct { uint32_t X; ll idx; } xi1;
static int cmp_xi1(const void *a, const void *b) {
    const xi1 *p = a, *q = b;
    if (p->X != q->X) return p->X < q->X ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

/* Particles ordered by (X, index) around the circle; gap[k] = distance (in
 * fixed-point units) from ordered particle k to ordered particle k+1. */
static int order1d(const float *px, ll np, double L, xi1 **ord, double **gap) {
    if (np < 2) return OR_EINVAL;
    xi1 *o = malloc(sizeof(xi1) * np);
    double *g = malloc(sizeof(double) * np);
    if (!o || !g) { free(o); free(g); return OR_ENOMEM; }
    for (ll k = 0; k < np; ++k) {
        if (fixcoord(px[k], L, &o[k].X)) { free(o); free(g); return OR_EINVAL; }
        o[k].idx = k;
    }
    qsort(o, np, sizeof(xi1), cmp_xi1);
    for (ll k = 0; k + 1 < np; ++k) g[k] = (double)(o[k + 1].X - o[k].X);
    g[np - 1] = TWO32 - (double)(o[np - 1].X - o[0].X);
    *ord = o;
    *gap = g;
    return OR_OK;
}

/* v_mu = int psi_mu = half the distance between the two neighbours (Eq. part_v). */
int or1_particle_volumes(double L, const float *px, ll np, double *v) {
    xi1 *o; double *g;
    int st = order1d(px, np, L, &o, &g);
    if (st) return st;
    double u = L / TWO32;
    for (ll k = 0; k < np; ++k) v[o[k].idx] = 0.5 * (g[k] + g[(k + np - 1) % np]) * u;
    free(o); free(g);
    return OR_OK;
}

/* Value of the particle interpolant A(x) (Eq. part_interp) at the fixed-point
 * position xi = num/den (den = n, num = i * 2^32 for node i): the two ordered
 * particles that bracket xi are found, then A is linear between them. */
static double eval_A1(const xi1 *o, const double *g, ll np, const double *vals, uint64_t num, uint64_t den) {
    /* last ordered particle with X*den <= num */
    ll lo = -1, a = 0, b = np - 1;
    while (a <= b) {
        ll m = (a + b) / 2;
        if ((uint64_t)o[m].X * den <= num) { lo = m; a = m + 1; } else b = m - 1;
    }
    double d;
    ll k;
    if (lo < 0) { k = np - 1; d = ((double)num / den + TWO32) - (double)o[k].X; }
    else { k = lo; d = (double)num / den - (double)o[k].X; }
    ll k1 = (k + 1) % np;
    double w = d / g[k];
    return vals[o[k].idx] * (1 - w) + vals[o[k1].idx] * w;
}

/* delta assignment (Sec. 2.2, Eq. delta): Ab_i = A(x_i). */
int or1_delta(int n, double L, const float *px, ll np, const double *vals, int F, double *mesh) {
    xi1 *o; double *g;
    int st = order1d(px, np, L, &o, &g);
    if (st) return st;
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < n; ++i)
            mesh[(ll)f * n + i] = eval_A1(o, g, np, vals + f * np, (uint64_t)i << 32, (uint64_t)n);
    free(o); free(g);
    return OR_OK;
}

/* FLIP (Sec. 2.3, Eqs. PIC and FLIP_vol) with particle volumes v (caller
 * computed, Eq. part_v). Nodes with no particle in their support get 0. */
int or_flip(int dim, int n, double L, const float *px, const float *py, ll np, const double *vals, int F,
            const double *v, double *mesh, double *node_vol, ll *empty, int p1) {
    ll nn = dim == 1 ? n : (ll)n * n;
    double *num = calloc((size_t)(nn * F + nn), sizeof(double));
    if (!num) return OR_ENOMEM;
    double *den = num + nn * F;
    for (ll k = 0; k < np; ++k) {
        uint32_t X, Y = 0;
        if (fixcoord(px[k], L, &X) || (dim == 2 && fixcoord(py[k], L, &Y))) { free(num); return OR_EINVAL; }
        int cx = cell_of(X, n);
        double s = frac_of(X, n);
        ll nd[4];
        double w[4];
        int m;
        if (dim == 1) {
            nd[0] = cx; nd[1] = wrapi(cx + 1, n); w[0] = 1 - s; w[1] = s; m = 2;
        } else {
            int cy = cell_of(Y, n);
            double t = frac_of(Y, n);
            int x1 = wrapi(cx + 1, n), y1 = wrapi(cy + 1, n);
            nd[0] = (ll)cy * n + cx; nd[1] = (ll)cy * n + x1; nd[2] = (ll)y1 * n + cx; nd[3] = (ll)y1 * n + x1;
            cell_hats(p1, s, t, w);
            m = 4;
        }
        for (int a = 0; a < m; ++a) {
            den[nd[a]] += v[k] * w[a];
            for (int f = 0; f < F; ++f) num[f * nn + nd[a]] += vals[f * np + k] * v[k] * w[a];
        }
    }
    ll e = 0;
    for (ll i = 0; i < nn; ++i) {
        if (den[i] == 0.0) ++e;
        if (node_vol) node_vol[i] = den[i];
        for (int f = 0; f < F; ++f) mesh[f * nn + i] = den[i] != 0.0 ? num[f * nn + i] / den[i] : 0.0;
    }
    if (empty) *empty = e;
    free(num);
    return OR_OK;
}

/* Mass right-hand side b_j = int A(x) psi_j(x) dx (Sec. 2.4, Eq. proj with
 * phi_def), 1D.
 * mode 0 (exact): A is linear between ordered particles and psi_j is linear
 *   inside a mesh element, so the integrand is quadratic on every piece cut
 *   by both particles and nodes; Simpson's rule on each piece is exact.
 * mode 1 (App. B quadrature): on each mesh element A is replaced by the
 *   parabola through its values at the two nodes and the midpoint, and the
 *   overlap integrals of that parabola with the two hats are taken exactly. */
int or1_rhs(int n, double L, const float *px, ll np, const double *vals, int F, int mode, double *b) {
    xi1 *o; double *g;
    int st = order1d(px, np, L, &o, &g);
    if (st) return st;
    const double h = L / n, u = L / TWO32;
    for (ll i = 0; i < (ll)F * n; ++i) b[i] = 0.0;
    if (mode == 1) {
        for (int f = 0; f < F; ++f) {
            const double *vf = vals + f * np;
            for (int e = 0; e < n; ++e) {
                double q0 = eval_A1(o, g, np, vf, (uint64_t)e << 32, (uint64_t)n);
                double qm = eval_A1(o, g, np, vf, ((uint64_t)(2 * e + 1)) << 32, (uint64_t)(2 * n));
                double q1 = eval_A1(o, g, np, vf, (uint64_t)(e + 1 == n ? 0 : e + 1) << 32, (uint64_t)n);
                b[(ll)f * n + e] += h * (q0 + 2 * qm) / 6.0;
                b[(ll)f * n + wrapi(e + 1, n)] += h * (2 * qm + q1) / 6.0;
            }
        }
        free(o); free(g);
        return OR_OK;
    }
    for (ll k = 0; k < np; ++k) {
        ll k1 = (k + 1) % np;
        double xa = (double)o[k].X * u, xb = xa + g[k] * u; /* unwrapped, xb may exceed L */
        if (g[k] == 0.0) continue;
        /* cut [xa, xb] at the mesh nodes inside it; element e = [e h, (e+1) h) */
        ll e = cell_of(o[k].X, n);
        double cur = xa;
        while (cur < xb) {
            double end = (double)(e + 1) * h < xb ? (double)(e + 1) * h : xb;
            int left = wrapi(e, n), right = wrapi(e + 1, n);
            double pts[3] = {cur, 0.5 * (cur + end), end}, wts[3] = {1, 4, 1};
            for (int q = 0; q < 3; ++q) {
                double x = pts[q];
                double la = (xb - x) / (xb - xa);       /* weight of particle k in A */
                double sl = (x - (double)e * h) / h;    /* local coordinate in element */
                double wq = wts[q] * (end - cur) / 6.0;
                for (int f = 0; f < F; ++f) {
                    double A = vals[f * np + o[k].idx] * la + vals[f * np + o[k1].idx] * (1 - la);
                    b[(ll)f * n + left] += wq * A * (1 - sl);
                    b[(ll)f * n + right] += wq * A * sl;
                }
            }
            cur = end;
            ++e;
        }
    }
    free(o); free(g);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 2D particle functions: P1 on the periodic Delaunay triangulation          */
/* (Sec. 3.2 and App. A). Brute force from the definition: (p,a,b) is a       */
/* Delaunay triangle iff its circumcircle contains no other particle.         */
/* ------------------------------------------------------------------------ */

/* Exact predicates on fixed-point coordinates taken relative to the site p
 * (p at the origin); |coordinate| <= 2^30 keeps every product in 128 bits. */
static i128 orient3(ll ax, ll ay, ll bx, ll by, ll cx, ll cy) {
    return (i128)(bx - ax) * (cy - ay) - (i128)(by - ay) * (cx - ax);
}
static int sgn128(i128 v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }

typedef struct { ll x, y; ll idx; int ox, oy; } cand;

/* Is s strictly inside the circle through (p=0, a, b), with (p,a,b)
 * counter-clockwise?  Exact sign of the lifted 4x4 determinant; an exactly
 * cocircular s is decided by symbolic perturbation of the lifted coordinate
 * z_k -> z_k + eps^(rank k), rank = particle index (lower index = larger
 * perturbation): the first point in index order whose cofactor is non-zero
 * fixes the sign. */
static int in_circle(ll pidx, const cand *a, const cand *b, const cand *s) {
    i128 al = (i128)a->x * a->x + (i128)a->y * a->y;
    i128 bl = (i128)b->x * b->x + (i128)b->y * b->y;
    i128 sl = (i128)s->x * s->x + (i128)s->y * s->y;
    i128 det3 = a->x * (b->y * sl - s->y * bl) - a->y * (b->x * sl - s->x * bl) + al * ((i128)b->x * s->y - (i128)b->y * s->x);
    if (det3 != 0) return det3 < 0;
    /* cofactors of the perturbed lifted coordinates */
    struct { ll idx; int sg; } t[4];
    t[0].idx = pidx;   t[0].sg = sgn128(orient3(a->x, a->y, b->x, b->y, s->x, s->y));
    t[1].idx = a->idx; t[1].sg = -sgn128(orient3(0, 0, b->x, b->y, s->x, s->y));
    t[2].idx = b->idx; t[2].sg = sgn128(orient3(0, 0, a->x, a->y, s->x, s->y));
    t[3].idx = s->idx; t[3].sg = -sgn128(orient3(0, 0, a->x, a->y, b->x, b->y));
    for (;;) {
        int best = -1;
        for (int k = 0; k < 4; ++k)
            if (t[k].idx >= 0 && (best < 0 || t[k].idx < t[best].idx)) best = k;
        if (best < 0) return 0;
        if (t[best].sg != 0) return t[best].sg > 0;
        t[best].idx = -1;
    }
}

typedef struct {
    int G;                 /* bucket grid G x G over the torus */
    ll *start, *items;     /* CSR buckets of particle indices  */
    uint32_t *X, *Y;
    ll np;
} buckets;

static void free_buckets(buckets *B) { free(B->start); free(B->items); free(B->X); free(B->Y); }

static int make_buckets(double L, const float *px, const float *py, ll np, buckets *B) {
    memset(B, 0, sizeof(*B));
    B->np = np;
    int G = (int)floor(sqrt((double)np / 4.0));
    if (G < 1) G = 1;
    if (G > 4096) G = 4096;
    B->G = G;
    B->X = malloc(sizeof(uint32_t) * np);
    B->Y = malloc(sizeof(uint32_t) * np);
    B->start = calloc((size_t)G * G + 1, sizeof(ll));
    B->items = malloc(sizeof(ll) * (np > 0 ? np : 1));
    if (!B->X || !B->Y || !B->start || !B->items) { free_buckets(B); return OR_ENOMEM; }
    for (ll k = 0; k < np; ++k)
        if (fixcoord(px[k], L, &B->X[k]) || fixcoord(py[k], L, &B->Y[k])) { free_buckets(B); return OR_EINVAL; }
    for (ll k = 0; k < np; ++k) B->start[(ll)cell_of(B->Y[k], G) * G + cell_of(B->X[k], G) + 1]++;
    for (ll c = 0; c < (ll)G * G; ++c) B->start[c + 1] += B->start[c];
    ll *fill = malloc(sizeof(ll) * (size_t)G * G);
    if (!fill) { free_buckets(B); return OR_ENOMEM; }
    memcpy(fill, B->start, sizeof(ll) * (size_t)G * G);
    for (ll k = 0; k < np; ++k) B->items[fill[(ll)cell_of(B->Y[k], G) * G + cell_of(B->X[k], G)]++] = k;
    free(fill);
    return OR_OK;
}

/* All particles q != p whose minimal-image offset from p lies in the box
 * |dx|,|dy| <= rho (rho <= 2^30, so each particle appears at most once). */
static ll gather_cands(const buckets *B, ll p, ll rho, cand *c, ll cap, int *dup) {
    int G = B->G;
    double cw = TWO32 / G;
    ll span = (ll)ceil((double)rho / cw) + 1;
    int bx = cell_of(B->X[p], G), by = cell_of(B->Y[p], G);
    ll lo_x = -span, hi_x = span, lo_y = -span, hi_y = span;
    if (2 * span + 1 >= G) { lo_x = lo_y = 0; hi_x = hi_y = G - 1; bx = by = 0; }
    ll m = 0;
    *dup = 0;
    for (ll jy = lo_y; jy <= hi_y; ++jy)
        for (ll jx = lo_x; jx <= hi_x; ++jx) {
            ll cidx = (ll)wrapi(by + jy, G) * G + wrapi(bx + jx, G);
            for (ll t = B->start[cidx]; t < B->start[cidx + 1]; ++t) {
                ll q = B->items[t];
                if (q == p) continue;
                ll dx = (ll)(int32_t)(B->X[q] - B->X[p]);
                ll dy = (ll)(int32_t)(B->Y[q] - B->Y[p]);
                if (dx == 0 && dy == 0) { *dup = 1; continue; }
                if (dx > rho || dx < -rho || dy > rho || dy < -rho) continue;
                if (m >= cap) return -1;
                c[m].x = dx; c[m].y = dy; c[m].idx = q;
                c[m].ox = (int)(((ll)B->X[p] + dx - (ll)B->X[q]) / (ll)4294967296LL);
                c[m].oy = (int)(((ll)B->Y[p] + dy - (ll)B->Y[q]) / (ll)4294967296LL);
                ++m;
            }
        }
    return m;
}

/* Delaunay star of particle p: the counter-clockwise cycle of triangles
 * (p, a_k, b_k) with b_k = a_{k+1}. Returns the number of triangles, or <0. */
static int star_of(const buckets *B, ll p, cand *cbuf, ll cap, cand *ta, cand *tb, int maxt) {
    double spacing = TWO32 / sqrt((double)B->np);
    ll rho = (ll)(3.0 * spacing);
    const ll RHO_MAX = (ll)1 << 30;
    if (rho < 16) rho = 16;
    if (rho > RHO_MAX) rho = RHO_MAX;
    for (;;) {
        int dup;
        ll m = gather_cands(B, p, rho, cbuf, cap, &dup);
        if (dup) return -OR_EDEGENERATE;
        if (m < 0) return -OR_ENOMEM;
        int nt = 0, ok = 1;
        for (ll i = 0; i < m && ok; ++i)
            for (ll j = 0; j < m && ok; ++j) {
                if (i == j || orient3(0, 0, cbuf[i].x, cbuf[i].y, cbuf[j].x, cbuf[j].y) <= 0) continue;
                int empty = 1;
                for (ll k = 0; k < m && empty; ++k)
                    if (k != i && k != j && in_circle(p, &cbuf[i], &cbuf[j], &cbuf[k])) empty = 0;
                if (!empty) continue;
                /* the circumcircle must lie inside the searched box */
                double ax = (double)cbuf[i].x, ay = (double)cbuf[i].y, bx = (double)cbuf[j].x, by = (double)cbuf[j].y;
                double d = 2.0 * (ax * by - ay * bx);
                double al = ax * ax + ay * ay, bl = bx * bx + by * by;
                double ux = (by * al - ay * bl) / d, uy = (ax * bl - bx * al) / d;
                double R = sqrt(ux * ux + uy * uy);
                if (fabs(ux) + R > (double)rho - 4.0 || fabs(uy) + R > (double)rho - 4.0) { ok = 0; break; }
                if (nt >= maxt) return -OR_EDEGENERATE;
                ta[nt] = cbuf[i]; tb[nt] = cbuf[j]; ++nt;
            }
        if (ok && nt >= 3) {
            /* the triangles must close into one fan around p */
            int closed = 1;
            for (int k = 0; k < nt && closed; ++k) {
                int na = 0, nb = 0;
                for (int l = 0; l < nt; ++l) { na += ta[l].idx == ta[k].idx; nb += tb[l].idx == ta[k].idx; }
                if (na != 1 || nb != 1) closed = 0;
            }
            if (closed) {
                /* order the fan: start at the triangle with the smallest a index */
                int first = 0;
                for (int k = 1; k < nt; ++k) if (ta[k].idx < ta[first].idx) first = k;
                cand oa[64], ob[64];
                int cur = first, cnt = 0;
                do {
                    oa[cnt] = ta[cur]; ob[cnt] = tb[cur]; ++cnt;
                    int nx = -1;
                    for (int l = 0; l < nt; ++l) if (ta[l].idx == tb[cur].idx) nx = l;
                    cur = nx;
                } while (cur != first && cur >= 0 && cnt < nt);
                if (cnt != nt || cur != first) closed = 0;
                else { memcpy(ta, oa, sizeof(cand) * nt); memcpy(tb, ob, sizeof(cand) * nt); return nt; }
            }
        }
        if (rho >= RHO_MAX) return -OR_EDEGENERATE;
        rho = rho * 3 / 2;
        if (rho > RHO_MAX) rho = RHO_MAX;
    }
}

#define MAXSTAR 64
#define CANDCAP 65536

/* Star of each particle in `which` (all particles if which == NULL):
 *   deg[k]           number of triangles around which[k]
 *   nbr[k*MAXSTAR+t] index of neighbour a_t (counter-clockwise order)
 *   nof[k*MAXSTAR*2+2t..] image offset (ox, oy) of a_t relative to p.      */
int or2_stars(double L, const float *px, const float *py, ll np, const ll *which, ll nwhich,
              int *deg, ll *nbr, int *nof) {
    buckets B;
    int st = make_buckets(L, px, py, np, &B);
    if (st) return st;
    cand *cb = malloc(sizeof(cand) * CANDCAP), ta[MAXSTAR], tb[MAXSTAR];
    if (!cb) { free_buckets(&B); return OR_ENOMEM; }
    ll cnt = which ? nwhich : np;
    for (ll k = 0; k < cnt; ++k) {
        ll p = which ? which[k] : k;
        int nt = star_of(&B, p, cb, CANDCAP, ta, tb, MAXSTAR);
        if (nt < 0) { free(cb); free_buckets(&B); return -nt; }
        deg[k] = nt;
        for (int t = 0; t < nt; ++t) {
            nbr[k * MAXSTAR + t] = ta[t].idx;
            nof[(k * MAXSTAR + t) * 2] = ta[t].ox;
            nof[(k * MAXSTAR + t) * 2 + 1] = ta[t].oy;
        }
    }
    free(cb);
    free_buckets(&B);
    return OR_OK;
}

/* The whole triangulation: every triangle once, listed from its smallest
 * particle index p as (p, a, b) counter-clockwise with the image offsets of
 * a and b relative to p; plus v_mu = int psi_mu = (1/3) area of the star
 * (Eq. part_v for P1 functions). */
int or2_triangulate(double L, const float *px, const float *py, ll np, ll *tri, int *off, ll max_tri,
                    ll *ntri, double *v) {
    buckets B;
    int st = make_buckets(L, px, py, np, &B);
    if (st) return st;
    cand *cb = malloc(sizeof(cand) * CANDCAP), ta[MAXSTAR], tb[MAXSTAR];
    if (!cb) { free_buckets(&B); return OR_ENOMEM; }
    const double u = L / TWO32;
    ll m = 0;
    for (ll p = 0; p < np; ++p) {
        int nt = star_of(&B, p, cb, CANDCAP, ta, tb, MAXSTAR);
        if (nt < 0) { free(cb); free_buckets(&B); return -nt; }
        double area2 = 0.0;
        for (int t = 0; t < nt; ++t) {
            area2 += (double)orient3(0, 0, ta[t].x, ta[t].y, tb[t].x, tb[t].y);
            if (p < ta[t].idx && p < tb[t].idx) {
                if (m >= max_tri) { free(cb); free_buckets(&B); return OR_ENOMEM; }
                tri[3 * m] = p; tri[3 * m + 1] = ta[t].idx; tri[3 * m + 2] = tb[t].idx;
                off[4 * m] = ta[t].ox; off[4 * m + 1] = ta[t].oy; off[4 * m + 2] = tb[t].ox; off[4 * m + 3] = tb[t].oy;
                ++m;
            }
        }
        if (v) v[p] = area2 * 0.5 * u * u / 3.0;
    }
    *ntri = m;
    free(cb);
    free_buckets(&B);
    return OR_OK;
}

/* Physical vertex coordinates of triangle t, unwrapped around its first vertex. */
static void tri_coords(double L, const uint32_t *X, const uint32_t *Y, const ll *tri, const int *off, ll t,
                       double *x, double *y) {
    const double u = L / TWO32;
    for (int k = 0; k < 3; ++k) {
        ll q = tri[3 * t + k];
        int ox = k ? off[4 * t + 2 * (k - 1)] : 0, oy = k ? off[4 * t + 2 * (k - 1) + 1] : 0;
        x[k] = (double)X[q] * u + ox * L;
        y[k] = (double)Y[q] * u + oy * L;
    }
}

static void bary(const double *x, const double *y, double px, double py, double *l) {
    double d = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    l[1] = ((px - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (py - y[0])) / d;
    l[2] = ((x[1] - x[0]) * (py - y[0]) - (px - x[0]) * (y[1] - y[0])) / d;
    l[0] = 1.0 - l[1] - l[2];
}

/* delta assignment in 2D (Eq. delta): Ab_i = A(r_i), A the P1 interpolant on
 * the particle triangulation. Each node takes the value from a triangle that
 * contains it (any one, A is continuous). nodes_per_side = n gives the mesh
 * nodes; the same routine evaluates A on any finer uniform grid. */
int or2_delta(int nside, double L, const float *px, const float *py, ll np, const double *vals, int F,
              const ll *tri, const int *off, ll ntri, double *mesh) {
    uint32_t *X = malloc(sizeof(uint32_t) * np), *Y = malloc(sizeof(uint32_t) * np);
    ll nn = (ll)nside * nside;
    char *seen = calloc((size_t)nn, 1);
    if (!X || !Y || !seen) { free(X); free(Y); free(seen); return OR_ENOMEM; }
    or_fixed_coords(px, np, L, X);
    or_fixed_coords(py, np, L, Y);
    const double h = L / nside;
    for (ll t = 0; t < ntri; ++t) {
        double x[3], y[3], l[3];
        tri_coords(L, X, Y, tri, off, t, x, y);
        double xmin = fmin(x[0], fmin(x[1], x[2])), xmax = fmax(x[0], fmax(x[1], x[2]));
        double ymin = fmin(y[0], fmin(y[1], y[2])), ymax = fmax(y[0], fmax(y[1], y[2]));
        for (ll j = (ll)ceil(ymin / h) - 1; j <= (ll)floor(ymax / h) + 1; ++j)
            for (ll i = (ll)ceil(xmin / h) - 1; i <= (ll)floor(xmax / h) + 1; ++i) {
                bary(x, y, i * h, j * h, l);
                if (l[0] < -1e-12 || l[1] < -1e-12 || l[2] < -1e-12) continue;
                ll node = (ll)wrapi(j, nside) * nside + wrapi(i, nside);
                for (int f = 0; f < F; ++f) {
                    const double *vf = vals + f * np;
                    mesh[f * nn + node] = l[0] * vf[tri[3 * t]] + l[1] * vf[tri[3 * t + 1]] + l[2] * vf[tri[3 * t + 2]];
                }
                seen[node] = 1;
            }
    }
    int st = OR_OK;
    for (ll i = 0; i < nn; ++i) if (!seen[i]) st = OR_EDEGENERATE;
    free(X); free(Y); free(seen);
    return st;
}

/* Sutherland-Hodgman clip of a convex polygon against x*sx + y*sy <= c. */
static int clip_half(const double *px, const double *py, int m, double sx, double sy, double c, double *qx, double *qy) {
    int k = 0;
    for (int i = 0; i < m; ++i) {
        int j = (i + 1) % m;
        double di = px[i] * sx + py[i] * sy - c, dj = px[j] * sx + py[j] * sy - c;
        if (di <= 0) { qx[k] = px[i]; qy[k] = py[i]; ++k; }
        if ((di < 0 && dj > 0) || (di > 0 && dj < 0)) {
            double t = di / (di - dj);
            qx[k] = px[i] + t * (px[j] - px[i]);
            qy[k] = py[i] + t * (py[j] - py[i]);
            ++k;
        }
    }
    return k;
}

/* Degree-3 triangle rule (Hammer-Marlowe-Stroud): weight -27/48 at the
 * centroid, 25/48 at the three points with barycentric (3/5,1/5,1/5). */
static const double HMS_W[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
static const double HMS_L[4][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {0.6, 0.2, 0.2}, {0.2, 0.6, 0.2}, {0.2, 0.2, 0.6}};

/* exposed for the quadrature pin: integral of x^a y^b over a triangle */
double or_tri_monomial(const double *x, const double *y, int a, int b) {
    double area = 0.5 * fabs((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
    double s = 0;
    for (int q = 0; q < 4; ++q) {
        double qx = HMS_L[q][0] * x[0] + HMS_L[q][1] * x[1] + HMS_L[q][2] * x[2];
        double qy = HMS_L[q][0] * y[0] + HMS_L[q][1] * y[1] + HMS_L[q][2] * y[2];
        s += HMS_W[q] * pow(qx, a) * pow(qy, b);
    }
    return area * s;
}

/* Mass right-hand side in 2D, b_j = int A(r) psi_j(r) dr (Eq. proj with
 * phi_def). mode 0 (exact): every particle triangle is clipped against every
 * mesh cell it overlaps; on each piece A is linear and psi_j bilinear, so the
 * integrand has degree 3 and the Hammer-Marlowe-Stroud rule on a fan of the
 * clipped polygon is exact. mode 1 (App. B analogue for bilinear cells): A is
 * sampled on the 3x3 points of every cell (corners, edge midpoints, centre),
 * replaced by its biquadratic interpolant, and the overlap integrals of that
 * interpolant with the four bilinear hats are taken exactly.
 * P1 mesh (p1 = 1, mode 0 only): every clipped polygon is cut again by the
 * cell's diagonal, so that the hats are linear on each part (degree 2). */
int or2_rhs(int n, double L, const float *px, const float *py, ll np, const double *vals, int F,
            const ll *tri, const int *off, ll ntri, int mode, double *b, int p1) {
    const ll nn = (ll)n * n;
    const double h = L / n;
    for (ll i = 0; i < nn * F; ++i) b[i] = 0.0;
    if (mode == 1 && p1) return OR_EINVAL;
    if (mode == 1) {
        ll n2 = (ll)2 * n;
        double *A2 = malloc(sizeof(double) * n2 * n2 * F);
        if (!A2) return OR_ENOMEM;
        int st = or2_delta((int)n2, L, px, py, np, vals, F, tri, off, ntri, A2);
        if (st) { free(A2); return st; }
        const double W[2][3] = {{1.0 / 6, 1.0 / 3, 0.0}, {0.0, 1.0 / 3, 1.0 / 6}};
        for (int f = 0; f < F; ++f)
            for (int ey = 0; ey < n; ++ey)
                for (int ex = 0; ex < n; ++ex)
                    for (int cb = 0; cb < 2; ++cb)
                        for (int ca = 0; ca < 2; ++ca) {
                            double s = 0;
                            for (int be = 0; be < 3; ++be)
                                for (int al = 0; al < 3; ++al)
                                    s += W[ca][al] * W[cb][be] *
                                         A2[f * n2 * n2 + (ll)wrapi(2 * ey + be, (int)n2) * n2 + wrapi(2 * ex + al, (int)n2)];
                            b[f * nn + (ll)wrapi(ey + cb, n) * n + wrapi(ex + ca, n)] += h * h * s;
                        }
        free(A2);
        return OR_OK;
    }
    uint32_t *X = malloc(sizeof(uint32_t) * np), *Y = malloc(sizeof(uint32_t) * np);
    if (!X || !Y) { free(X); free(Y); return OR_ENOMEM; }
    or_fixed_coords(px, np, L, X);
    or_fixed_coords(py, np, L, Y);
    for (ll t = 0; t < ntri; ++t) {
        double x[3], y[3];
        tri_coords(L, X, Y, tri, off, t, x, y);
        double xmin = fmin(x[0], fmin(x[1], x[2])), xmax = fmax(x[0], fmax(x[1], x[2]));
        double ymin = fmin(y[0], fmin(y[1], y[2])), ymax = fmax(y[0], fmax(y[1], y[2]));
        for (ll cy = (ll)floor(ymin / h); cy * h < ymax; ++cy)
            for (ll cx = (ll)floor(xmin / h); cx * h < xmax; ++cx) {
                double ax[16], ay[16], bx[16], by[16];
                int m = 3;
                for (int k = 0; k < 3; ++k) { ax[k] = x[k]; ay[k] = y[k]; }
                m = clip_half(ax, ay, m, -1, 0, -(double)cx * h, bx, by);
                m = clip_half(bx, by, m, 1, 0, (double)(cx + 1) * h, ax, ay);
                m = clip_half(ax, ay, m, 0, -1, -(double)cy * h, bx, by);
                m = clip_half(bx, by, m, 0, 1, (double)(cy + 1) * h, ax, ay);
                if (m < 3) continue;
                ll nd[4] = {(ll)wrapi(cy, n) * n + wrapi(cx, n), (ll)wrapi(cy, n) * n + wrapi(cx + 1, n),
                            (ll)wrapi(cy + 1, n) * n + wrapi(cx, n), (ll)wrapi(cy + 1, n) * n + wrapi(cx + 1, n)};
                for (int half = 0; half < (p1 ? 2 : 1); ++half) {
                    double hx[16], hy[16];
                    int mh = m;
                    if (p1)  /* half 0: s >= t, half 1: s <= t */
                        mh = half == 0 ? clip_half(ax, ay, m, -1, 1, (double)(cy - cx) * h, hx, hy)
                                       : clip_half(ax, ay, m, 1, -1, (double)(cx - cy) * h, hx, hy);
                    else
                        for (int k = 0; k < m; ++k) { hx[k] = ax[k]; hy[k] = ay[k]; }
                    for (int k = 1; k + 1 < mh; ++k) {
                        double fx[3] = {hx[0], hx[k], hx[k + 1]}, fy[3] = {hy[0], hy[k], hy[k + 1]};
                        double area = 0.5 * fabs((fx[1] - fx[0]) * (fy[2] - fy[0]) - (fx[2] - fx[0]) * (fy[1] - fy[0]));
                        for (int q = 0; q < 4; ++q) {
                            double qx = HMS_L[q][0] * fx[0] + HMS_L[q][1] * fx[1] + HMS_L[q][2] * fx[2];
                            double qy = HMS_L[q][0] * fy[0] + HMS_L[q][1] * fy[1] + HMS_L[q][2] * fy[2];
                            double l[3];
                            bary(x, y, qx, qy, l);
                            double psi[4];
                            cell_hats(p1, (qx - cx * h) / h, (qy - cy * h) / h, psi);
                            double w = area * HMS_W[q];
                                for (int f = 0; f < F; ++f) {
                                    const double *vf = vals + f * np;
                                    double A = l[0] * vf[tri[3 * t]] + l[1] * vf[tri[3 * t + 1]] + l[2] * vf[tri[3 * t + 2]];
                                    for (int c = 0; c < 4; ++c) b[f * nn + nd[c]] += w * A * psi[c];
                                }
                        }
                    }
                }
            }
    }
    free(X); free(Y);
    return OR_OK;
}

/* Conservation diagnostics (Sec. 2.1, Eq. cons) in FP64. */
double or_sum_weighted(const double *w, const double *a, ll m) {
    double s = 0;
    for (ll i = 0; i < m; ++i) s += (w ? w[i] : 1.0) * a[i];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Mesh -> particle projections other than delta (Table 1, right column):    */
/*   c_mu = int Ab psi_mu   with Ab(r) = sum_i Ab_i psi_i(r) (mesh interpolant) */
/*   lumped:    Abb_mu = c_mu / v_mu                 (Eq. lumped)             */
/*   full mass: sum_nu m_{mu nu} Abb_nu = c_mu, m_{mu nu} = int psi_mu psi_nu */
/*              (Eq. proj2 with phi_mu from Eq. phi_def on the particles)      */
/* ------------------------------------------------------------------------ */

/* 1D: c_mu over the merged breakpoints of particles and nodes; on each piece
 * the integrand (linear x linear) is integrated by Simpson's rule (exact). */
int or1_g2p_int(int n, double L, const float *px, ll np, const double *mesh, int F, double *c) {
    xi1 *o; double *g;
    int st = order1d(px, np, L, &o, &g);
    if (st) return st;
    const double h = L / n, u = L / TWO32;
    for (ll i = 0; i < (ll)F * np; ++i) c[i] = 0.0;
    for (ll k = 0; k < np; ++k) {
        ll k1 = (k + 1) % np;
        double xa = (double)o[k].X * u, xb = xa + g[k] * u;
        if (g[k] == 0.0) continue;
        ll e = cell_of(o[k].X, n);
        double cur = xa;
        while (cur < xb) {
            double end = (double)(e + 1) * h < xb ? (double)(e + 1) * h : xb;
            int left = wrapi(e, n), right = wrapi(e + 1, n);
            double pts[3] = {cur, 0.5 * (cur + end), end}, wts[3] = {1, 4, 1};
            for (int q = 0; q < 3; ++q) {
                double x = pts[q];
                double la = (xb - x) / (xb - xa);    /* psi of particle k at x */
                double sl = (x - (double)e * h) / h; /* local coordinate in element */
                double wq = wts[q] * (end - cur) / 6.0;
                for (int f = 0; f < F; ++f) {
                    double Ab = mesh[(ll)f * n + left] * (1 - sl) + mesh[(ll)f * n + right] * sl;
                    c[f * np + o[k].idx] += wq * Ab * la;
                    c[f * np + o[k1].idx] += wq * Ab * (1 - la);
                }
            }
            cur = end;
            ++e;
        }
    }
    free(o); free(g);
    return OR_OK;
}

/* 2D: c_mu by clipping every particle triangle against every cell and
 * integrating Ab psi_mu (bilinear x linear, degree 3) with the
 * Hammer-Marlowe-Stroud rule on a fan of each clipped polygon. P1 mesh
 * (p1 = 1): every clipped polygon is cut again by the cell's diagonal. */
int or2_g2p_int(int n, double L, const float *px, const float *py, ll np, const double *mesh, int F,
                const ll *tri, const int *off, ll ntri, double *c, int p1) {
    const ll nn = (ll)n * n;
    const double h = L / n;
    for (ll i = 0; i < (ll)F * np; ++i) c[i] = 0.0;
    uint32_t *X = malloc(sizeof(uint32_t) * np), *Y = malloc(sizeof(uint32_t) * np);
    if (!X || !Y) { free(X); free(Y); return OR_ENOMEM; }
    or_fixed_coords(px, np, L, X);
    or_fixed_coords(py, np, L, Y);
    for (ll t = 0; t < ntri; ++t) {
        double x[3], y[3];
        tri_coords(L, X, Y, tri, off, t, x, y);
        double xmin = fmin(x[0], fmin(x[1], x[2])), xmax = fmax(x[0], fmax(x[1], x[2]));
        double ymin = fmin(y[0], fmin(y[1], y[2])), ymax = fmax(y[0], fmax(y[1], y[2]));
        for (ll cy = (ll)floor(ymin / h); cy * h < ymax; ++cy)
            for (ll cx = (ll)floor(xmin / h); cx * h < xmax; ++cx) {
                double ax[16], ay[16], bx[16], by[16];
                int m = 3;
                for (int k = 0; k < 3; ++k) { ax[k] = x[k]; ay[k] = y[k]; }
                m = clip_half(ax, ay, m, -1, 0, -(double)cx * h, bx, by);
                m = clip_half(bx, by, m, 1, 0, (double)(cx + 1) * h, ax, ay);
                m = clip_half(ax, ay, m, 0, -1, -(double)cy * h, bx, by);
                m = clip_half(bx, by, m, 0, 1, (double)(cy + 1) * h, ax, ay);
                if (m < 3) continue;
                ll nd[4] = {(ll)wrapi(cy, n) * n + wrapi(cx, n), (ll)wrapi(cy, n) * n + wrapi(cx + 1, n),
                            (ll)wrapi(cy + 1, n) * n + wrapi(cx, n), (ll)wrapi(cy + 1, n) * n + wrapi(cx + 1, n)};
                for (int half = 0; half < (p1 ? 2 : 1); ++half) {
                    double hx[16], hy[16];
                    int mh = m;
                    if (p1)  /* half 0: s >= t, half 1: s <= t */
                        mh = half == 0 ? clip_half(ax, ay, m, -1, 1, (double)(cy - cx) * h, hx, hy)
                                       : clip_half(ax, ay, m, 1, -1, (double)(cx - cy) * h, hx, hy);
                    else
                        for (int k = 0; k < m; ++k) { hx[k] = ax[k]; hy[k] = ay[k]; }
                    for (int k = 1; k + 1 < mh; ++k) {
                        double fx[3] = {hx[0], hx[k], hx[k + 1]}, fy[3] = {hy[0], hy[k], hy[k + 1]};
                        double area = 0.5 * fabs((fx[1] - fx[0]) * (fy[2] - fy[0]) - (fx[2] - fx[0]) * (fy[1] - fy[0]));
                        for (int q = 0; q < 4; ++q) {
                            double qx = HMS_L[q][0] * fx[0] + HMS_L[q][1] * fx[1] + HMS_L[q][2] * fx[2];
                            double qy = HMS_L[q][0] * fy[0] + HMS_L[q][1] * fy[1] + HMS_L[q][2] * fy[2];
                            double l[3];
                            bary(x, y, qx, qy, l);
                            double psi[4];
                            cell_hats(p1, (qx - cx * h) / h, (qy - cy * h) / h, psi);
                            double w = area * HMS_W[q];
                                for (int f = 0; f < F; ++f) {
                                    double Ab = 0;
                                    for (int cc = 0; cc < 4; ++cc) Ab += mesh[f * nn + nd[cc]] * psi[cc];
                                    for (int k2 = 0; k2 < 3; ++k2) c[f * np + tri[3 * t + k2]] += w * Ab * l[k2];
                                }
                        }
                    }
                }
            }
    }
    free(X); free(Y);
    return OR_OK;
}

/* Particle mass matrix applied to x ([F][np]):
 *   1D: on each gap g between ordered particles a, b the element matrix
 *       (g/6) [[2, 1], [1, 2]];
 *   2D: on each triangle T the P1 element matrix (|T|/12)(1 + delta_ab). */
int or_particle_mass_apply(int dim, double L, const float *px, const float *py, ll np, const ll *tri,
                           const int *off, ll ntri, const double *x, int F, double *y) {
    for (ll i = 0; i < (ll)F * np; ++i) y[i] = 0.0;
    if (dim == 1) {
        xi1 *o; double *g;
        int st = order1d(px, np, L, &o, &g);
        if (st) return st;
        const double u = L / TWO32;
        for (ll k = 0; k < np; ++k) {
            ll a = o[k].idx, b = o[(k + 1) % np].idx;
            double e = g[k] * u / 6.0;
            for (int f = 0; f < F; ++f) {
                y[f * np + a] += e * (2 * x[f * np + a] + x[f * np + b]);
                y[f * np + b] += e * (x[f * np + a] + 2 * x[f * np + b]);
            }
        }
        free(o); free(g);
        return OR_OK;
    }
    uint32_t *X = malloc(sizeof(uint32_t) * np), *Y = malloc(sizeof(uint32_t) * np);
    if (!X || !Y) { free(X); free(Y); return OR_ENOMEM; }
    or_fixed_coords(px, np, L, X);
    or_fixed_coords(py, np, L, Y);
    for (ll t = 0; t < ntri; ++t) {
        double xs[3], ys[3];
        tri_coords(L, X, Y, tri, off, t, xs, ys);
        double area = 0.5 * fabs((xs[1] - xs[0]) * (ys[2] - ys[0]) - (xs[2] - xs[0]) * (ys[1] - ys[0]));
        for (int f = 0; f < F; ++f) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += x[f * np + tri[3 * t + k]];
            for (int k = 0; k < 3; ++k) y[f * np + tri[3 * t + k]] += area / 12.0 * (s + x[f * np + tri[3 * t + k]]);
        }
    }
    free(X); free(Y);
    return OR_OK;
}

/* Solve M_p x = c (all F fields) by conjugate gradients in FP64 to relative
 * residual rtol, from x = 0. Returns the iterations taken (or < 0). */
int or_particle_mass_solve(int dim, double L, const float *px, const float *py, ll np, const ll *tri,
                           const int *off, ll ntri, const double *c, int F, double rtol, int max_iter, double *x) {
    double *r = malloc(sizeof(double) * np), *p = malloc(sizeof(double) * np), *q = malloc(sizeof(double) * np);
    if (!r || !p || !q) { free(r); free(p); free(q); return -OR_ENOMEM; }
    int worst = 0;
    for (int f = 0; f < F; ++f) {
        double *xf = x + (ll)f * np;
        const double *cf = c + (ll)f * np;
        double bb = 0;
        for (ll i = 0; i < np; ++i) { xf[i] = 0; r[i] = cf[i]; p[i] = cf[i]; bb += cf[i] * cf[i]; }
        double rr = bb;
        int it = 0;
        while (it < max_iter && rr > rtol * rtol * bb && bb > 0) {
            int st = or_particle_mass_apply(dim, L, px, py, np, tri, off, ntri, p, 1, q);
            if (st) { free(r); free(p); free(q); return -st; }
            double pq = 0;
            for (ll i = 0; i < np; ++i) pq += p[i] * q[i];
            double al = rr / pq, rn = 0;
            for (ll i = 0; i < np; ++i) { xf[i] += al * p[i]; r[i] -= al * q[i]; rn += r[i] * r[i]; }
            double be = rn / rr;
            rr = rn;
            for (ll i = 0; i < np; ++i) p[i] = r[i] + be * p[i];
            ++it;
        }
        if (it > worst) worst = it;
    }
    free(r); free(p); free(q);
    return worst;
}
