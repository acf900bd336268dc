// Internal declarations shared by the CUDA translation units of libpmt.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pmt.h"

#define PM_MAXDEG 24   // Delaunay degree stored per particle
#define PM_MAXW 32     // capacity of the working Voronoi polygon
#define PM_MAXF 8      // fields per call
#define PM_RCAP 12     // rings of cells searched by the triangulation
#define PM_NET_RSCALE 64.0f  // scale of the residual input and of the output of the warm-start network
#define PM_NET_GATE 1e-4     // delta-start relative residual above which a field gets the network's correction

typedef long long ll;
typedef unsigned long long ull;
typedef __int128 i128;

// Device status bits (OR-ed into one word, mapped to pm_status on the host).
enum {
    ST_NONFINITE = 1,
    ST_DUP = 2,
    ST_SPARSE = 4,
    ST_DEGREE = 8,
    ST_NOTCONV = 16,
    ST_TIMEOUT = 32,
    ST_RANGE = 64,
};

// One periodic mesh.
struct Geo {
    int dim;       // 1 or 2
    int n;         // nodes (= cells) per side
    double L;      // box length
    float invL;    // fl32(1/L), defines the torus coordinate
    float h;       // fl32(L/n)
    ll ncell;      // n^dim
    int p1;        // 2D mesh functions: 0 bilinear, 1 P1 on cells split by the (0,0)-(1,1) diagonal
    ll fstride;    // field stride of the [F][...] node arrays a kernel writes (ncell for one mesh; the
                   // packed total for the instances of a batch); 0 reads as ncell
};

__host__ __device__ __forceinline__ ll field_stride(const Geo &g) { return g.fstride ? g.fstride : g.ncell; }

// ---------------------------------------------------------------------------
// Batches of independent 2D instances packed into one workspace: instance k
// owns the particle slots [poff[k], poff[k+1]) and the cells/nodes
// [coff[k], coff[k+1]) of the packed arrays; node arrays are [F][NC] and
// particle arrays [F][NP] over all instances.
// ---------------------------------------------------------------------------
struct BInst {
    int n;            // nodes per side
    float invL, h;    // fl32(1/L), fl32(L/n)
    double L;
    float vol_scale;  // (L / 2^32)^2 / 6: particle volume per unit of twice the star area
};
struct BTab {
    const BInst *inst;  // [ninst] (device)
    const ll *poff;     // [ninst + 1] packed particle offsets (device)
    const ll *coff;     // [ninst + 1] packed cell offsets (device)
    int ninst;
    ll NP, NC;
};

// Largest k in [0, m) with off[k] <= x (off ascending, off[0] = 0).
__device__ __forceinline__ int find_slot(const ll *__restrict__ off, int m, ll x) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int find_slot(const int *__restrict__ off, int m, int x) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The mesh of instance k as a Geo whose node arrays use the packed stride NC.
__device__ __forceinline__ Geo batch_geo(const BTab &t, int k) {
    const BInst I = t.inst[k];
    Geo g;
    g.dim = 2;
    g.n = I.n;
    g.L = I.L;
    g.invL = I.invL;
    g.h = I.h;
    g.ncell = (ll)I.n * I.n;
    g.p1 = 0;
    g.fstride = t.NC;
    return g;
}

// Exponent E of the 64-bit fixed point in which the right-hand side of a
// field with max|A| = amax is accumulated: |b_j| <= amax h^dim < 2^(60 - E).
// Capped so that h^dim 2^E stays below 2^120, a finite float scale; the cap
// binds only for amax below about 2^-60, where over 40 bits of the fixed
// point remain in use. Every producer and reader of the fixed point uses it.
__device__ __forceinline__ int fixed_point_exp(float amax, float hd) {
    const float m = amax * hd;
    if (!(m > 0.0f)) return 0;
    int e, eh;
    frexpf(m, &e);
    frexpf(hd, &eh);
    return min(60 - e, 120 - eh);
}

// The four mesh functions non-zero on a 2D cell at local (s, t), corner order
// (0,0), (1,0), (0,1), (1,1): bilinear, or P1 on the triangles s >= t and
// s <= t of the cell's (0,0)-(1,1) diagonal (barycentric coordinates of their
// corners; the fourth corner's hat is zero there).
__device__ __forceinline__ void cell_weights(bool p1, float s, float t, float &w00, float &w10, float &w01,
                                             float &w11) {
    if (!p1) {
        w00 = (1.0f - s) * (1.0f - t);
        w10 = s * (1.0f - t);
        w01 = (1.0f - s) * t;
        w11 = s * t;
    } else if (s >= t) {
        w00 = 1.0f - s;
        w10 = s - t;
        w01 = 0.0f;
        w11 = t;
    } else {
        w00 = 1.0f - t;
        w10 = 0.0f;
        w01 = t - s;
        w11 = s;
    }
}

// Device workspace of a context (all sized at creation).
struct Work {
    ll np_max;
    int F_max;
    // sort
    uint2 *fx;          // torus coordinates, caller order
    int *key, *slot;    // cell and arrival slot, caller order
    int *count;         // [ncell] particles per cell
    int *cell_start;    // [ncell + 1]
    int *scan_tmp;      // block sums of the scan
    int *tmp;           // caller indices placed by cell, before canonical order
    int *perm;          // sorted slot -> caller index
    uint2 *pos;         // torus coordinates, sorted
    float *vals;        // [F][np] particle fields, sorted
    unsigned *maxabs;   // [F] max |A| bit patterns
    // particle functions
    int *nbr;           // [PM_MAXDEG][np] Delaunay neighbours (sorted index | image code << 28)
    unsigned char *deg; // [np]
    float *vol;         // [np] v_mu, sorted order
    // scatter / rhs
    float *part;        // [4 (F+1)][ncell] per-cell corner partials (FLIP)
    ll *bfix;           // [F][ncell] fixed-point right-hand side
    double *psum;       // [2 F][nblk] per-block particle sums (sum v A, sum v |A|)
    int nblk_psum;
    double *epart;      // [2 PM_MAXF][energy_blocks()] block partials of the stability diagnostics
    // solver
    float *r, *p, *q, *b;  // [F][ncell]
    double *red;           // reduction partials [slots][grid]
    int red_blocks;        // grid capacity of red (blocks per slot); persistent solves never exceed it
    double *scal;          // solver scalars per field
    unsigned *bar;         // grid barrier words (2)
    int *status;           // device status word
    int *hstatus;          // pinned host mirror
    int *empty;            // empty-node counter
    ll *ntri;              // triangle counter
    // learned warm start (2D, n a multiple of 128)
    float *feat;           // [F][2][ncell] network input
    float *corr;           // [F][ncell] network output
    double *hres;          // [PM_MAXF] pinned host: delta-start residual per field (network gating)
    ull *wsum;             // [8] triangulation work counters (counting mode)
    int *nretry;           // particles handed to the triangulation's retry pass
    // mesh -> particle projections (particle-sized, sorted order)
    unsigned *meshmax;     // [PM_MAXF] max |Ab| bit patterns
    float *pc;             // [F][np] right-hand side c
    float *px, *pq;        // [np][W] iterate, M_p p; the solution ends in pq (W = pcg_width(F_max),
                           // fields interleaved; the solve of F fields uses stride pcg_width(F))
    float *prp;            // [2][np][W] D^-1 r and the even iterations' search direction
    float *pp2;            // [np][W] the odd iterations' search direction
    float *r2;             // [F][ncell] second residual buffer of the blocked Chebyshev passes (2D)
    ll *cfix;              // = (ll *)prp: fixed-point c before conversion
    float *pcoef;          // [PM_MAXDEG][np] particle mass matrix rows (2D)
    float *mesh_il;        // [ncell][g2p_width(F_max)] mesh fields interleaved per node (G2P)
};

// ---------------------------------------------------------------------------
// Torus coordinate: X = floor(frac(fl32(x * fl32(1/L))) 2^32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t torus_coord(float x, float invL) {
    float t = __fmul_rn(x, invL);
    float f = __fsub_rn(t, floorf(t));
    if (!(f < 1.0f)) f = 0.0f;
    return (uint32_t)__fmul_rn(f, 4294967296.0f);
}
__device__ __forceinline__ int cell_of(uint32_t X, int n) { return (int)(((ull)X * (ull)n) >> 32); }
__device__ __forceinline__ uint32_t cell_frac(uint32_t X, int n) { return (uint32_t)((ull)X * (ull)n); }
__device__ __forceinline__ float frac_f(uint32_t X, int n) { return (float)cell_frac(X, n) * 2.3283064365386963e-10f; }
__device__ __forceinline__ int wrapi(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

// Accumulators. The library's arithmetic is the compensated one (PM_SUMS
// unset): FP32 values with error-free transformations. Two other builds exist
// only for the precision study of the tests (the build script's variants):
// PM_PLAIN_SUMS accumulates in plain FP32, PM_FP64_SUMS in FP64.
#if defined(PM_PLAIN_SUMS)
struct KSum {
    float s;
    __device__ __forceinline__ KSum() : s(0.f) {}
    __device__ __forceinline__ void add(float x) { s += x; }
    __device__ __forceinline__ float get() const { return s; }
};
struct Dot2 {
    float hi, lo;
    __device__ __forceinline__ Dot2() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ void fma_acc(float a, float b) { hi = fmaf(a, b, hi); }
    __device__ __forceinline__ void add(float a) { hi += a; }
};
#elif defined(PM_FP64_SUMS)
struct KSum {
    double s;
    __device__ __forceinline__ KSum() : s(0.0) {}
    __device__ __forceinline__ void add(float x) { s += (double)x; }
    __device__ __forceinline__ float get() const { return (float)s; }
};
struct Dot2 {
    double hi;
    float lo;
    __device__ __forceinline__ Dot2() : hi(0.0), lo(0.f) {}
    __device__ __forceinline__ void fma_acc(float a, float b) { hi = fma((double)a, (double)b, hi); }
    __device__ __forceinline__ void add(float a) { hi += (double)a; }
};
#else
// Compensated (Kahan-Babuska/Neumaier) accumulator in FP32.
struct KSum {
    float s, c;
    __device__ __forceinline__ KSum() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ float get() const { return s + c; }
};

// Error-free product and sum (for compensated dot products).
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// Dot2-style accumulator: sum of products carried as (hi, lo).
struct Dot2 {
    float hi, lo;
    __device__ __forceinline__ Dot2() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ void fma_acc(float a, float b) {
        float p, e, s, e2;
        two_prod(a, b, p, e);
        two_sum(hi, p, s, e2);
        hi = s;
        lo += e + e2;
    }
    __device__ __forceinline__ void add(float a) {
        float s, e;
        two_sum(hi, a, s, e);
        hi = s;
        lo += e;
    }
};

#endif

// Compensated M x at node i of field array xf; returns (hi, lo) of the
// unscaled stencil sum; the caller multiplies by c = h/6, h^2/36 (bilinear)
// or h^2/12 (P1: 6 at the node, 1 at its six neighbours along the cell
// edges and the (0,0)-(1,1) diagonals).
template <int DIM, int P1 = 0>
__device__ __forceinline__ void stencil(const float *__restrict__ xf, int n, ll i, float &hi, float &lo) {
    Dot2 acc;
    if (DIM == 1) {
        int ix = (int)i, xm = ix == 0 ? n - 1 : ix - 1, xp = ix + 1 == n ? 0 : ix + 1;
        acc.add(4.0f * xf[ix]);
        acc.add(xf[xm]);
        acc.add(xf[xp]);
    } else {
        int ix = (int)(i % n), iy = (int)(i / n);
        int xm = ix == 0 ? n - 1 : ix - 1, xp = ix + 1 == n ? 0 : ix + 1;
        int ym = iy == 0 ? n - 1 : iy - 1, yp = iy + 1 == n ? 0 : iy + 1;
        const float *r0 = xf + (ll)ym * n, *r1 = xf + (ll)iy * n, *r2 = xf + (ll)yp * n;
        if (P1) {
            acc.add(6.0f * r1[ix]);
            acc.add(r1[xm]);
            acc.add(r1[xp]);
            acc.add(r0[ix]);
            acc.add(r2[ix]);
            acc.add(r0[xm]);
            acc.add(r2[xp]);
        } else {
            acc.add(16.0f * r1[ix]);
            acc.add(4.0f * r1[xm]);
            acc.add(4.0f * r1[xp]);
            acc.add(4.0f * r0[ix]);
            acc.add(4.0f * r2[ix]);
            acc.add(r0[xm]);
            acc.add(r0[xp]);
            acc.add(r2[xm]);
            acc.add(r2[xp]);
        }
    }
    hi = acc.hi;
    lo = acc.lo;
}

// Power of two 2^-ilogb(m) that scales a field of mean absolute value m to
// order one (1 for m = 0).
__device__ __forceinline__ float solve_scale(double m) {
    if (!(m > 0.0)) return 1.0f;
    return ldexpf(1.0f, min(120, max(-120, -ilogb(m))));
}

static inline int div_up(ll a, int b) { return (int)((a + b - 1) / b); }

// Checked build (-DPM_CHECKED, a debugging aid): every data-derived index is
// validated; the first violation's site code is recorded in a per-file
// device word and the access is skipped (`action` is return/continue/break).
#ifdef PM_CHECKED
#define PM_DEBUG_DECL(tu)                                                        \
    static __device__ int pm_dbg_word[2];                                       \
    void pm_dbg_fetch_##tu(int *o) {                                            \
        cudaMemcpyFromSymbol(o, pm_dbg_word, 2 * sizeof(int));                  \
        int z[2] = {0, 0};                                                      \
        cudaMemcpyToSymbol(pm_dbg_word, z, 2 * sizeof(int));                    \
    }
#define PM_CHK(cond, code, action)                   \
    if (!(cond)) {                                   \
        atomicCAS(&pm_dbg_word[0], 0, (code));       \
        atomicAdd(&pm_dbg_word[1], 1);               \
        action;                                      \
    }
#else
#define PM_DEBUG_DECL(tu)
#define PM_CHK(cond, code, action)
#endif

// Process-wide count of kernel launches issued by the library (each launcher
// adds the number of kernels it queued).
void count_launches(int k);

// Launchers (one per translation unit, all asynchronous on `st`).
void launch_sort(const Geo &g, Work &w, const float *px, const float *py, ll np, const float *vals, int F,
                 cudaStream_t st);
// The field rows of the sort's gather alone, for a sort launched with vals =
// NULL (positions and cell order only): sorted values and max|A| per field.
void launch_gather_vals(Work &w, ll np, const float *vals, int F, cudaStream_t st);
// G2P; il is workspace for the mesh fields interleaved per node
// ([n^dim][g2p_width(F)] floats, unused for F = 1).
int g2p_width(int F);
void launch_g2p(const Geo &g, const float *mesh, int F, const float *px, const float *py, ll np, float *out,
                float *il, int *status, cudaStream_t st);
// G2P at the particles of the sort in w.pos (torus coordinates, sorted
// order); out [F][np] in that order. il as for launch_g2p.
void launch_g2p_sorted(const Geo &g, const float *mesh, int F, const uint2 *pos, ll np, float *out, float *il,
                       cudaStream_t st);
void launch_triangulate(const Geo &g, Work &w, ll np, cudaStream_t st, bool count_work = false);
void launch_volumes_1d(const Geo &g, Work &w, ll np, cudaStream_t st);
void launch_delta(const Geo &g, Work &w, ll np, int F, float *mesh_out, cudaStream_t st);
// FLIP (pic_vol = 0: node volumes v_i = sum v_mu psi_i, Eq. FLIP_vol) or PIC
// (pic_vol = h^dim: the mesh volumes v_i = int psi_i of Eq. mesh_v).
void launch_flip(const Geo &g, Work &w, ll np, int F, float *mesh_out, float *node_vol, cudaStream_t st,
                 float pic_vol = 0.0f);
void rhs_prepare_device();
// x = M^-1 b exactly (to ~1e-9) by separable circulant convolutions; tmp is scratch.
void launch_mass_direct(const Geo &g, const float *b, int F, float *x, float *tmp, cudaStream_t st);
void launch_g2p_integral(const Geo &g, Work &w, ll np, int F, const float *mesh, float *c, cudaStream_t st);
void launch_div_vol(ll np, int F, const float *vol, float *c, cudaStream_t st);
void launch_scale(ll m, float s, float *x, cudaStream_t st);
// Full-mass mesh -> particle solve M_p x = c (c sorted, [F][np]); writes the
// solution to out in caller order [F][np], and leaves it in w.pq, sorted and
// interleaved with stride pcg_width(F). 0 or a CUDA error.
int launch_pcg(const Geo &g, Work &w, ll np, int F, const float *c, float *out, double rtol, int max_iter,
               cudaStream_t st);
// Interleaved width of the particle solve's vectors for F fields (2, 4 or PM_MAXF).
int pcg_width(int F);
void launch_rhs(const Geo &g, Work &w, ll np, int F, cudaStream_t st);
void launch_rhs_appb(const Geo &g, Work &w, ll np, int F, cudaStream_t st);
void launch_rhs_to_float(const Geo &g, Work &w, int F, float *b_out, cudaStream_t st);
void launch_mass_apply(const Geo &g, const float *x, int F, float *y, cudaStream_t st);
int launch_cg(const Geo &g, Work &w, int F, const float *b_float, bool b_from_fix, float *x, bool x_has_start,
              double rtol, int max_iter, cudaStream_t st);
int launch_cheb(const Geo &g, Work &w, int F, const float *b_float, bool b_from_fix, float *x, bool x_has_start,
              double rtol, int max_iter, cudaStream_t st);
void launch_scatter_sorted(ll np, const int *perm, const float *src, float *dst, cudaStream_t st);
void launch_export_tris(const Geo &g, Work &w, ll np, int *tri, int *off, ll max_tri, cudaStream_t st);
void launch_psum(const Geo &g, Work &w, ll np, int F, cudaStream_t st);
void launch_features(const Geo &g, Work &w, int F, const float *delta, cudaStream_t st);
// ||b - M delta|| / ||b|| of the delta start per field (from the network's
// input features) into out[F] (device).
void launch_start_resid(const Geo &g, Work &w, int F, double *out, cudaStream_t st);
void launch_apply_correction(const Geo &g, Work &w, int F, float *mesh, cudaStream_t st);
// Stability diagnostics (Eq. stab): int Ab^2 = Ab^T M Ab of mesh [F][n^dim]
// and int A^2 = A^T M_p A of the sorted particle values (value of field f at
// sorted particle s: pvals[f fs + s ss]; pvals may be null) into the report
// slots 6 and 7 of w.scal.
int energy_blocks();
void launch_energies(const Geo &g, Work &w, int F, const float *mesh, ll np, const float *pvals, ll fs, ll ss,
                     cudaStream_t st);
// Batched phases (one launch each over all instances of a BTab; the Work
// holds the packed arrays, sized for NP particles and NC cells).
void launch_sort_batched(const BTab &t, Work &w, const float *px, const float *py, const float *vals, int F,
                         cudaStream_t st);
void launch_triangulate_batched(const BTab &t, Work &w, cudaStream_t st);
// tile_start [ninst + 1]: prefix of the instances' right-hand-side tiles.
int rhs_tile_side();
void launch_delta_batched(const BTab &t, Work &w, int F, float *mesh_out, cudaStream_t st);
void launch_rhs_batched(const BTab &t, Work &w, int F, const int *tile_start, int ntiles, cudaStream_t st);
void launch_rhs_to_float_batched(const BTab &t, Work &w, int F, float *b_out, cudaStream_t st);
// Direct solve per instance: taps [ninst] (device, opaque records of
// direct_taps_bytes() each, written by make_direct_taps), tile_start
// [ninst + 1] prefix of direct_tile_count(n_k).
size_t direct_taps_bytes();
void make_direct_taps(int n, double L, void *out);
int direct_tile_count(int n);
void launch_mass_direct_batched(const BTab &t, const void *taps, const int *tile_start, int ntiles, const float *b,
                                int F, float *x, float *tmp, cudaStream_t st);
void launch_advect_shift(const Geo &g, float *px, float *py, ll np, double dx, double dy, cudaStream_t st);
void launch_advect_rotate(const Geo &g, float *px, float *py, ll np, double cx, double cy, double c, double s,
                          cudaStream_t st);
void launch_advect_rk2(const Geo &g, const float *mesh_vel, const float *vel, float *px, float *py, ll np, float dt,
                       float *vals, int F, float factor, int *status, cudaStream_t st);
