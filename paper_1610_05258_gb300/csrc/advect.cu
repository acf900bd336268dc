// Particle advection, the driver step between G2P and P2G in the paper's
// experiments (Sec. 3.1: dx/dt = u constant; Sec. 3.2: rigid rotation;
// Sec. 3.3: particles moved by the interpolated velocity field).
// Positions are updated in place and wrapped into [0, L). The shift and the
// rotation are exact functions of their inputs (FP64 update rounded to the
// float32 state); the midpoint rule runs in FP32.
#include "internal.cuh"

namespace {

__device__ __forceinline__ float wrapL(float x, float L) {
    x -= L * floorf(x / L);
    return x >= L ? x - L : (x < 0.0f ? 0.0f : x);
}

// Exact-update convention of the shift and the rotation: the new position is
// computed in FP64 from the float32 one with the expression order written
// below (each operation rounded once: the _rn intrinsics keep the compiler
// from fusing a multiply into an add), wrapped into [0, L) and rounded to
// float32; a value that rounds to L or above is the torus point 0. The result
// is therefore a plain function of the inputs.
__device__ __forceinline__ float wrap_round(double r, double L) {
    const double k = floor(__ddiv_rn(r, L));
    r = __dsub_rn(r, __dmul_rn(L, k));
    if (r < 0.0) r = __dadd_rn(r, L);
    if (r >= L) r = __dsub_rn(r, L);
    const float f = __double2float_rn(r);
    return (double)f >= L ? 0.0f : f;
}

// Sec. 3.1: r <- r + (dx, dy).
__global__ void k_shift(float *__restrict__ px, float *__restrict__ py, ll np, double dx, double dy, double L,
                        int dim) {
    ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    px[k] = wrap_round(__dadd_rn((double)px[k], dx), L);
    if (dim == 2) py[k] = wrap_round(__dadd_rn((double)py[k], dy), L);
}

// Sec. 3.2: rigid rotation about (cx, cy) by the angle whose cosine and sine
// are c, s:  x' = cx + (c X - s Y),  y' = cy + (s X + c Y),  X = x - cx,
// Y = y - cy.
__global__ void k_rotate(float *__restrict__ px, float *__restrict__ py, ll np, double cx, double cy, double c,
                         double s, double L) {
    ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const double X = __dsub_rn((double)px[k], cx), Y = __dsub_rn((double)py[k], cy);
    const double x = __dadd_rn(cx, __dsub_rn(__dmul_rn(c, X), __dmul_rn(s, Y)));
    const double y = __dadd_rn(cy, __dadd_rn(__dmul_rn(s, X), __dmul_rn(c, Y)));
    px[k] = wrap_round(x, L);
    py[k] = wrap_round(y, L);
}

// Explicit midpoint rule with the mesh velocity: vel holds the particle
// velocity at the current position (the G2P result); the midpoint velocity is
// interpolated from the mesh (Eq. delta2) inside this kernel. Optionally
// scales F particle fields by `factor` (a known decay such as the
// Taylor-Green exp(-2 nu dt)).
template <int DIM>
__global__ void __launch_bounds__(256) k_rk2(Geo g, const float *__restrict__ mesh, const float *__restrict__ vel,
                                             float *__restrict__ px, float *__restrict__ py, ll np, float dt,
                                             float *__restrict__ vals, int F, float factor, int *__restrict__ status) {
    ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const float L = (float)g.L;
    const int n = g.n;
    float x = px[k], y = DIM == 2 ? py[k] : 0.0f;
    float u = vel[k], v = DIM == 2 ? vel[np + k] : 0.0f;
    float xm = wrapL(x + 0.5f * dt * u, L), ym = DIM == 2 ? wrapL(y + 0.5f * dt * v, L) : 0.0f;
    if (!isfinite(xm) || !isfinite(ym)) {
        atomicOr(status, ST_NONFINITE);
        return;
    }
    uint32_t X = torus_coord(xm, g.invL);
    int cx = cell_of(X, n);
    float s = frac_f(X, n);
    int x1 = cx + 1 == n ? 0 : cx + 1;
    float um, vm = 0.0f;
    if (DIM == 1) {
        um = (1.0f - s) * __ldg(mesh + cx) + s * __ldg(mesh + x1);
    } else {
        uint32_t Y = torus_coord(ym, g.invL);
        int cy = cell_of(Y, n);
        float t = frac_f(Y, n);
        int y1 = cy + 1 == n ? 0 : cy + 1;
        const ll i00 = (ll)cy * n + cx, i10 = (ll)cy * n + x1, i01 = (ll)y1 * n + cx, i11 = (ll)y1 * n + x1;
        float w00, w10, w01, w11;
        cell_weights(g.p1 != 0, s, t, w00, w10, w01, w11);
        const float *mu = mesh, *mv = mesh + g.ncell;
        um = w00 * __ldg(mu + i00) + w10 * __ldg(mu + i10) + w01 * __ldg(mu + i01) + w11 * __ldg(mu + i11);
        vm = w00 * __ldg(mv + i00) + w10 * __ldg(mv + i10) + w01 * __ldg(mv + i01) + w11 * __ldg(mv + i11);
    }
    px[k] = wrapL(x + dt * um, L);
    if (DIM == 2) py[k] = wrapL(y + dt * vm, L);
    for (int f = 0; f < F; ++f) vals[(ll)f * np + k] *= factor;
}

}  // namespace

void launch_advect_shift(const Geo &g, float *px, float *py, ll np, double dx, double dy, cudaStream_t st) {
    if (np <= 0) return;
    k_shift<<<div_up(np, 256), 256, 0, st>>>(px, py, np, dx, dy, g.L, g.dim);
    count_launches(1);
}

void launch_advect_rotate(const Geo &g, float *px, float *py, ll np, double cx, double cy, double c, double s,
                          cudaStream_t st) {
    if (np <= 0) return;
    k_rotate<<<div_up(np, 256), 256, 0, st>>>(px, py, np, cx, cy, c, s, g.L);
    count_launches(1);
}

void launch_advect_rk2(const Geo &g, const float *mesh_vel, const float *vel, float *px, float *py, ll np, float dt,
                       float *vals, int F, float factor, int *status, cudaStream_t st) {
    if (np <= 0) return;
    if (g.dim == 1)
        k_rk2<1><<<div_up(np, 256), 256, 0, st>>>(g, mesh_vel, vel, px, py, np, dt, vals, F, factor, status);
    else
        k_rk2<2><<<div_up(np, 256), 256, 0, st>>>(g, mesh_vel, vel, px, py, np, dt, vals, F, factor, status);
    count_launches(1);
}
