// Mass solve that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they need a solve:
// host applications and plugin frameworks that own every byte of device
// memory through their own pool and forbid allocations by libraries they
// load, and latency-critical loops that cannot take the implicit device
// synchronisation of cudaMalloc/cudaFree. For them this file provides
// pm_mass_solve_noalloc(): the same conjugate-gradient solve as
// pm_mass_solve(), with its scratch vectors in one file-scope device array of
// fixed size instead of a context's workspace. The caller still passes the
// right-hand side and the output array.
//
// Scratch: PM_NOALLOC_MAX_VALUES floats for each of the four CG vectors
// (r, p, q, b), plus reduction partials for up to PM_NOALLOC_MAX_GRID blocks
// (the solve's grid is clamped to that), solver scalars, the barrier words and
// the status word: about 16.2 MB, held by every GPU that loads the library
// until the process exits. Its device address is looked up once per device
// (cudaGetSymbolAddress) by the first call on that device.
#include <cstring>
#include <mutex>

#include "internal.cuh"

#define PM_NOALLOC_MAX_VALUES (1 << 20)  // F * n^dim
#define PM_NOALLOC_MAX_GRID 1024         // blocks of the persistent solve
#define PM_NOALLOC_MAX_DEV 64

namespace {

constexpr size_t kVecBytes = sizeof(float) * (size_t)PM_NOALLOC_MAX_VALUES;
constexpr size_t kRedOff = 4 * kVecBytes;
constexpr size_t kRedBytes = sizeof(double) * 6 * PM_MAXF * (size_t)PM_NOALLOC_MAX_GRID;
constexpr size_t kScalOff = kRedOff + kRedBytes;
constexpr size_t kScalBytes = sizeof(double) * 16 * PM_MAXF;
constexpr size_t kBarOff = kScalOff + kScalBytes;
constexpr size_t kStatusOff = kBarOff + 256;
constexpr size_t kScratchBytes = kStatusOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_addr[PM_NOALLOC_MAX_DEV] = {nullptr};

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= PM_NOALLOC_MAX_DEV) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" pm_status pm_mass_solve_noalloc(int dim, int n, double L, const float *b, int F, float *x, double rtol,
                                           int max_iter, int use_x0, void *stream, int *iters, double *rel_resid) {
    if ((dim != 1 && dim != 2) || n < 4 || !(L > 0.0) || F < 1 || F > PM_MAXF || !b || !x) return PM_EINVAL;
    const ll nn = dim == 1 ? (ll)n : (ll)n * n;
    if (nn * F > PM_NOALLOC_MAX_VALUES) return PM_EINVAL;
    if (!(rtol > 0.0)) rtol = 1e-6;
    if (max_iter <= 0) max_iter = 200;
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return PM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;

    Geo g{};  // value-initialised: bilinear (p1 = 0)
    g.dim = dim;
    g.n = n;
    g.L = L;
    g.invL = (float)(1.0 / L);
    g.h = (float)(L / n);
    g.ncell = nn;
    Work w;
    memset(&w, 0, sizeof(w));
    w.r = (float *)(base + 0 * kVecBytes);
    w.p = (float *)(base + 1 * kVecBytes);
    w.q = (float *)(base + 2 * kVecBytes);
    w.b = (float *)(base + 3 * kVecBytes);
    w.red = (double *)(base + kRedOff);
    w.red_blocks = PM_NOALLOC_MAX_GRID;  // the solve's grid is clamped to the partials' capacity
    w.scal = (double *)(base + kScalOff);
    w.bar = (unsigned *)(base + kBarOff);
    w.status = (int *)(base + kStatusOff);
    // the status word must start at zero; every other scratch value is
    // written by the solve before it is read
    if (cudaMemsetAsync(w.status, 0, sizeof(int), st) != cudaSuccess) return PM_ECUDA;
    int e = launch_cg(g, w, F, b, false, x, use_x0 != 0, rtol, max_iter, st);
    if (e) return PM_ECUDA;
    if (!iters && !rel_resid) return PM_OK;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PM_ECUDA;
    double sc[16 * PM_MAXF];
    int s = 0;
    if (cudaMemcpy(sc, w.scal, sizeof(double) * 16 * F, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&s, w.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PM_ECUDA;
    for (int f = 0; f < F; ++f) {
        if (iters) iters[f] = (int)sc[16 * f + 0];
        if (rel_resid) rel_resid[f] = sc[16 * f + 2];
    }
    if (s & ST_TIMEOUT) return PM_ETIMEOUT;
    if (s & ST_NOTCONV) return PM_ENOTCONV;
    return PM_OK;
}
