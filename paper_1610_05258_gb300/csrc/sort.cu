// Counting sort of particles by mesh cell.
//
// The particles of one cell end up contiguous ("particles around node",
// Sec. 2.3), which every scatter and the triangulation rely on. Order inside a
// cell is canonical: by caller index in 2D, by (torus coordinate, caller
// index) in 1D, so that the sorted array is the periodic particle order that
// defines the 1D hat functions (Sec. 3.1). Arrival slots are taken with
// integer atomics (order-free), then every cell segment is put in canonical
// order, so the result is deterministic.
#include "internal.cuh"

PM_DEBUG_DECL(sort)

namespace {

__global__ void k_key(Geo g, const float *__restrict__ px, const float *__restrict__ py, ll np,
                      uint2 *__restrict__ fx, int *__restrict__ key, int *__restrict__ slot, int *__restrict__ count,
                      int *__restrict__ status) {
    ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    float x = px[k];
    float y = g.dim == 2 ? py[k] : 0.0f;
    if (!isfinite(x) || !isfinite(y)) {
        atomicOr(status, ST_NONFINITE);
        x = 0.0f;
        y = 0.0f;
    }
    uint32_t X = torus_coord(x, g.invL);
    uint32_t Y = g.dim == 2 ? torus_coord(y, g.invL) : 0u;
    int c = cell_of(X, g.n);
    if (g.dim == 2) c += cell_of(Y, g.n) * g.n;
    PM_CHK(c >= 0 && c < g.ncell, 101, return)
    fx[k] = make_uint2(X, Y);
    key[k] = c;
    slot[k] = atomicAdd(&count[c], 1);
}

// Block-wide exclusive scan of 4 values per thread (1024 threads).
__device__ int block_scan4(int v[4], int *sh) {
    int t = v[0] + v[1] + v[2] + v[3];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = t;
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        sh[lane] = wi - w;       // exclusive warp offsets
        if (lane == 31) sh[32] = wi;  // block total
    }
    __syncthreads();
    int base = sh[wid] + inc - t;
    int run = base;
    for (int i = 0; i < 4; ++i) {
        int x = v[i];
        v[i] = run;
        run += x;
    }
    int total = sh[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(1024) k_scan_local(const int *__restrict__ in, ll m, int *__restrict__ out,
                                                     int *__restrict__ bsum) {
    __shared__ int sh[33];
    ll base = (ll)blockIdx.x * 4096 + threadIdx.x * 4;
    int v[4];
    for (int i = 0; i < 4; ++i) v[i] = base + i < m ? in[base + i] : 0;
    int tot = block_scan4(v, sh);
    for (int i = 0; i < 4; ++i)
        if (base + i < m) out[base + i] = v[i];
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(int *__restrict__ bsum, int nb, int *__restrict__ total_out) {
    __shared__ int sh[33];
    int carry = 0;
    for (int c0 = 0; c0 < nb; c0 += 4096) {
        int v[4];
        int base = c0 + threadIdx.x * 4;
        for (int i = 0; i < 4; ++i) v[i] = base + i < nb ? bsum[base + i] : 0;
        int tot = block_scan4(v, sh);
        for (int i = 0; i < 4; ++i)
            if (base + i < nb) bsum[base + i] = v[i] + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int *__restrict__ out, ll m, const int *__restrict__ bsum) {
    ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] += bsum[i / 4096];
}

__global__ void k_place(ll np, const int *__restrict__ key, const int *__restrict__ slot,
                        const int *__restrict__ cell_start, int *__restrict__ tmp) {
    ll k = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    PM_CHK(key[k] >= 0, 102, return)
    PM_CHK((ll)cell_start[key[k]] + slot[k] < np, 103, return)
    tmp[cell_start[key[k]] + slot[k]] = (int)k;
}

// One thread per cell: canonical order of the caller indices inside the cell
// (ascending index in 2D; by coordinate, then index, in 1D).
__global__ void k_canon(Geo g, ll np, const int *__restrict__ cell_start, int *__restrict__ tmp,
                        const uint2 *__restrict__ fx) {
    ll c = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    int s0 = cell_start[c], s1 = cell_start[c + 1];
    PM_CHK(s0 >= 0 && s0 <= s1 && s1 <= np, 104, return)
    for (int i = s0 + 1; i < s1; ++i) {
        int v = tmp[i];
        uint32_t xv = g.dim == 1 ? fx[v].x : 0u;
        int j = i - 1;
        while (j >= s0) {
            int u = tmp[j];
            bool greater;
            if (g.dim == 1) {
                uint32_t xu = fx[u].x;
                greater = xu > xv || (xu == xv && u > v);
            } else {
                greater = u > v;
            }
            if (!greater) break;
            tmp[j + 1] = u;
            --j;
        }
        tmp[j + 1] = v;
    }
}

// One thread per sorted slot and one array per grid row: row 0 gathers the
// positions and the permutation, row 1 + f the values of field f (coalesced
// writes in sorted order; reads at the caller indices, in random order). The
// block scheduler dispatches the rows one after another, so the random reads
// of a row stay within one array, which the L2 holds (a field of 16.8M
// particles is 67 MB), instead of spreading over all arrays at once. Each
// field's row tracks max |A| of that field.
#define GATHER_BLK 256
// row0 = 1 gathers the fields only (grid rows 0..F-1 take rows 1..F), after a
// sort that gathered the positions alone.
__global__ void __launch_bounds__(GATHER_BLK) k_gather(ll np, const int *__restrict__ tmp, const uint2 *__restrict__ fx,
                         const float *__restrict__ vals, int *__restrict__ perm, uint2 *__restrict__ pos,
                         float *__restrict__ vals_s, unsigned *__restrict__ maxabs, int *__restrict__ status,
                         int row0) {
    const ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    const int row = (int)blockIdx.y + row0;
    int idx = -1;
    if (s < np) {
        idx = tmp[s];
        PM_CHK(idx >= 0 && idx < np, 105, idx = -1)
    }
    if (row == 0) {
        if (idx >= 0) {
            perm[s] = idx;
            pos[s] = __ldg(fx + idx);
        }
        return;
    }
    const int f = row - 1;
    float mx = 0.0f;
    bool bad = false;
    if (idx >= 0) {
        const float a = __ldg(vals + (ll)f * np + idx);
        bad = !isfinite(a);
        vals_s[(ll)f * np + s] = a;
        mx = fmaxf(mx, fabsf(a));
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    // block maximum, then one atomic per block, issued only when it raises
    // the stored value (the word every block of the row updates)
    __shared__ float wmax[GATHER_BLK / 32];
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int k = 0; k < GATHER_BLK / 32; ++k) m = fmaxf(m, wmax[k]);
        const unsigned mu = __float_as_uint(m);
        if (m > 0.0f && *(volatile const unsigned *)&maxabs[f] < mu) atomicMax(&maxabs[f], mu);
    }
}

// ---------------------------------------------------------------------------
// Batched: every instance's particles in one packed array (instance k at
// [poff[k], poff[k+1])), cells numbered globally (instance k's cell c at
// coff[k] + c). Cell ranges of consecutive instances follow each other, so one
// scan over all cells gives every instance's cell_start, and the sorted slots
// of instance k are again [poff[k], poff[k+1]).
// ---------------------------------------------------------------------------
__global__ void k_key_b(BTab t, const float *__restrict__ px, const float *__restrict__ py, uint2 *__restrict__ fx,
                        int *__restrict__ key, int *__restrict__ slot, int *__restrict__ count,
                        int *__restrict__ status) {
    const ll j = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= t.NP) return;
    const int k = find_slot(t.poff, t.ninst, j);
    const BInst I = t.inst[k];
    float x = px[j], y = py[j];
    if (!isfinite(x) || !isfinite(y)) {
        atomicOr(status, ST_NONFINITE);
        x = 0.0f;
        y = 0.0f;
    }
    const uint32_t X = torus_coord(x, I.invL), Y = torus_coord(y, I.invL);
    const ll c = __ldg(t.coff + k) + (ll)cell_of(Y, I.n) * I.n + cell_of(X, I.n);
    PM_CHK(c >= 0 && c < t.NC, 106, return)
    fx[j] = make_uint2(X, Y);
    key[j] = (int)c;
    slot[j] = atomicAdd(&count[c], 1);
}

// As k_gather, with max|A| per instance and field (maxabs [ninst][PM_MAXF]):
// a warp whose slots all belong to one instance reduces before its atomic.
__global__ void __launch_bounds__(GATHER_BLK) k_gather_b(BTab t, const int *__restrict__ tmp,
                                                         const uint2 *__restrict__ fx, const float *__restrict__ vals,
                                                         int F, int *__restrict__ perm, uint2 *__restrict__ pos,
                                                         float *__restrict__ vals_s, unsigned *__restrict__ maxabs,
                                                         int *__restrict__ status) {
    const ll np = t.NP;
    ll s = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s < np;
    const int k = find_slot(t.poff, t.ninst, live ? s : np - 1);
    float mx[PM_MAXF];
    for (int f = 0; f < PM_MAXF; ++f) mx[f] = 0.0f;
    bool bad = false;
    if (live) {
        const int idx = tmp[s];
        PM_CHK(idx >= 0 && idx < np, 107, s = np)
        if (s < np) {
            perm[s] = idx;
            pos[s] = __ldg(fx + idx);
            for (int f = 0; f < F; ++f) {
                const float a = __ldg(vals + (ll)f * np + idx);
                if (!isfinite(a)) bad = true;
                vals_s[(ll)f * np + s] = a;
                mx[f] = fabsf(a);
            }
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    const int k0 = __shfl_sync(0xffffffffu, k, 0);
    const bool uniform = __all_sync(0xffffffffu, k == k0);
    for (int f = 0; f < F; ++f) {
        float m = mx[f];
        if (uniform) {
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&maxabs[k0 * PM_MAXF + f], __float_as_uint(m));
        } else if (m > 0.0f) {
            atomicMax(&maxabs[k * PM_MAXF + f], __float_as_uint(m));
        }
    }
}

}  // namespace

void launch_sort_batched(const BTab &t, Work &w, const float *px, const float *py, const float *vals, int F,
                         cudaStream_t st) {
    const ll NC = t.NC, NP = t.NP;
    cudaMemsetAsync(w.count, 0, sizeof(int) * NC, st);
    cudaMemsetAsync(w.maxabs, 0, sizeof(unsigned) * PM_MAXF * t.ninst, st);
    k_key_b<<<div_up(NP, 256), 256, 0, st>>>(t, px, py, w.fx, w.key, w.slot, w.count, w.status);
    const int nb = div_up(NC, 4096);
    k_scan_local<<<nb, 1024, 0, st>>>(w.count, NC, w.cell_start, w.scan_tmp);
    k_scan_top<<<1, 1024, 0, st>>>(w.scan_tmp, nb, w.cell_start + NC);
    k_scan_add<<<div_up(NC, 256), 256, 0, st>>>(w.cell_start, NC, w.scan_tmp);
    k_place<<<div_up(NP, 256), 256, 0, st>>>(NP, w.key, w.slot, w.cell_start, w.tmp);
    Geo all{};
    all.dim = 2;
    all.ncell = NC;  // 2D canonical order inside a cell is by packed index: no geometry needed
    k_canon<<<div_up(NC, 128), 128, 0, st>>>(all, NP, w.cell_start, w.tmp, w.fx);
    k_gather_b<<<div_up(NP, GATHER_BLK), GATHER_BLK, 0, st>>>(t, w.tmp, w.fx, vals, F, w.perm, w.pos, w.vals,
                                                                w.maxabs, w.status);
    count_launches(8);
}

void launch_sort(const Geo &g, Work &w, const float *px, const float *py, ll np, const float *vals, int F,
                 cudaStream_t st) {
    cudaMemsetAsync(w.count, 0, sizeof(int) * g.ncell, st);
    cudaMemsetAsync(w.maxabs, 0, sizeof(unsigned) * PM_MAXF, st);
    if (np > 0) k_key<<<div_up(np, 256), 256, 0, st>>>(g, px, py, np, w.fx, w.key, w.slot, w.count, w.status);
    int nb = div_up(g.ncell, 4096);
    k_scan_local<<<nb, 1024, 0, st>>>(w.count, g.ncell, w.cell_start, w.scan_tmp);
    k_scan_top<<<1, 1024, 0, st>>>(w.scan_tmp, nb, w.cell_start + g.ncell);
    k_scan_add<<<div_up(g.ncell, 256), 256, 0, st>>>(w.cell_start, g.ncell, w.scan_tmp);
    if (np > 0) k_place<<<div_up(np, 256), 256, 0, st>>>(np, w.key, w.slot, w.cell_start, w.tmp);
    if (np > 0) {
        k_canon<<<div_up(g.ncell, 128), 128, 0, st>>>(g, np, w.cell_start, w.tmp, w.fx);
        const dim3 grid((unsigned)div_up(np, GATHER_BLK), 1 + (vals ? F : 0));
        k_gather<<<grid, GATHER_BLK, 0, st>>>(np, w.tmp, w.fx, vals, w.perm, w.pos, w.vals, w.maxabs, w.status, 0);
    }
    count_launches(np > 0 ? 7 : 3);
}

void launch_gather_vals(Work &w, ll np, const float *vals, int F, cudaStream_t st) {
    if (np <= 0 || F <= 0) return;
    const dim3 grid((unsigned)div_up(np, GATHER_BLK), F);
    // caller indices from w.perm (row 0 copied them there; w.tmp may have been
    // reused since, e.g. as the triangulation's retry list); the position
    // row's outputs are not touched by these rows, so none are passed
    k_gather<<<grid, GATHER_BLK, 0, st>>>(np, w.perm, nullptr, vals, nullptr, nullptr, w.vals, w.maxabs, w.status, 1);
    count_launches(1);
}
