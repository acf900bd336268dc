// Learned warm start for the mass solve (no counterpart in the paper).
//
// A small fully convolutional network on the periodic mesh predicts the mass
// assignment (Sec. 2.4, Eqs. proj and phi_def) from the delta assignment
// (Sec. 2.2, Eq. delta) and the lumped-mass solution b / h^2 (b the exact
// right-hand side of Eq. proj);
// its prediction starts the conjugate-gradient solve, which still finishes to
// the requested residual. Layers: 3x3 periodic convolutions 2 -> 32 -> 32 ->
// 32 -> 1 with bias, ReLU after the first three. Activations are stored in
// BF16 (NHWC, 32 channels = 64 bytes per pixel), products accumulate in FP32.
//
// The two 32 -> 32 layers run on the 5th-generation tensor cores: an implicit
// GEMM per tile of 128 output pixels of one mesh row, M = 128 pixels, N = 32
// output channels, K = 9 taps x 32 input channels = 288 (18 MMAs of K = 16),
// FP32 accumulators in tensor memory. The input rows y-1, y, y+1 of the tile
// (130 pixels each, periodic) are staged in shared memory as planes of 8
// channels x 130 pixels, so that the A operand of tap (dy, dx) is the plane
// of row y+dy shifted by dx pixels: a 16-byte offset of the descriptor start.
// The same kernel computes the data gradient of these layers (weights
// transposed in channels and flipped in taps), with the ReLU mask of the
// layer below fused into its epilogue. The thin first and last layers and the
// weight gradients run on the CUDA cores (deterministic two-stage sums).
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

#define NCH 32
#define NPARAM 19393
// parameter offsets (layer l: W [Co][Ci][3][3], b [Co])
#define P_W0 0
#define P_B0 576
#define P_W1 608
#define P_B1 9824
#define P_W2 9856
#define P_B2 19072
#define P_W3 19104
#define P_B3 19392

typedef __nv_bfloat16 bf16;

namespace {

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------------------
// weight packing
// ---------------------------------------------------------------------------
struct Packed {
    float *w0, *b0;        // [32][2][9] (bf16-rounded), [32]
    bf16 *f1, *d1, *f2, *d2;  // [32][288]: forward (k = tap*32 + ci) and data-gradient (k = tap*32 + co)
    float *b1, *b2;        // [32]
    float *w3, *b3;        // [32][9] (bf16-rounded), [1]
};

__global__ void k_pack(const float *__restrict__ th, Packed P) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 576) P.w0[i] = __bfloat162float(__float2bfloat16(th[P_W0 + i]));
    if (i < 32) {
        P.b0[i] = th[P_B0 + i];
        P.b1[i] = th[P_B1 + i];
        P.b2[i] = th[P_B2 + i];
    }
    if (i < 288) P.w3[i] = __bfloat162float(__float2bfloat16(th[P_W3 + i]));
    if (i == 0) P.b3[0] = th[P_B3];
    if (i < 9216) {
        // i = co*288 + tap*32 + ci  (forward B matrix row co, column k)
        int co = i / 288, k = i % 288, tap = k / 32, ci = k % 32;
        P.f1[i] = __float2bfloat16(th[P_W1 + (co * 32 + ci) * 9 + tap]);
        P.f2[i] = __float2bfloat16(th[P_W2 + (co * 32 + ci) * 9 + tap]);
        // data gradient: row ci' = co (of this matrix), column k = tap'*32 + c, weight W[c][co][8 - tap']
        int r = co, tp = tap, c = ci;
        P.d1[i] = __float2bfloat16(th[P_W1 + (c * 32 + r) * 9 + (8 - tp)]);
        P.d2[i] = __float2bfloat16(th[P_W2 + (c * 32 + r) * 9 + (8 - tp)]);
    }
}

// ---------------------------------------------------------------------------
// first layer (2 -> 32) and last layer (32 -> 1) on CUDA cores
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_first(const float *__restrict__ x, int B, int n, const float *__restrict__ w0,
                                               const float *__restrict__ b0, bf16 *__restrict__ out) {
    // weights transposed to [c][tap][co] so that 4 output channels' weights
    // are one 16-byte shared-memory read
    __shared__ __align__(16) float sw[18 * 32];
    __shared__ float sb[32];
    for (int i = threadIdx.x; i < 576; i += blockDim.x) {
        const int co = i % 32, ct = i / 32;  // ct = c * 9 + tap
        sw[i] = w0[co * 18 + ct];
    }
    if (threadIdx.x < 32) sb[threadIdx.x] = b0[threadIdx.x];
    __syncthreads();
    ll p = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    const ll npx = (ll)n * n;
    if (p >= npx * B) return;
    const int img = (int)(p / npx), yx = (int)(p % npx), y = yx / n, xx = yx % n;
    float s[32];
#pragma unroll
    for (int co = 0; co < 32; ++co) s[co] = sb[co];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = wrapn(y + t / 3 - 1, n), xs = wrapn(xx + t % 3 - 1, n);
            const float in = __bfloat162float(__float2bfloat16(x[((ll)img * 2 + c) * npx + (ll)yy * n + xs]));
            const float4 *w4 = (const float4 *)(sw + (c * 9 + t) * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 w = w4[q];
                s[4 * q] = fmaf(w.x, in, s[4 * q]);
                s[4 * q + 1] = fmaf(w.y, in, s[4 * q + 1]);
                s[4 * q + 2] = fmaf(w.z, in, s[4 * q + 2]);
                s[4 * q + 3] = fmaf(w.w, in, s[4 * q + 3]);
            }
        }
    alignas(16) bf16 o[32];
#pragma unroll
    for (int co = 0; co < 32; ++co) o[co] = __float2bfloat16(fmaxf(s[co], 0.0f));
    uint4 *dst = (uint4 *)(out + p * 32);
    const uint4 *src = (const uint4 *)o;
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = src[q];
}

// 32 -> 1: one block per tile of LTX x LTY output pixels; the tile's input
// with its one-pixel periodic halo is staged in shared memory (80-byte pixel
// stride against bank conflicts), then every thread sums its 9 x 32 products
// in the same order as before (tap, then channel).
#define LTX 32
#define LTY 8
__global__ void __launch_bounds__(256) k_last(const bf16 *__restrict__ a, int B, int n, const float *__restrict__ w3,
                                              const float *__restrict__ b3, float *__restrict__ out) {
    __shared__ float sw[9 * 32 + 1];
    __shared__ uint4 tile[(LTX + 2) * (LTY + 2)][5];
    for (int i = threadIdx.x; i < 289; i += blockDim.x) sw[i] = i < 288 ? w3[(i % 32) * 9 + i / 32] : b3[0];
    const int tiles_x = n / LTX, tiles_y = n / LTY;
    const int img = blockIdx.x / (tiles_x * tiles_y), rem = blockIdx.x % (tiles_x * tiles_y);
    const int x0 = (rem % tiles_x) * LTX, y0 = (rem / tiles_x) * LTY;
    const ll npx = (ll)n * n;
    for (int i = threadIdx.x; i < (LTX + 2) * (LTY + 2) * 4; i += blockDim.x) {
        const int px = i >> 2, q = i & 3;
        const int ty = px / (LTX + 2), tx = px % (LTX + 2);
        const int gy = wrapn(y0 + ty - 1, n), gx = wrapn(x0 + tx - 1, n);
        tile[px][q] = __ldg((const uint4 *)(a + ((ll)img * npx + (ll)gy * n + gx) * 32) + q);
    }
    __syncthreads();
    const int tx = threadIdx.x % LTX, ty = threadIdx.x / LTX;
    float s = sw[288];
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
        const int px = (ty + t / 3) * (LTX + 2) + tx + t % 3;
        const float *wt = sw + t * 32;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 u = tile[px][q];
            const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float lo = __uint_as_float(w4[j] << 16), hi = __uint_as_float(w4[j] & 0xffff0000u);
                s = fmaf(wt[q * 8 + 2 * j], lo, s);
                s = fmaf(wt[q * 8 + 2 * j + 1], hi, s);
            }
        }
    }
    out[(ll)img * npx + (ll)(y0 + ty) * n + x0 + tx] = s;
}

// ---------------------------------------------------------------------------
// 32 -> 32 layer on the tensor cores
// ---------------------------------------------------------------------------
#define CT 128           // output pixels per tile
#define CPW 130          // staged pixels per row (1 halo each side)
#define PLANE (CPW * 16) // bytes of one 8-channel plane

struct ConvArgs {
    const bf16 *in;    // [B][n][n][32]
    bf16 *out;         // [B][n][n][32]
    const bf16 *w;     // [32][288]
    const float *bias; // [32] or null
    const bf16 *mask;  // [B][n][n][32] or null: out = acc if mask > 0 else 0
    int relu;
    int B, n;
    int *status;
};

// One work item is a strip of CR output rows of CT pixels. Input rows live in
// a ring of 4 slots in shared memory, each slot 4 planes of 8 channels x CPW
// pixels (16 bytes per pixel); a row is staged once and serves the three
// output rows that need it. Two accumulators of 32 TMEM columns alternate
// between rows: while the tensor cores run the 18 MMAs of row y (issued by
// one thread), the block stores row y-1 from the other accumulator and stages
// row y+2 into the slot that row y-2 used (free once the MMAs of row y-1, the
// last to read it, have signalled their mbarrier).
#define CR 16                      // output rows per work item
#define RING (4 * 4 * PLANE)       // 4 row slots of 4 planes (33,280 B)
#define RING_PAD 33792             // ring rounded up to 1 KB
// Dynamic shared memory: ring, B (18,432 B), and 4 KB of slack so that every
// address an operand descriptor can reach stays inside this CTA's allocation.
#define CONV_SMEM (RING_PAD + 18432 + 4096)

// Stage one input row into a ring slot with 16-byte asynchronous copies
// (cp.async): the copies proceed while the block stores the previous output
// row; cp.async.wait_all before the next barrier makes them complete.
__device__ __forceinline__ void stage_row(uint8_t *sA, const bf16 *in, ll img_off, int n, int gy, int x0, int slot,
                                          int tid) {
    for (int i = tid; i < CPW * 4; i += 128) {
        const int px = i >> 2, c = i & 3;
        const int gx = wrapn(x0 + px - 1, n);
        const bf16 *src = in + (img_off + (ll)gy * n + gx) * 32 + c * 8;
        const uint32_t dst = tc::smem_u32(sA + (slot * 4 + c) * PLANE + px * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__global__ void __launch_bounds__(128) k_conv_mma(ConvArgs a) {
    extern __shared__ __align__(1024) uint8_t conv_smem[];
    uint8_t *sA = conv_smem;
    uint8_t *sB = conv_smem + RING_PAD;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::alloc(&tmem_base, 64);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        abort_flag = 0;
    }
    // weights: B operand, 36 chunks of [32 rows][8 k] (16 bytes per row)
    for (int i = tid; i < 32 * 36; i += blockDim.x) {
        int row = i / 36, ch = i % 36;
        *(uint4 *)(sB + ch * 512 + row * 16) = *(const uint4 *)(a.w + row * 288 + ch * 8);
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const int n = a.n, strips = n / CT, groups = n / CR;
    const ll nitems = (ll)a.B * strips * groups;
    const uint32_t idesc = tc::idesc_bf16(128, 32);
    const uint32_t sa = tc::smem_u32(sA), sb = tc::smem_u32(sB);
    uint32_t phase[2] = {0u, 0u};
    bool pend[2] = {false, false};  // a commit on this mbarrier not yet waited for
    float bias[32];
    for (int c = 0; c < 32; ++c) bias[c] = a.bias ? a.bias[c] : 0.0f;

    // epilogue of output row yo from accumulator buf: warp w owns TMEM lanes
    // (pixels) 32w .. 32w+31
    // completion of the MMAs of accumulator buf (bounded wait)
    auto mma_wait = [&](int buf) {
        if (!tc::mbar_wait(&mbar[buf], phase[buf], 1LL << 24)) {
            atomicOr(a.status, ST_TIMEOUT);
            abort_flag = 1;
        }
        phase[buf] ^= 1u;
        pend[buf] = false;
        tc::fence_after();
    };
    // epilogue of output row yo from accumulator buf: warp w owns TMEM lanes
    // (pixels) 32w .. 32w+31
    auto epilogue = [&](int buf, ll img_off, int yo, int x0) {
        float acc[32];
        tc::ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * 32), acc);
        const ll p = img_off + (ll)yo * n + x0 + warp * 32 + lane;
        alignas(16) bf16 o[32];
        if (a.mask) {
            alignas(16) bf16 mk[32];
            const uint4 *ms = (const uint4 *)(a.mask + p * 32);
            for (int q = 0; q < 4; ++q) ((uint4 *)mk)[q] = ms[q];
            for (int c = 0; c < 32; ++c) o[c] = __float2bfloat16(__bfloat162float(mk[c]) > 0.0f ? acc[c] : 0.0f);
        } else {
            for (int c = 0; c < 32; ++c) {
                const float v = acc[c] + bias[c];
                o[c] = __float2bfloat16(a.relu ? fmaxf(v, 0.0f) : v);
            }
        }
        uint4 *dst = (uint4 *)(a.out + p * 32);
        for (int q = 0; q < 4; ++q) dst[q] = ((const uint4 *)o)[q];
    };

    for (ll item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x) {
        const int img = (int)(item / ((ll)strips * groups));
        const int rem = (int)(item % ((ll)strips * groups));
        const int y0 = (rem / strips) * CR, x0 = (rem % strips) * CT;
        const ll img_off = (ll)img * n * n;
        // prologue: rows y0-1, y0, y0+1
        for (int r = -1; r <= 1; ++r) stage_row(sA, a.in, img_off, n, wrapn(y0 + r, n), x0, (y0 + r) & 3, tid);
        stage_wait();
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        for (int i = 0; i < CR; ++i) {
            const int y = y0 + i, buf = i & 1;
            if (tid == 0) {
                tc::fence_after();
                for (int kb = 0; kb < 18; ++kb) {
                    const int t = kb >> 1, h = kb & 1, dy = t / 3, dx = t % 3;  // dy, dx in 0..2
                    const int slot = (y + dy - 1) & 3;
                    const uint64_t ad = tc::desc(sa + (slot * 4 + 2 * h) * PLANE + dx * 16, PLANE, 128);
                    const uint64_t bd = tc::desc(sb + (2 * kb) * 512, 512, 128);
                    tc::mma_bf16(tmem + (uint32_t)(buf * 32), ad, bd, idesc, kb > 0 ? 1u : 0u);
                }
                tc::commit(&mbar[buf]);
            }
            pend[buf] = true;
            __syncwarp();
            // once the MMAs of row y-1 are done, the ring slot of row y-2 is
            // free: start staging row y+2 there, then store row y-1 out of
            // the other accumulator while the copies are in flight
            if (i > 0) mma_wait(buf ^ 1);
            if (i + 1 < CR) stage_row(sA, a.in, img_off, n, wrapn(y + 2, n), x0, (y + 2) & 3, tid);
            if (i > 0) epilogue(buf ^ 1, img_off, y - 1, x0);
            stage_wait();
            tc::fence_proxy_async();
            tc::fence_before();
            __syncthreads();
            if (abort_flag) break;
        }
        if (abort_flag) break;
        mma_wait((CR - 1) & 1);
        epilogue((CR - 1) & 1, img_off, y0 + CR - 1, x0);
        tc::fence_before();
        __syncthreads();
    }
    // after an abort, give MMAs still in flight a bounded time to finish
    // before the accumulators are freed
    for (int b = 0; b < 2; ++b)
        if (pend[b]) tc::mbar_wait(&mbar[b], phase[b], 1LL << 20);
    tc::fence_after();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, 64);
}

// ---------------------------------------------------------------------------
// training: loss, backward of the thin layers, weight gradients, Adam
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_loss(const float *__restrict__ out, const float *__restrict__ tgt, ll m,
                                              float *__restrict__ g, double *__restrict__ part) {
    __shared__ double sh[8];
    double s = 0.0;
    const float inv = 1.0f / (float)m;
    for (ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (ll)gridDim.x * blockDim.x) {
        float r = out[i] - tgt[i];
        g[i] = r * inv;
        s += (double)(r * r);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// g_a3[p][c] = sum_tap w3[c][tap] g_out[p - tap], masked by a3 > 0.
__global__ void __launch_bounds__(256) k_last_back(const float *__restrict__ gout, const bf16 *__restrict__ a3, int B,
                                                   int n, const float *__restrict__ w3, bf16 *__restrict__ gz) {
    __shared__ float sw[288];
    for (int i = threadIdx.x; i < 288; i += blockDim.x) sw[i] = w3[i];
    __syncthreads();
    ll p = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    const ll npx = (ll)n * n;
    if (p >= npx * B) return;
    const int img = (int)(p / npx), yx = (int)(p % npx), y = yx / n, xx = yx % n;
    float gt[9];
    for (int t = 0; t < 9; ++t) {
        int yy = wrapn(y - (t / 3 - 1), n), xs = wrapn(xx - (t % 3 - 1), n);
        gt[t] = gout[(ll)img * npx + (ll)yy * n + xs];
    }
    alignas(16) bf16 mk[32];
    for (int q = 0; q < 4; ++q) ((uint4 *)mk)[q] = ((const uint4 *)(a3 + p * 32))[q];
    alignas(16) bf16 o[32];
    for (int c = 0; c < 32; ++c) {
        float s = 0.0f;
        for (int t = 0; t < 9; ++t) s = fmaf(sw[c * 9 + t], gt[t], s);
        o[c] = __float2bfloat16(__bfloat162float(mk[c]) > 0.0f ? s : 0.0f);
    }
    for (int q = 0; q < 4; ++q) ((uint4 *)(gz + p * 32))[q] = ((const uint4 *)o)[q];
}

// Weight gradient of a 32 -> 32 layer for a set of 128-pixel row tiles:
// dW[co][ci][tap] = sum_p g[p][co] a[p + tap][ci], db[co] = sum_p g[p][co].
// Thread t owns the (co, ci) pairs t, t+256, t+512, t+768 (9 taps each).
// Per-block partials [block][9216 + 32]; fixed-order reduction afterwards.
__global__ void __launch_bounds__(256) k_wgrad_mid(const bf16 *__restrict__ g, const bf16 *__restrict__ a, int B,
                                                   int n, float *__restrict__ part) {
    extern __shared__ float sm[];
    float *sg = sm;             // [128][32]
    float *sa = sm + 128 * 32;  // [3][130][32]
    const int tid = threadIdx.x;
    float acc[4][9];
    float accb = 0.0f;
    for (int j = 0; j < 4; ++j)
        for (int t = 0; t < 9; ++t) acc[j][t] = 0.0f;
    const int tiles_row = n / CT;
    const ll ntiles = (ll)B * n * tiles_row;
    for (ll tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int img = (int)(tile / ((ll)n * tiles_row));
        const int rem = (int)(tile % ((ll)n * tiles_row));
        const int y = rem / tiles_row, x0 = (rem % tiles_row) * CT;
        const ll off = (ll)img * n * n;
        __syncthreads();
        for (int i = tid; i < 128 * 32; i += blockDim.x) sg[i] = __bfloat162float(g[(off + (ll)y * n + x0) * 32 + i]);
        for (int i = tid; i < 3 * CPW * 32; i += blockDim.x) {
            int r = i / (CPW * 32), rm = i % (CPW * 32), px = rm / 32, c = rm % 32;
            int gy = wrapn(y + r - 1, n), gx = wrapn(x0 + px - 1, n);
            sa[i] = __bfloat162float(a[(off + (ll)gy * n + gx) * 32 + c]);
        }
        __syncthreads();
        for (int j = 0; j < 4; ++j) {
            const int pr = tid + 256 * j, co = pr / 32, ci = pr % 32;
            for (int px = 0; px < CT; ++px) {
                const float gv = sg[px * 32 + co];
#pragma unroll
                for (int t = 0; t < 9; ++t)
                    acc[j][t] = fmaf(gv, sa[((t / 3) * CPW + px + (t % 3)) * 32 + ci], acc[j][t]);
            }
        }
        if (tid < 32)
            for (int px = 0; px < CT; ++px) accb += sg[px * 32 + tid];
    }
    float *dst = part + (ll)blockIdx.x * (9216 + 32);
    for (int j = 0; j < 4; ++j) {
        const int pr = tid + 256 * j, co = pr / 32, ci = pr % 32;
        for (int t = 0; t < 9; ++t) dst[(co * 32 + ci) * 9 + t] = acc[j][t];
    }
    if (tid < 32) dst[9216 + tid] = accb;
}

// Weight gradients of the first (2 -> 32) and last (32 -> 1) layers, per
// block partials [block][608] and [block][289].
__global__ void __launch_bounds__(256) k_wgrad_thin(const bf16 *__restrict__ gz1, const float *__restrict__ x,
                                                    const float *__restrict__ gout, const bf16 *__restrict__ a3, int B,
                                                    int n, float *__restrict__ part0, float *__restrict__ part3) {
    // thread t: first layer outputs t (< 608: W0 then b0) and last layer t (< 289)
    const int tid = threadIdx.x;
    const ll npx = (ll)n * n, m = npx * B;
    float acc0[3] = {0, 0, 0}, acc3[2] = {0, 0};
    for (ll p = blockIdx.x; p < m; p += gridDim.x) {
        const int img = (int)(p / npx), yx = (int)(p % npx), y = yx / n, xx = yx % n;
        for (int j = 0; j < 3; ++j) {
            const int o = tid + 256 * j;
            if (o < 576) {
                const int co = o / 18, ci = (o / 9) % 2, t = o % 9;
                const int yy = wrapn(y + t / 3 - 1, n), xs = wrapn(xx + t % 3 - 1, n);
                const float xv = __bfloat162float(__float2bfloat16(x[((ll)img * 2 + ci) * npx + (ll)yy * n + xs]));
                acc0[j] = fmaf(__bfloat162float(gz1[p * 32 + co]), xv, acc0[j]);
            } else if (o < 608) {
                acc0[j] += __bfloat162float(gz1[p * 32 + (o - 576)]);
            }
        }
        for (int j = 0; j < 2; ++j) {
            const int o = tid + 256 * j;
            if (o < 288) {
                const int ci = o / 9, t = o % 9;
                const int yy = wrapn(y + t / 3 - 1, n), xs = wrapn(xx + t % 3 - 1, n);
                acc3[j] = fmaf(gout[p], __bfloat162float(a3[((ll)img * npx + (ll)yy * n + xs) * 32 + ci]), acc3[j]);
            } else if (o == 288) {
                acc3[j] += gout[p];
            }
        }
    }
    for (int j = 0; j < 3; ++j)
        if (tid + 256 * j < 608) part0[(ll)blockIdx.x * 608 + tid + 256 * j] = acc0[j];
    for (int j = 0; j < 2; ++j)
        if (tid + 256 * j < 289) part3[(ll)blockIdx.x * 289 + tid + 256 * j] = acc3[j];
}

// grad[off + i] = sum over blocks of part[b][i] (fixed order, FP64).
__global__ void k_reduce(const float *__restrict__ part, int nblk, int len, float *__restrict__ grad, int off) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(ll)b * len + i];
    grad[off + i] = (float)s;
}

// mid-layer partial layout [9216 W then 32 b] -> parameter offsets
__global__ void k_reduce_mid(const float *__restrict__ part, int nblk, float *__restrict__ grad, int offW, int offB) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9248) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(ll)b * 9248 + i];
    grad[i < 9216 ? offW + i : offB + (i - 9216)] = (float)s;
}

__global__ void k_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int np, float lr, float b1, float b2, float c1, float c2, float eps) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct pm_net {
    int max_n, max_b;
    cudaStream_t st;
    float *theta, *grad, *m, *v;
    Packed P;
    bf16 *a1, *a2, *a3, *g1, *g2;  // activations and gradients [B][n][n][32]
    float *out, *gout;             // [B][n][n]
    float *part_mid, *part0, *part3;
    double *loss_part;
    double *h_loss;
    int *status;
    long long step;
    int nsm;
    std::vector<void *> allocs;
};

namespace {

template <class T>
bool nalloc(pm_net *t, T **p, size_t count) {
    if (cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)) != cudaSuccess) return false;
    t->allocs.push_back((void *)*p);
    return true;
}

const int WG_BLOCKS = 256;   // weight-gradient partial blocks
const int LOSS_BLOCKS = 256;

void net_pack(pm_net *t) {
    k_pack<<<div_up(9216, 256), 256, 0, t->st>>>(t->theta, t->P);
    count_launches(1);
}

// At most 4 CTAs per SM (shared memory bound), so at most 128 of the 512
// tensor-memory columns of an SM are ever requested.
int conv_grid(pm_net *t, ll ntiles) {
    ll g = (ll)t->nsm * 4;
    return (int)(ntiles < g ? ntiles : g);
}

void net_forward(pm_net *t, const float *x, int B, int n, float *out) {
    const ll m = (ll)B * n * n;
    net_pack(t);
    k_first<<<div_up(m, 256), 256, 0, t->st>>>(x, B, n, t->P.w0, t->P.b0, t->a1);
    const ll ntiles = (ll)B * (n / CR) * (n / CT);
    ConvArgs a1{t->a1, t->a2, t->P.f1, t->P.b1, nullptr, 1, B, n, t->status};
    k_conv_mma<<<conv_grid(t, ntiles), 128, CONV_SMEM, t->st>>>(a1);
    ConvArgs a2{t->a2, t->a3, t->P.f2, t->P.b2, nullptr, 1, B, n, t->status};
    k_conv_mma<<<conv_grid(t, ntiles), 128, CONV_SMEM, t->st>>>(a2);
    k_last<<<B * (n / LTX) * (n / LTY), LTX * LTY, 0, t->st>>>(t->a3, B, n, t->P.w3, t->P.b3, out);
    count_launches(4);
}

}  // namespace

extern "C" {

int pm_net_num_params(void) { return NPARAM; }

pm_status pm_net_create(pm_net **out, int max_n, int max_batch, void *stream) {
    if (!out || max_n < CT || max_n % CT || max_batch < 1) return PM_EINVAL;
    *out = nullptr;
    pm_net *t = new pm_net();
    t->max_n = max_n;
    t->max_b = max_batch;
    t->st = (cudaStream_t)stream;
    t->step = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&t->nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t m = (size_t)max_n * max_n * max_batch;
    bool ok = nalloc(t, &t->theta, NPARAM) && nalloc(t, &t->grad, NPARAM) && nalloc(t, &t->m, NPARAM) &&
              nalloc(t, &t->v, NPARAM) && nalloc(t, &t->P.w0, 576) && nalloc(t, &t->P.b0, 32) &&
              nalloc(t, &t->P.f1, 9216) && nalloc(t, &t->P.d1, 9216) && nalloc(t, &t->P.f2, 9216) &&
              nalloc(t, &t->P.d2, 9216) && nalloc(t, &t->P.b1, 32) && nalloc(t, &t->P.b2, 32) &&
              nalloc(t, &t->P.w3, 288) && nalloc(t, &t->P.b3, 1) && nalloc(t, &t->a1, m * 32) &&
              nalloc(t, &t->a2, m * 32) && nalloc(t, &t->a3, m * 32) && nalloc(t, &t->g1, m * 32) &&
              nalloc(t, &t->g2, m * 32) && nalloc(t, &t->out, m) && nalloc(t, &t->gout, m) &&
              nalloc(t, &t->part_mid, (size_t)WG_BLOCKS * 9248) && nalloc(t, &t->part0, (size_t)WG_BLOCKS * 608) &&
              nalloc(t, &t->part3, (size_t)WG_BLOCKS * 289) && nalloc(t, &t->loss_part, LOSS_BLOCKS) &&
              nalloc(t, &t->status, 1);
    if (ok && cudaMallocHost((void **)&t->h_loss, sizeof(double) * (LOSS_BLOCKS + 1)) != cudaSuccess) ok = false;
    if (!ok) {
        pm_net_destroy(t);
        cudaGetLastError();
        return PM_ENOMEM;
    }
    cudaMemset(t->theta, 0, sizeof(float) * NPARAM);
    cudaMemset(t->m, 0, sizeof(float) * NPARAM);
    cudaMemset(t->v, 0, sizeof(float) * NPARAM);
    cudaMemset(t->status, 0, sizeof(int));
    cudaFuncSetAttribute(k_wgrad_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (128 * 32 + 3 * CPW * 32) * 4);
    cudaFuncSetAttribute(k_conv_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        pm_net_destroy(t);
        return PM_ECUDA;
    }
    *out = t;
    return PM_OK;
}

void pm_net_destroy(pm_net *t) {
    if (!t) return;
    for (void *p : t->allocs) cudaFree(p);
    if (t->h_loss) cudaFreeHost(t->h_loss);
    delete t;
}

pm_status pm_net_set_stream(pm_net *t, void *stream) {
    if (!t) return PM_EINVAL;
    t->st = (cudaStream_t)stream;
    return PM_OK;
}

pm_status pm_net_state(pm_net *t, float *host_out, long long *step_out) {
    if (!t || !host_out) return PM_EINVAL;
    cudaStreamSynchronize(t->st);
    if (cudaMemcpy(host_out, t->theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host_out + NPARAM, t->m, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(host_out + 2 * NPARAM, t->v, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PM_ECUDA;
    if (step_out) *step_out = t->step;
    return PM_OK;
}

pm_status pm_net_load(pm_net *t, const float *host_in, int with_moments, long long step) {
    if (!t || !host_in) return PM_EINVAL;
    cudaStreamSynchronize(t->st);
    if (cudaMemcpy(t->theta, host_in, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return PM_ECUDA;
    if (with_moments) {
        if (cudaMemcpy(t->m, host_in + NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(t->v, host_in + 2 * NPARAM, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess)
            return PM_ECUDA;
    } else {
        cudaMemset(t->m, 0, sizeof(float) * NPARAM);
        cudaMemset(t->v, 0, sizeof(float) * NPARAM);
    }
    t->step = step;
    return PM_OK;
}

pm_status pm_net_forward(pm_net *t, const float *x, int B, int n, float *out) {
    if (!t || !x || !out || B < 1 || B > t->max_b || n < CT || n % CT || n > t->max_n) return PM_EINVAL;
    net_forward(t, x, B, n, out);
    return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

pm_status pm_net_train_step(pm_net *t, const float *x, const float *target, int B, int n, float lr, double *loss) {
    if (!t || !x || !target || B < 1 || B > t->max_b || n < CT || n % CT || n > t->max_n) return PM_EINVAL;
    const ll m = (ll)B * n * n;
    net_forward(t, x, B, n, t->out);
    k_loss<<<LOSS_BLOCKS, 256, 0, t->st>>>(t->out, target, m, t->gout, t->loss_part);
    k_last_back<<<div_up(m, 256), 256, 0, t->st>>>(t->gout, t->a3, B, n, t->P.w3, t->g2);  // g2 = dL/dz3 (pre-ReLU)
    const ll ntiles = (ll)B * (n / CR) * (n / CT);
    const size_t wsm = (128 * 32 + 3 * CPW * 32) * 4;
    // layer 2 (input a2, output gradient g2)
    k_wgrad_mid<<<WG_BLOCKS, 256, wsm, t->st>>>(t->g2, t->a2, B, n, t->part_mid);
    k_reduce_mid<<<div_up(9248, 256), 256, 0, t->st>>>(t->part_mid, WG_BLOCKS, t->grad, P_W2, P_B2);
    ConvArgs d2{t->g2, t->g1, t->P.d2, nullptr, t->a2, 0, B, n, t->status};  // g1 = dL/dz2
    k_conv_mma<<<conv_grid(t, ntiles), 128, CONV_SMEM, t->st>>>(d2);
    // layer 1 (input a1, output gradient g1)
    k_wgrad_mid<<<WG_BLOCKS, 256, wsm, t->st>>>(t->g1, t->a1, B, n, t->part_mid);
    k_reduce_mid<<<div_up(9248, 256), 256, 0, t->st>>>(t->part_mid, WG_BLOCKS, t->grad, P_W1, P_B1);
    ConvArgs d1{t->g1, t->g2, t->P.d1, nullptr, t->a1, 0, B, n, t->status};  // g2 = dL/dz1
    k_conv_mma<<<conv_grid(t, ntiles), 128, CONV_SMEM, t->st>>>(d1);
    // first and last layers
    k_wgrad_thin<<<WG_BLOCKS, 256, 0, t->st>>>(t->g2, x, t->gout, t->a3, B, n, t->part0, t->part3);
    k_reduce<<<div_up(608, 256), 256, 0, t->st>>>(t->part0, WG_BLOCKS, 608, t->grad, P_W0);
    k_reduce<<<div_up(289, 256), 256, 0, t->st>>>(t->part3, WG_BLOCKS, 289, t->grad, P_W3);
    t->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)t->step), c2 = 1.0f - powf(b2, (float)t->step);
    k_adam<<<div_up(NPARAM, 256), 256, 0, t->st>>>(t->theta, t->grad, t->m, t->v, NPARAM, lr, b1, b2, c1, c2, 1e-8f);
    count_launches(12);
    if (cudaGetLastError() != cudaSuccess) return PM_ECUDA;
    if (loss) {
        if (cudaMemcpyAsync(t->h_loss, t->loss_part, sizeof(double) * LOSS_BLOCKS, cudaMemcpyDeviceToHost, t->st) !=
                cudaSuccess ||
            cudaStreamSynchronize(t->st) != cudaSuccess)
            return PM_ECUDA;
        double s = 0.0;
        for (int b = 0; b < LOSS_BLOCKS; ++b) s += t->h_loss[b];
        *loss = 0.5 * s / (double)m;
        int st = 0;
        cudaMemcpy(&st, t->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (st & ST_TIMEOUT) return PM_ETIMEOUT;
    }
    return PM_OK;
}

// Gradient of the last train step (host, NPARAM floats), for tests.
pm_status pm_net_grad(pm_net *t, float *host_out) {
    if (!t || !host_out) return PM_EINVAL;
    cudaStreamSynchronize(t->st);
    return cudaMemcpy(host_out, t->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess ? PM_OK
                                                                                                           : PM_ECUDA;
}

}  // extern "C"
