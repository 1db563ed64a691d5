// power_iteration (Alg. 4) and min_eig (Alg. 5) on the device.
//
// One launch per product w = (A + shift I) (s * v): A is streamed once, upper
// triangle only, in 32 x 128 tiles.  A thread block owns a segment of one
// block row: the row sums accumulate in registers, the transposed
// contributions of each tile are summed over the block's 8 warps and added
// with atomics.  A small kernel after each product (pi_norm_kernel) forms
// ||w|| in FP64, stores the scale 1/||w|| that the next product applies on
// load and clears the other vector for the next product.  sigma = ||A v||
// after the N normalised steps is written to *d_sigma.
#include "ctx.h"
#include "tc_common.cuh"

namespace {

constexpr int TRW = 32;    // rows per tile
constexpr int TCW = 128;   // columns per tile
constexpr int SEGW = 8;    // tiles per block
constexpr int NTW = 256;

// scal[0]: scale of the input vector; scal[1]: norm of the last output.
// A block owns a segment of SEGW tiles (32 rows x 128 columns each) of one
// block row.  Warp w holds rows 4w..4w+3, lane l columns 4l..4l+3 of every
// tile; the loads of the whole segment are independent, and the column
// partial sums stay in registers until the segment ends (one barrier).
__global__ void __launch_bounds__(NTW)
sym_gemv_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                const float *__restrict__ x, float *__restrict__ y, const double *scal,
                const double *d_shift_neg, int vec)
{
    __shared__ float colsum[8][SEGW * TCW];
    // grid: x = segment within the block row, y = block row; segments past
    // the end of a row exit at once
    const int I = blockIdx.y;
    const int64_t row0 = (int64_t)I * TRW;
    const int tiles = (int)((n - row0 + TCW - 1) / TCW);
    const int t0 = (int)blockIdx.x * SEGW;
    if (t0 >= tiles) return;
    const float sc = (float)scal[0];
    const float shift = d_shift_neg ? (float)(-(*d_shift_neg)) : 0.0f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    float rowacc[4] = {0.f, 0.f, 0.f, 0.f};
    float xr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = row0 + warp * 4 + i;
        xr[i] = gr < n ? x[gr] * sc : 0.0f;
    }
    // Interior tiles (strictly above the diagonal block, not past column n)
    // take an unmasked path: per row one float4 load, 4 FMAs into the row sum
    // and 4 into the column partials.  The diagonal tile, the ragged last
    // tile and unaligned rows take the masked path.
    const float *rowp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = row0 + warp * 4 + i;
        rowp[i] = A + (gr < n ? gr : 0) * lda;
    }
    auto is_interior = [&](int tt) {
        const int64_t cb = row0 + (int64_t)tt * TCW;
        return vec && tt > 0 && tt < tiles && cb + TCW <= n && row0 + 32 <= n;
    };
    // software pipeline: the loads of tile t+1 are issued before tile t is used
    float4 nxt[4];
    bool nxt_int = is_interior(t0);
    if (nxt_int) {
        const int64_t c0 = row0 + (int64_t)t0 * TCW + lane * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) nxt[i] = __ldcs(reinterpret_cast<const float4 *>(rowp[i] + c0));
    }
#pragma unroll 1
    for (int t = 0; t < SEGW; ++t) {
        const int tt = t0 + t;
        const int64_t c0 = row0 + (int64_t)tt * TCW + lane * 4;
        float colacc[4] = {0.f, 0.f, 0.f, 0.f};
        const bool interior = nxt_int;
        float4 a4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a4[i] = nxt[i];
        nxt_int = (t + 1 < SEGW) && is_interior(tt + 1);
        if (nxt_int) {
            const int64_t c1 = c0 + TCW;
#pragma unroll
            for (int i = 0; i < 4; ++i) nxt[i] = __ldcs(reinterpret_cast<const float4 *>(rowp[i] + c1));
        }
        if (interior) {
            const float4 xv = __ldg(reinterpret_cast<const float4 *>(x + c0));
            const float xc[4] = {xv.x * sc, xv.y * sc, xv.z * sc, xv.w * sc};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float a[4] = {a4[i].x, a4[i].y, a4[i].z, a4[i].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    rowacc[i] = fmaf(a[j], xc[j], rowacc[i]);
                    colacc[j] = fmaf(a[j], xr[i], colacc[j]);
                }
            }
        } else if (tt < tiles) {
            float xc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) xc[j] = (c0 + j < n) ? x[c0 + j] * sc : 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t gr = row0 + warp * 4 + i;
                if (gr >= n) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // strictly-lower entries of the diagonal tile are never loaded
                    const float a = (c0 + j < n && c0 + j >= gr) ? rowp[i][c0 + j] : 0.0f;
                    rowacc[i] = fmaf(a, xc[j], rowacc[i]);
                    if (c0 + j > gr) colacc[j] = fmaf(a, xr[i], colacc[j]);
                }
            }
        }
        // this thread's column partials of tile t (one owner per slot)
#pragma unroll
        for (int j = 0; j < 4; ++j) colsum[warp][t * TCW + lane * 4 + j] = colacc[j];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < SEGW * TCW; c += NTW) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += colsum[w][c];
        const int64_t gc = row0 + (int64_t)t0 * TCW + c;
        if (gc < n && s != 0.0f) atomicAdd(&y[gc], s);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s = rowacc[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int64_t gr = row0 + warp * 4 + i;
        if (lane == 0 && gr < n) {
            if (t0 == 0) s = fmaf(shift, xr[i], s);  // the segment holding the diagonal
            atomicAdd(&y[gr], s);
        }
    }

}

// The same product on the tiled BF16 image A' of the block upper triangle
// (A = A' + A'^T; written by the tensor-core pass's pack kernel, tiles of
// 256 x 64 in 128-byte-swizzled rows, stored in row-major tile order).  A
// persistent CTA (two per SM) streams a contiguous range of tiles into a three-stage ring
// by bulk copies (one producer thread, bounded mbarrier waits) and eight
// compute warps read them from shared memory: thread (g, k) owns rows
// 8g..8g+7 and columns 8k..8k+7 of a tile.  Row sums stay in registers over
// a run of tiles in one block row and are reduced when the run ends; column
// sums are reduced per tile (warp shuffles, then a shared table over the
// eight warps) and added to y with atomics.  No entry needs masking; the
// diagonal block's halved diagonal enters once through each side.
namespace gt {
constexpr int STAGES = 3;
constexpr int CTAS_PER_SM = 2;    // two CTAs per SM: one computes while the other waits
constexpr uint32_t TILE_BYTES = (uint32_t)PSD_TILE_ELEMS * 2;
constexpr int NCOMP = 256;               // compute threads (warps 0-7)
constexpr int NTG = NCOMP + 32;          // + producer warp 8
constexpr uint32_t SMEM = STAGES * TILE_BYTES + 1024;
constexpr long long WAIT_LIMIT = 4000000000LL;
}

struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = err + a.lo + b.lo;
    const float h = s + lo;
    return {h, lo - (h - s)};
}

// ||v|| and 1/||v|| of a sum of squares t = acc (double-float): the FP32
// estimate of 1/sqrt(t) with one FP32 Newton step, then one double-float
// Newton step for each, r = x + (t - x^2) y / 2 with x = t y, and
// 1/r = y + y (1 - y r); 0 and 0 when t = 0.
__device__ __forceinline__ void dfl_norm_inv(dfl acc, double &nrm, double &inv)
{
    nrm = 0.0;
    inv = 0.0;
    if (acc.hi > 0.0f) {
        float q = rsqrtf(acc.hi);
        q = q * fmaf(-0.5f * acc.hi, q * q, 1.5f);
        const float x = acc.hi * q;
        const float x2 = x * x;
        const dfl d = dfl_add(acc, {-x2, -fmaf(x, x, -x2)});          // t - x^2
        const float rc = d.hi * (0.5f * q);
        const float rh = x + rc, rl = rc - (rh - x);                  // r = rh + rl
        const float yr = q * rh, yre = fmaf(q, rh, -yr);
        const float res = ((1.0f - yr) - yre) - q * rl;               // 1 - q r
        nrm = (double)rh + (double)rl;
        inv = (double)q + (double)(q * res);
    }
}

// Per-thread part of sum v_i^2 over i = first, first + stride, ... < n, as
// an unevaluated double-float sum (the square split exactly by FMA, Knuth's
// two-sum per term).
__device__ __forceinline__ dfl dfl_sumsq(const float *__restrict__ v, int64_t n, int64_t first, int64_t stride,
                                         float *__restrict__ clear)
{
    float hi = 0.0f, lo = 0.0f;
#pragma unroll 4
    for (int64_t i = first; i < n; i += stride) {
        const float a = v[i];
        const float p = a * a, e = fmaf(a, a, -p);          // a^2 = p + e exactly
        const float s = hi + p;
        const float bb = s - hi;
        lo += ((hi - (s - bb)) + (p - bb)) + e;
        hi = s;
        if (clear) clear[i] = 0.0f;
    }
    return {hi + lo, lo - ((hi + lo) - hi)};
}

// The same over all of v by nthr threads (thread tid), four float4 loads in
// flight per thread: v 16-byte aligned.  The order of the terms depends only
// on (n, tid, nthr), so every block that calls it gets the same sum.
__device__ __forceinline__ void dfl_sq_acc(float a, float &hi, float &lo)
{
    const float p = a * a, e = fmaf(a, a, -p);
    const float s = hi + p;
    const float bb = s - hi;
    lo += ((hi - (s - bb)) + (p - bb)) + e;
    hi = s;
}
__device__ __forceinline__ dfl dfl_sumsq_vec(const float *__restrict__ v, int64_t n, int tid, int nthr)
{
    float hi = 0.0f, lo = 0.0f;
    const int64_t n4 = n >> 2;
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
    int64_t j = tid;
    for (; j + 3 * (int64_t)nthr < n4; j += 4 * (int64_t)nthr) {
        float4 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = v4[j + u * (int64_t)nthr];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            dfl_sq_acc(a[u].x, hi, lo); dfl_sq_acc(a[u].y, hi, lo);
            dfl_sq_acc(a[u].z, hi, lo); dfl_sq_acc(a[u].w, hi, lo);
        }
    }
    for (; j < n4; j += nthr) {
        const float4 a = v4[j];
        dfl_sq_acc(a.x, hi, lo); dfl_sq_acc(a.y, hi, lo); dfl_sq_acc(a.z, hi, lo); dfl_sq_acc(a.w, hi, lo);
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += nthr) dfl_sq_acc(v[i], hi, lo);
    return {hi + lo, lo - ((hi + lo) - hi)};
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start before the previous kernel on
// its stream has finished; griddep_wait() returns once that kernel has
// completed and its writes are visible, and griddep_launch_dependents() lets
// the next such kernel start.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ dfl dfl_warp_sum(dfl acc)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc = dfl_add(acc, {__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)});
    return acc;
}

// v_i of three vectors (i = 0, 1, 2) without an indexed local array
__device__ __forceinline__ float *pick3(float *a, float *b, float *c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

__device__ __forceinline__ void bf16x8_to_f32(const uint4 u, float (&a)[8])
{
    a[0] = __uint_as_float(u.x << 16); a[1] = __uint_as_float(u.x & 0xFFFF0000u);
    a[2] = __uint_as_float(u.y << 16); a[3] = __uint_as_float(u.y & 0xFFFF0000u);
    a[4] = __uint_as_float(u.z << 16); a[5] = __uint_as_float(u.z & 0xFFFF0000u);
    a[6] = __uint_as_float(u.w << 16); a[7] = __uint_as_float(u.w & 0xFFFF0000u);
}

// Launched with programmatic stream serialization: the producer streams the
// image (written before the previous kernel started) at once; the compute
// warps wait for the previous kernel before they touch x, y, scal, the
// shift or `clear`.  self_norm: x is scaled by 1/||x||, computed by every
// CTA in the same order (so every CTA uses the same scale); else by
// scal[0].  clear (may be NULL): zeroed, each CTA its slice (the next
// product's output, this product's input no longer being read).
__device__ __forceinline__ void sym_gemv_tiles_body(const uint16_t *__restrict__ Ab, int64_t n, int nbr,
                                                    int64_t tiles, const float *__restrict__ x,
                                                    float *__restrict__ y, const double *scal, int self_norm,
                                                    float *__restrict__ clear, const double *d_shift_neg,
                                                    int *d_status, long long wait_limit, int bid, int nb)
{
    const long long WL = wait_limit > 0 ? wait_limit : gt::WAIT_LIMIT;
    using namespace tc;
    extern __shared__ __align__(1024) uint8_t smt[];
    __shared__ uint64_t full[gt::STAGES], empty[gt::STAGES];
    __shared__ float colred[2][8][PSD_TILE_N];
    __shared__ int s_abort;       // any role gave up: stop waiting
    __shared__ int s_cabort;      // compute warps: written before, read after their barrier
    __shared__ dfl s_red[8];
    __shared__ float s_sc;
    const int nbc = nbr * PSD_TILE_R;
    const int64_t t0 = tiles * bid / nb;
    const int64_t t1 = tiles * (bid + 1) / nb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < gt::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 8);
        }
        s_abort = 0;
        s_cabort = 0;
        fence_proxy_async_smem();
    }
    __syncthreads();
    volatile int *abort = &s_abort;
    volatile int *cabort = &s_cabort;
    // the next product's loads do not depend on this one
    griddep_launch_dependents();

    if (warp == 8) {
        // ---- producer: one bulk copy per tile
        if (lane == 0) {
            int64_t it = 0;
            for (int64_t t = t0; t < t1; ++t, ++it) {
                const int s = (int)(it % gt::STAGES);
                const uint32_t us = (uint32_t)(it / gt::STAGES);
                if (!mbar_wait(&empty[s], (us & 1) ^ 1, abort, WL)) {
                    s_abort = 1;
                    psd_set_status(d_status, PSDPROJ_ETIMEOUT);
                    break;
                }
                mbar_arrive_expect_tx(&full[s], gt::TILE_BYTES);
                bulk_load(smt + s * gt::TILE_BYTES, Ab + t * PSD_TILE_ELEMS, gt::TILE_BYTES, &full[s]);
            }
            const int64_t n_it = it;
            for (int64_t k = (n_it > gt::STAGES ? n_it - gt::STAGES : 0); k < n_it; ++k)
                mbar_wait_drain(&full[k % gt::STAGES], (uint32_t)((k / gt::STAGES) & 1), gt::WAIT_LIMIT);
        }
    } else {
        griddep_wait();
        if (clear) {
            const int64_t c0 = n * bid / nb, c1 = n * (bid + 1) / nb;
            for (int64_t i = c0 + threadIdx.x; i < c1; i += gt::NCOMP) clear[i] = 0.0f;
        }
        if (t0 >= t1) return;      // no tile: the producer issues no copy either
        float sc;
        if (self_norm) {
            dfl acc = dfl_warp_sum(dfl_sumsq_vec(x, n, threadIdx.x, gt::NCOMP));
            if (lane == 0) s_red[warp] = acc;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (warp == 0) {
                acc = dfl_warp_sum(lane < 8 ? s_red[lane] : dfl{0.0f, 0.0f});
                if (lane == 0) {
                    double nrm, inv;
                    dfl_norm_inv(acc, nrm, inv);
                    s_sc = (float)inv;
                }
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");
            sc = s_sc;
        } else {
            sc = (float)scal[0];
        }
        const float shift = d_shift_neg ? (float)(-(*d_shift_neg)) : 0.0f;
        // ---- compute: thread (g, k): rows 8g..8g+7, columns 8k..8k+7 of each tile
        const int g = threadIdx.x >> 3, k = threadIdx.x & 7;
        int I = 0, J = 0;
        {
            int lo = 0, hi = nbr - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (psd_tile_row_start(mid, nbc) <= t0) lo = mid; else hi = mid - 1;
            }
            I = lo;
            J = PSD_TILE_R * lo + (int)(t0 - psd_tile_row_start(lo, nbc));
        }
        float rowacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float xr[8];
        bool has_diag = false;
        auto load_xr = [&](int Iv) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t gr = (int64_t)Iv * PSD_TILE_M + 8 * g + u;
                xr[u] = gr < n ? x[gr] * sc : 0.0f;
            }
        };
        load_xr(I);
        // column values of x for tile column Jv (zero past n)
        auto load_xc = [&](int Jv, float (&out)[8]) {
            const int64_t c0 = (int64_t)Jv * PSD_TILE_N + 8 * k;
            if (c0 + 8 <= n) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(x + c0));
                const float4 b = __ldg(reinterpret_cast<const float4 *>(x + c0 + 4));
                out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
                out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
            } else {
#pragma unroll
                for (int v = 0; v < 8; ++v) out[v] = (c0 + v < n) ? x[c0 + v] : 0.0f;
            }
        };
        float xn[8];
        load_xc(J, xn);
        int64_t it = 0;
        for (int64_t t = t0; t < t1; ++t, ++it) {
            if (J == PSD_TILE_R * I) has_diag = true;
            const int s = (int)(it % gt::STAGES);
            const uint32_t us = (uint32_t)(it / gt::STAGES);
            // a warp whose bounded wait fails records the abort but still
            // reaches the barrier below; every warp leaves after it together
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&full[s], us & 1, abort, WL) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok && lane == 0) {
                *cabort = 1;
                *abort = 1;
                psd_set_status(d_status, PSDPROJ_ETIMEOUT);
            }
            // this tile's column values of x (loaded one tile ahead), then the next tile's
            float xc[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) xc[v] = xn[v] * sc;
            {
                int In = I, Jn = J + 1;
                if (Jn == nbc) { ++In; Jn = PSD_TILE_R * In; }
                load_xc(Jn, xn);
            }
            float colacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const uint8_t *tile = smt + s * gt::TILE_BYTES;
#pragma unroll
            for (int u = 0; u < 8 && ok; ++u) {
                const int r = 8 * g + u;                        // r & 7 == u
                const uint4 q = *reinterpret_cast<const uint4 *>(tile + r * 128 + ((k ^ u) << 4));
                float a[8];
                bf16x8_to_f32(q, a);
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    rowacc[u] = fmaf(a[v], xc[v], rowacc[u]);
                    colacc[v] = fmaf(a[v], xr[u], colacc[v]);
                }
            }
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive(&empty[s]);
            // column sums: over the four row groups of the warp, then the 8 warps
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                colacc[v] += __shfl_xor_sync(0xffffffffu, colacc[v], 8);
                colacc[v] += __shfl_xor_sync(0xffffffffu, colacc[v], 16);
            }
            const int pb = (int)(it & 1);
            if (lane < 8) {
#pragma unroll
                for (int v = 0; v < 8; ++v) colred[pb][warp][8 * k + v] = colacc[v];
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (*cabort) break;                      // uniform: read after the barrier
            if (threadIdx.x < PSD_TILE_N) {
                float cs = 0.0f;
#pragma unroll
                for (int w = 0; w < 8; ++w) cs += colred[pb][w][threadIdx.x];
                const int64_t gc = (int64_t)J * PSD_TILE_N + threadIdx.x;
                if (gc < n && cs != 0.0f) atomicAdd(&y[gc], cs);
            }
            // run end: the row sums of block row I
            const bool last = (J == nbc - 1) || (t + 1 == t1);
            if (last) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float v = rowacc[u];
                    v += __shfl_xor_sync(0xffffffffu, v, 1);
                    v += __shfl_xor_sync(0xffffffffu, v, 2);
                    v += __shfl_xor_sync(0xffffffffu, v, 4);
                    rowacc[u] = 0.0f;
                    const int64_t gr = (int64_t)I * PSD_TILE_M + 8 * g + u;
                    if (k == 0 && gr < n) {
                        if (has_diag) v = fmaf(shift, xr[u], v);
                        atomicAdd(&y[gr], v);
                    }
                }
                has_diag = false;
            }
            if (++J == nbc) {
                ++I;
                J = PSD_TILE_R * I;
                load_xr(I);
            }
        }
    }

}

__global__ void __launch_bounds__(gt::NTG, gt::CTAS_PER_SM)
sym_gemv_tiles_kernel(const uint16_t *__restrict__ Ab, int64_t n, int nbr, int64_t tiles,
                      const float *__restrict__ x, float *__restrict__ y, const double *scal, int self_norm,
                      float *__restrict__ clear, const double *d_shift_neg, int *d_status, long long wait_limit)
{
    sym_gemv_tiles_body(Ab, n, nbr, tiles, x, y, scal, self_norm, clear, d_shift_neg, d_status, wait_limit,
                        blockIdx.x, gridDim.x);
}

// product `it` of many power iterations in one launch: block b runs CTA
// bmap[b].y of entry bmap[b].x's product (its own rotation of v0, v1, v2)
__global__ void __launch_bounds__(gt::NTG, gt::CTAS_PER_SM)
sym_gemv_tiles_grouped_kernel(const psd_g_pi *__restrict__ tab, const int2 *__restrict__ bmap, int it,
                              int *d_status, long long wait_limit)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_pi a = tab[b.x];
    sym_gemv_tiles_body(a.Ab, a.n, (int)((a.n + PSD_TILE_M - 1) / PSD_TILE_M), psd_tile_count(a.n),
                        pick3(a.v0, a.v1, a.v2, it % 3), pick3(a.v0, a.v1, a.v2, (it + 1) % 3), a.scal,
                        it > 0 ? 1 : 0, pick3(a.v0, a.v1, a.v2, (it + 2) % 3), a.shift_neg, d_status, wait_limit,
                        b.y, a.nb);
}

// ||y|| of a finished product and the clearing of the next product's output
// (the previous input, no longer read), as a kernel of its own after the
// product: one block of 1024 threads, each summing y_i^2 over a strided slice
// as an unevaluated double-float sum hi + lo (the square split exactly by
// FMA, Knuth's two-sum per term), the partial sums added in double-float over
// the warps; the root and its reciprocal by Newton steps in double-float
// from the FP32 estimate.  Writes scal[0] = 1/||y||, scal[1] = ||y|| and,
// when asked, *d_sigma = ||y|| (0 and 0 when y = 0).  FP64 arithmetic, a
// handful of operations per SM and clock on this GPU, is kept out of the
// sum; this replaced an eight-block FP64 kernel with an atomic ticket
// (9.8 us -> a few us per product).
__device__ __forceinline__ void pi_norm_body(const float *__restrict__ y, float *__restrict__ other, int64_t n,
                                             double *scal, double *d_sigma)
{
    __shared__ dfl red[32];
    dfl acc = dfl_warp_sum(dfl_sumsq(y, n, threadIdx.x, 1024, other));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = dfl_warp_sum(red[threadIdx.x]);
        if (threadIdx.x == 0) {
            double nrm, inv;
            dfl_norm_inv(acc, nrm, inv);
            scal[1] = nrm;
            scal[0] = inv;
            if (d_sigma) *d_sigma = nrm;
        }
    }
}

__global__ void __launch_bounds__(1024)
pi_norm_kernel(const float *__restrict__ y, float *__restrict__ other, int64_t n, double *scal,
               double *d_sigma)
{
    pi_norm_body(y, other, n, scal, d_sigma);
}

// the norms closing many power iterations of N + 1 products: block b, entry b
__global__ void __launch_bounds__(1024)
pi_norm_grouped_kernel(const psd_g_pi *__restrict__ tab, int N)
{
    const psd_g_pi a = tab[blockIdx.x];
    pi_norm_body(pick3(a.v0, a.v1, a.v2, (N + 1) % 3), pick3(a.v0, a.v1, a.v2, (N + 2) % 3), a.n, a.scal,
                 a.sigma);
}

__global__ void pi_init_kernel(double *scal, float *v1, int64_t n)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) { scal[0] = 1.0; scal[1] = 0.0; }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v1[i] = 0.0f;
}

// alpha = alpha_in if alpha_in > 0, else |sigma1 - sigma2|.  The shift used by
// the range finder is alpha when alpha is finite and > 1e-300; otherwise 0
// and bit 0 of *d_info is set (the call degrades to Alg. 2).
__global__ void alpha_finish_kernel(const double *d_s1, const double *d_s2, double alpha_in,
                                    double *d_alpha, double *d_shift, int *d_info)
{
    double a = alpha_in;
    if (!(alpha_in > 0.0)) a = fabs(*d_s1 - *d_s2);
    const bool ok = isfinite(a) && a > 1e-300;
    if (d_alpha) *d_alpha = a;
    *d_shift = ok ? a : 0.0;
    if (d_info) *d_info = ok ? 0 : 1;
}

// Variant of Alg. 5 (alpha from the sketch's Ritz values): alpha = -min_i d_i
// over the eigenvalues d of the core C = Q^T A Q of an unshifted sketch
// (Ritz values lie in [lambda_min(A), lambda_max(A)], so this estimates
// |lambda_min| from inside); outputs as alpha_finish_kernel.
// alpha_finish for many problems: thread i, entry i
__global__ void alpha_finish_grouped_kernel(const psd_g_alpha *__restrict__ tab, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const psd_g_alpha a = tab[i];
    double al = a.alpha_in;
    if (!(a.alpha_in > 0.0)) al = fabs(*a.s1 - *a.s2);
    const bool ok = isfinite(al) && al > 1e-300;
    if (a.d_alpha) *a.d_alpha = al;
    *a.d_shift = ok ? al : 0.0;
    if (a.d_info) *a.d_info = ok ? 0 : 1;
}

__global__ void ritz_alpha_kernel(const double *d, int m, double *d_alpha, double *d_shift, int *d_info)
{
    double lo = 0.0;
    bool finite = true;
    for (int i = 0; i < m; ++i) {
        finite = finite && isfinite(d[i]);
        lo = fmin(lo, d[i]);
    }
    const double a = finite ? -lo : nan("");
    const bool ok = finite && a > 1e-300;
    if (d_alpha) *d_alpha = a;
    *d_shift = ok ? a : 0.0;
    if (d_info) *d_info = ok ? 0 : 1;
}

// Y += shift X for n x m column-major blocks (leading dimension ld each)
__global__ void add_shift_kernel(float *__restrict__ Y, const float *__restrict__ X, int64_t n, int m,
                                 int64_t ld, const double *d_shift)
{
    const float a = (float)*d_shift;
    if (a == 0.0f) return;
    const int64_t total = n * (int64_t)m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        Y[c * ld + i] = fmaf(a, X[c * ld + i], Y[c * ld + i]);
    }
}

}  // namespace

cudaError_t launch_ritz_alpha(cudaStream_t s, const double *d, int m, double *d_alpha, double *d_shift,
                              int *d_info)
{
    ritz_alpha_kernel<<<1, 1, 0, s>>>(d, m, d_alpha, d_shift, d_info);
    return cudaGetLastError();
}

cudaError_t launch_add_shift(cudaStream_t s, float *Y, const float *X, int64_t n, int m, int64_t ld,
                             const double *d_shift)
{
    int64_t blocks = (n * (int64_t)m + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    add_shift_kernel<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(Y, X, n, m, ld, d_shift);
    return cudaGetLastError();
}

cudaError_t launch_power_iteration(cudaStream_t s, const float *A, int64_t n, int64_t lda, int N,
                                   uint64_t seed, uint32_t stream_id, const double *d_shift_neg,
                                   float *v0, float *v1, double *scal, double *d_sigma)
{
    cudaError_t e = launch_gaussian(s, seed, stream_id, n, 1, 1, n, v0, n);
    if (e != cudaSuccess) return e;
    pi_init_kernel<<<64, 256, 0, s>>>(scal, v1, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = (int)((n + TRW - 1) / TRW);
    const int maxseg = (int)(((n + TCW - 1) / TCW + SEGW - 1) / SEGW);  // row 0 has the most
    const dim3 grid((unsigned)maxseg, (unsigned)nb);
    const int vec = ((lda % 4) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    float *in = v0, *out = v1;
    for (int it = 0; it <= N; ++it) {
        sym_gemv_kernel<<<grid, NTW, 0, s>>>(A, n, lda, in, out, scal, d_shift_neg, vec);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        pi_norm_kernel<<<1, 1024, 0, s>>>(out, in, n, scal, it == N ? d_sigma : nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float *t = in; in = out; out = t;
    }
    return cudaSuccess;
}

cudaError_t launch_power_iteration_bf16(cudaStream_t s, int sm_count, const uint16_t *Ab, int64_t n,
                                        int N, uint64_t seed, uint32_t stream_id,
                                        const double *d_shift_neg, float *v0, float *v1, float *v2,
                                        double *scal, double *d_sigma, int *d_status, long long wait_limit)
{
    if ((reinterpret_cast<uintptr_t>(Ab) & 15) != 0 || (reinterpret_cast<uintptr_t>(v0) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(v1) & 15) != 0 || (reinterpret_cast<uintptr_t>(v2) & 15) != 0)
        return cudaErrorInvalidValue;
    cudaError_t e = launch_gaussian(s, seed, stream_id, n, 1, 1, n, v0, n);
    if (e != cudaSuccess) return e;
    pi_init_kernel<<<64, 256, 0, s>>>(scal, v1, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sym_gemv_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gt::SMEM);
    if (e != cudaSuccess) return e;
    const int nbr = (int)((n + PSD_TILE_M - 1) / PSD_TILE_M);
    const int64_t tiles = psd_tile_count(n);
    int grid = (sm_count > 0 ? sm_count : 148) * gt::CTAS_PER_SM;
    if ((int64_t)grid > tiles) grid = (int)tiles;
    // product it reads v[it % 3] (v0: the Gaussian start, scaled by
    // scal[0] = 1; later ones by their own norm), accumulates into
    // v[(it + 1) % 3] (zeroed by pi_init or by the product before) and
    // clears v[(it + 2) % 3], its predecessor's input
    float *v[3] = {v0, v1, v2};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(gt::NTG);
    cfg.dynamicSmemBytes = gt::SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    for (int it = 0; it <= N; ++it) {
        e = cudaLaunchKernelEx(&cfg, sym_gemv_tiles_kernel, Ab, n, nbr, tiles, (const float *)v[it % 3],
                               v[(it + 1) % 3], (const double *)scal, it > 0 ? 1 : 0, v[(it + 2) % 3],
                               d_shift_neg, d_status, wait_limit);
        if (e != cudaSuccess) return e;
    }
    // ||y|| of the last product (sigma)
    pi_norm_kernel<<<1, 1024, 0, s>>>(v[(N + 1) % 3], v[(N + 2) % 3], n, scal, d_sigma);
    return cudaGetLastError();
}

cudaError_t launch_power_iteration_grouped(cudaStream_t s, const psd_g_pi *tab, int count, const int2 *bmap,
                                          int nb, int N, int *d_status, long long wait_limit)
{
    if (count < 1 || nb < 1 || N < 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(sym_gemv_tiles_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gt::SMEM);
    if (e != cudaSuccess) return e;
    // the products chained by programmatic dependent launch, as in the
    // single-problem iteration
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nb);
    cfg.blockDim = dim3(gt::NTG);
    cfg.dynamicSmemBytes = gt::SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    for (int it = 0; it <= N; ++it) {
        e = cudaLaunchKernelEx(&cfg, sym_gemv_tiles_grouped_kernel, tab, bmap, it, d_status, wait_limit);
        if (e != cudaSuccess) return e;
    }
    pi_norm_grouped_kernel<<<(unsigned)count, 1024, 0, s>>>(tab, N);
    return cudaGetLastError();
}

cudaError_t launch_alpha_finish_grouped(cudaStream_t s, const psd_g_alpha *tab, int count)
{
    if (count < 1) return cudaErrorInvalidValue;
    alpha_finish_grouped_kernel<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(tab, count);
    return cudaGetLastError();
}

cudaError_t launch_pi_init(cudaStream_t s, double *scal, float *v1, int64_t n)
{
    pi_init_kernel<<<64, 256, 0, s>>>(scal, v1, n);
    return cudaGetLastError();
}

cudaError_t launch_pi_norm(cudaStream_t s, const float *y, float *other, int64_t n, double *scal,
                           double *d_sigma)
{
    pi_norm_kernel<<<1, 1024, 0, s>>>(y, other, n, scal, d_sigma);
    return cudaGetLastError();
}

cudaError_t launch_alpha_finish(cudaStream_t s, const double *d_s1, const double *d_s2,
                                double alpha_in, double *d_alpha, double *d_shift, int *d_info)
{
    alpha_finish_kernel<<<1, 1, 0, s>>>(d_s1, d_s2, alpha_in, d_alpha, d_shift, d_info);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of min_eig.
//
// For callers that cannot call cudaMalloc: code running inside another
// library's memory manager or a custom allocator that forbids allocations in
// its hot path, plug-ins whose host cannot grant device allocations, or
// contexts whose memory is capped and fully reserved up front.  Its scratch
// (the two power-iteration vectors and the norms and scales) is a
// fixed file-scope device array, present on every GPU that loads this
// library until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NOALLOC_MAX_N = PSDPROJ_NOALLOC_MAX_N;
constexpr size_t NOALLOC_VEC_BYTES = sizeof(float) * (size_t)NOALLOC_MAX_N;
constexpr size_t NOALLOC_BYTES = 2 * NOALLOC_VEC_BYTES + 32 * sizeof(double);

// the shared scratch: v0, v1, then 32 doubles (scales, sigmas, shift, info)
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

__global__ void noalloc_copy_kernel(const double *s1, const double *s2, double *d1, double *d2)
{
    if (d1) *d1 = *s1;
    if (d2) *d2 = *s2;
}

}  // namespace

#include <mutex>

extern "C" int psdproj_min_eig_noalloc(const float *dA, int64_t n, int64_t lda, int N, uint64_t seed,
                                       double *d_alpha, double *d_sigma1, double *d_sigma2,
                                       void *stream)
{
    if (!dA || !d_alpha || n < 1 || lda < n || N < 0) return PSDPROJ_EINVAL;
    if (n > NOALLOC_MAX_N) return PSDPROJ_ETOOLARGE;
    // set-up, once per device, with that device current: the device address
    // of the scratch array (its name in host code is only a host-side stand-in)
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PSDPROJ_ECUDA;
    // A must live on the current device (the scratch address is that device's)
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, dA) != cudaSuccess) {
        cudaGetLastError();
        return PSDPROJ_EINVAL;
    }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) return PSDPROJ_EINVAL;
    if (pa.device != dev) return PSDPROJ_EINVAL;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PSDPROJ_ECUDA;
            addr[dev] = p;
        }
        base = static_cast<unsigned char *>(addr[dev]);
    }
    float *v0 = reinterpret_cast<float *>(base);
    float *v1 = reinterpret_cast<float *>(base + NOALLOC_VEC_BYTES);
    double *scal = reinterpret_cast<double *>(base + 2 * NOALLOC_VEC_BYTES);
    double *sig1 = scal + 16, *sig2 = scal + 17, *shift = scal + 18;
    int *info = reinterpret_cast<int *>(scal + 19);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_power_iteration(s, dA, n, lda, N, seed, 3u, nullptr, v0, v1, scal, sig1) != cudaSuccess)
        return PSDPROJ_ECUDA;
    if (launch_power_iteration(s, dA, n, lda, N, seed, 4u, sig1, v0, v1, scal, sig2) != cudaSuccess)
        return PSDPROJ_ECUDA;
    if (launch_alpha_finish(s, sig1, sig2, 0.0, d_alpha, shift, info) != cudaSuccess) return PSDPROJ_ECUDA;
    if (d_sigma1 || d_sigma2) {
        noalloc_copy_kernel<<<1, 1, 0, s>>>(sig1, sig2, d_sigma1, d_sigma2);
        if (cudaGetLastError() != cudaSuccess) return PSDPROJ_ECUDA;
    }
    return PSDPROJ_OK;
}
