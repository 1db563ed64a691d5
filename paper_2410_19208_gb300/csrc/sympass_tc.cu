// Symmetric pass Y = A X + shift X on the 5th-generation tensor cores
// (tcgen05, sm_103a): the sketch and power products of the range finder
// (Alg. 1) and the core product Z = A Q of Alg. 2, in BF16 with FP32
// accumulation.
//
// The pass reads a BF16 image A' of A written once per projection by
// pack_upper_bf16_kernel: the tiles (I, J) of BM = 256 rows x 64 columns with
// J >= 4 I (the block upper triangle), where the 256 x 256 blocks on the
// diagonal hold a_ij for j > i, a_ii / 2 on the diagonal and 0 below it, so
// that A = A' + A'^T exactly; entries past row or column n are zero.  The
// tiles are stored one after another in row-major tile order, each 32 KB
// already in the 128-byte-swizzled layout of a UMMA operand, so a CTA streams
// a contiguous range of the image, one bulk copy per tile, and every later
// pass over A reads 2 bytes per upper-triangle entry instead of 4.
//
// Each tile (with the X_J tile loaded by TMA beside it, three stages in
// flight) feeds two products straight from shared memory:
//   P1  D1^T (m x BM) += X_J^T (m x 64) . A'_IJ^T   (B operand K-major)
//   P2  D2^T (m x 64)   = X_I^T (m x BM) . A'_IJ    (B operand MN-major)
// with M = 128 rows of X^T (m <= 128; rows m..127 are zero).  D1^T
// accumulates over the run of tiles a CTA owns in one block row and is
// flushed once; D2^T is double-buffered in TMEM and added to Y after every
// tile.  The shift term is not in the pass: the sweep that converts X to
// BF16 starts Y at shift X (or adds it), so a run that holds a diagonal
// block drains D1 without extra global reads.  Both are
// added by TMA bulk reduce-add from a swizzled 32 x 32 staging box per warp
// (scalar atomics when Y is not 16-byte aligned with ld % 4 == 0).
//
// Warp roles (256 threads, one CTA per SM, persistent over a cost-balanced
// range of the tiles in row-major order): warp 0 issues the copies, warp 1
// owns TMEM and issues the row-product MMAs, warp 2 the transposed-product
// MMAs (one thread each), warps 4-7 drain TMEM.  Every mbarrier
// wait is bounded; on a timeout the CTA records PSDPROJ_ETIMEOUT, unwinds and
// frees its TMEM.
#include <cuda_bf16.h>
#include <cstring>
#include <cudaTypedefs.h>

#include "ctx.h"
#include "tc_common.cuh"

namespace {

using namespace tc;

constexpr int BN = PSD_TILE_N;
constexpr int BM = PSD_TILE_M;
constexpr int R = PSD_TILE_R;                    // column tiles per block-row step
constexpr int NSTAGE = 3;
constexpr uint32_t A_BYTES = BM * BN * 2;        // BF16 tile of A'
constexpr uint32_t XJ_BYTES = 128 * BN * 2;      // X_J^T rows 0..127 (16 KB)
constexpr uint32_t STAGE = A_BYTES + XJ_BYTES;   // one stage: A' tile, then X_J
constexpr uint32_t XI_BYTES = 128 * BM * 2;      // 64 KB
constexpr uint32_t STG_BYTES = 32 * 32 * 4;      // epilogue staging box per warp
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_XI = NSTAGE * STAGE;
constexpr uint32_t OFF_STG = OFF_XI + XI_BYTES;
constexpr uint32_t OFF_BAR = OFF_STG + 4 * STG_BYTES;
constexpr uint32_t SMEM_BYTES = OFF_BAR + 256;
constexpr uint32_t D1_COL = 0, D2_COL = BM;      // TMEM columns: D1 256, D2 2 x 64
constexpr uint32_t TMEM_COLS = 512;
constexpr int NT = 256;
constexpr long long WAIT_LIMIT = 4000000000LL;  // ~2 s at 2 GHz
static_assert(SMEM_BYTES <= 232448, "shared memory");
static_assert(STAGE % 1024 == 0 && OFF_XI % 1024 == 0 && OFF_STG % 1024 == 0, "swizzle atoms");

struct Bars {
    uint64_t full[NSTAGE], empty[NSTAGE];
    uint64_t fullXI, emptyXI;
    uint64_t d2full[2], d2empty[2];
    uint64_t d1full, d1empty;
    uint64_t mmadone;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(Bars) <= 256, "barrier block");

struct Params {
    int64_t n;
    int m;
    int nbr, nbc;
    int64_t tiles;
    float *Y;
    int64_t ldy;
    int *d_status;
    int tma_y;          // Y reduced by TMA (aligned Y); else scalar atomics
};

__device__ __forceinline__ void tile_of(int64_t t, int nbc, int nbr, int &I, int &J)
{
    int lo = 0, hi = nbr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (psd_tile_row_start(mid, nbc) <= t) lo = mid; else hi = mid - 1;
    }
    I = lo;
    J = R * lo + (int)(t - psd_tile_row_start(lo, nbc));
}

// the next tile in row-major order over the block upper triangle
__device__ __forceinline__ void tile_next(int &I, int &J, int nbc)
{
    if (++J == nbc) {
        ++I;
        J = R * I;
    }
}

__device__ __forceinline__ void fail(Bars &B, int *st)
{
    B.abort = 1;
    psd_set_status(st, PSDPROJ_ETIMEOUT);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Epilogue: add 32 rows (r0 .. r0+31) of column c = 32 q + lane, held in v,
// to Y.  With TMA: stage as a 32 x 32 box (128-byte swizzle: the 16-byte
// chunk j of column c at c*128 + ((j ^ (c & 7)) << 4)) and reduce-add it;
// the staging box is reused after the previous reduce has read it.
__device__ __forceinline__ void flush32(const Params &P, const CUtensorMap *tmY, uint8_t *stg, int q,
                                        int lane, int64_t r0, const float (&v)[32])
{
    const int c = 32 * q + lane;
    if (P.tma_y) {
        if (r0 >= P.n || 32 * q >= P.m) return;               // the whole box is outside Y
        if (lane == 0) bulk_wait_read();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j)
            *reinterpret_cast<float4 *>(stg + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            tma_reduce_add_2d(tmY, (int)r0, 32 * q, stg);
            bulk_commit();
        }
    } else if (c < P.m) {
        float *ycol = P.Y + (int64_t)c * P.ldy;
#pragma unroll
        for (int e = 0; e < 32; ++e)
            if (r0 + e < P.n) atomicAdd(ycol + r0 + e, v[e]);
    }
}

__global__ void __launch_bounds__(NT, 1)
sym_pass_bf16_kernel(const uint16_t *__restrict__ Ab, const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmY, const Params P)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    Bars &B = *reinterpret_cast<Bars *>(sm + OFF_BAR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // equal shares of cost(t) = t + SEGC * (row of t): a block-row start costs
    // about SEGC tiles (D1 drained, X_I reloaded, the pipeline refilled), so
    // CTAs whose range crosses many short rows near the end get fewer tiles
    auto first_tile = [&](int64_t b) -> int64_t {
        constexpr int64_t SEGC = 4;
        const int64_t target = (P.tiles + SEGC * P.nbr) * b / gridDim.x;
        int64_t lo = 0, hi = P.tiles;                // smallest t with cost(t) >= target
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            int Im, Jm;
            tile_of(mid, P.nbc, P.nbr, Im, Jm);
            if (mid + SEGC * Im >= target) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    const int64_t t0 = first_tile(blockIdx.x);
    const int64_t t1 = blockIdx.x + 1 == gridDim.x ? P.tiles : first_tile(blockIdx.x + 1);
    if ((smem_u32(sm) & 1023u) != 0u) {
        if (threadIdx.x == 0) psd_set_status(P.d_status, PSDPROJ_ECUDA);
        return;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&B.full[s], 1);
            mbar_init(&B.empty[s], 2);    // both MMA threads
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B.d2full[b], 1);
            mbar_init(&B.d2empty[b], 4);
        }
        mbar_init(&B.fullXI, 1);
        mbar_init(&B.emptyXI, 1);
        mbar_init(&B.d1full, 1);
        mbar_init(&B.d1empty, 4);
        mbar_init(&B.mmadone, 2);
        B.abort = 0;
        fence_proxy_async_smem();
        prefetch_tmap(&tmX);
        if (P.tma_y) prefetch_tmap(&tmY);
    }
    if (warp == 1) {
        tmem_alloc(&B.tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = B.tmem_base;
    volatile int *abort = &B.abort;
    int I0 = 0, J0 = 0;
    if (t0 < t1) tile_of(t0, P.nbc, P.nbr, I0, J0);

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            int I = I0, J = J0, curI = -1, xi_uses = 0;
            int64_t it = 0;
            for (int64_t t = t0; t < t1; ++t, ++it, tile_next(I, J, P.nbc)) {
                if (I != curI) {
                    if (!mbar_wait(&B.emptyXI, (xi_uses & 1) ^ 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                    mbar_arrive_expect_tx(&B.fullXI, XI_BYTES);
                    for (int kk = 0; kk < BM / 64; ++kk)
                        tma_load_2d(sm + OFF_XI + kk * 16384, &tmX, BM * I + 64 * kk, 0, &B.fullXI);
                    ++xi_uses;
                    curI = I;
                }
                const int s = (int)(it % NSTAGE);
                const uint32_t us = (uint32_t)(it / NSTAGE);
                if (!mbar_wait(&B.empty[s], (us & 1) ^ 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                mbar_arrive_expect_tx(&B.full[s], STAGE);
                bulk_load(sm + OFF_A + s * STAGE, Ab + t * PSD_TILE_ELEMS, A_BYTES, &B.full[s]);
                tma_load_2d(sm + OFF_A + s * STAGE + A_BYTES, &tmX, BN * J, 0, &B.full[s]);
            }
            // wait (bounded) for the copies still in flight to land
            const int64_t n_it = it;
            for (int64_t k = (n_it > NSTAGE ? n_it - NSTAGE : 0); k < n_it; ++k)
                mbar_wait(&B.full[k % NSTAGE], (uint32_t)((k / NSTAGE) & 1), abort, WAIT_LIMIT);
            if (xi_uses > 0) mbar_wait(&B.fullXI, (uint32_t)((xi_uses - 1) & 1), abort, WAIT_LIMIT);
        }
    } else if (warp == 1 || warp == 2) {
        // ------------------------------------------------------------ MMA
        // two issuing threads: warp 1 the four long row-product MMAs (P1,
        // D1), warp 2 the sixteen short transposed-product MMAs (P2, D2).
        // tcgen05.mma issue blocks once the tensor pipe's queue is full, so
        // while one thread does its bookkeeping the other's MMAs keep the
        // pipe busy; each commits its own MMAs (a stage is free after both).
        if (lane == 0) {
            const bool p1 = (warp == 1);
            const uint32_t id1 = idesc_bf16(128, BM, 0, 0);
            const uint32_t id2 = idesc_bf16(128, BN, 0, 1);
            int I = I0, J = J0, curI = -1, seg = 0;
            int64_t it = 0;
            bool issued = false;
            for (int64_t t = t0; t < t1; ++t, ++it, tile_next(I, J, P.nbc)) {
                const bool first = (I != curI);
                const bool last = (J == P.nbc - 1) || (t + 1 == t1);
                if (first) {
                    const bool ok = p1 ? mbar_wait(&B.d1empty, (seg & 1) ^ 1, abort, WAIT_LIMIT)
                                       : mbar_wait(&B.fullXI, seg & 1, abort, WAIT_LIMIT);
                    if (!ok) { fail(B, P.d_status); break; }
                    curI = I;
                }
                const int s = (int)(it % NSTAGE);
                const uint32_t us = (uint32_t)(it / NSTAGE);
                const int b = (int)(it & 1);
                const uint32_t ub = (uint32_t)(it >> 1);
                if (!mbar_wait(&B.full[s], us & 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                if (!p1 && !mbar_wait(&B.d2empty[b], (ub & 1) ^ 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                tc_fence_after();
                const uint32_t a_tile = smem_u32(sm + OFF_A + s * STAGE);
                if (p1) {
                    // P1: D1^T += X_J^T A_IJ^T   (K = 64 tile columns)
                    const uint32_t xj = a_tile + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BN / 16; ++kk) {
                        const uint64_t ad = sdesc_sw128(xj + kk * 32, 16, 1024);
                        const uint64_t bd = sdesc_sw128(a_tile + kk * 32, 16, 1024);
                        mma_bf16_ss(tmem + D1_COL, ad, bd, id1, (!first || kk > 0) ? 1u : 0u);
                    }
                } else {
                    // P2: D2^T = X_I^T A_IJ   (K = 256 tile rows)
                    const uint32_t xi = smem_u32(sm + OFF_XI);
#pragma unroll
                    for (int kk = 0; kk < BM / 16; ++kk) {
                        const uint64_t ad = sdesc_sw128(xi + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024);
                        const uint64_t bd = sdesc_sw128(a_tile + kk * 2048, 16384, 1024);
                        mma_bf16_ss(tmem + D2_COL + BN * b, ad, bd, id2, kk > 0 ? 1u : 0u);
                    }
                }
                issued = true;
                mma_commit(&B.empty[s]);
                if (!p1) mma_commit(&B.d2full[b]);
                if (last) {
                    mma_commit(p1 ? &B.d1full : &B.emptyXI);
                    ++seg;
                }
            }
            if (issued) {
                // all MMAs of this CTA (both threads) complete before TMEM is released
                mma_commit(&B.mmadone);
                if (p1) mbar_wait(&B.mmadone, 0, abort, WAIT_LIMIT);
            }
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------- epilogue
        const int q = warp & 3;                // TMEM lane quarter of this warp
        uint8_t *stg = sm + OFF_STG + q * STG_BYTES;
        int I = I0, J = J0, seg = 0;
        int64_t it = 0;
        for (int64_t t = t0; t < t1; ++t, ++it, tile_next(I, J, P.nbc)) {
            const bool last = (J == P.nbc - 1) || (t + 1 == t1);
            const int b = (int)(it & 1);
            const uint32_t ub = (uint32_t)(it >> 1);
            {
                // lane 0 waits (bounded); the warp leaves together
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&B.d2full[b], ub & 1, abort, WAIT_LIMIT) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { if (lane == 0) fail(B, P.d_status); break; }
            }
            tc_fence_after();
            float v0[32], v1[32];
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + D2_COL + BN * b;
            tmem_ld32(ta, v0);
            tmem_ld32(ta + 32, v1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.d2empty[b]);
            flush32(P, &tmY, stg, q, lane, (int64_t)BN * J, v0);
            flush32(P, &tmY, stg, q, lane, (int64_t)BN * J + 32, v1);
            if (last) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&B.d1full, seg & 1, abort, WAIT_LIMIT) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { if (lane == 0) fail(B, P.d_status); break; }
                tc_fence_after();
                const int64_t r0 = (int64_t)BM * I;
#pragma unroll 1
                for (int ch = 0; ch < BM / 32; ++ch) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + D1_COL + 32 * ch, v);
                    flush32(P, &tmY, stg, q, lane, r0 + 32 * ch, v);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&B.d1empty);
                ++seg;
            }
        }
        if (lane == 0 && P.tma_y) bulk_wait_all();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// X (FP32, column-major) -> BF16 image used by the TMA loads of the pass:
// part 0 = bf16(x) (the high part), part 1 = bf16(x - bf16(x)) (the low part
// of the split-BF16 form).  The same sweep starts Y for the pass (Y is a
// different buffer): y_mode 1 sets Y = shift X, y_mode 2 adds shift X to Y,
// y_mode 0 leaves Y alone; shift = *d_shift, 0 when d_shift is NULL.  Grid:
// x over 1024-row chunks, y over the m columns (coalesced, no division).
__global__ void __launch_bounds__(256)
to_bf16_kernel(const float *__restrict__ X, int64_t ldx, int64_t n, __nv_bfloat16 *__restrict__ H, int64_t ldh,
               int part, float *__restrict__ Y, int64_t ldy, const double *__restrict__ d_shift, int y_mode)
{
    const int c = blockIdx.y;
    const float *xc = X + (int64_t)c * ldx;
    __nv_bfloat16 *hc = H + (int64_t)c * ldh;
    float *yc = Y + (int64_t)c * ldy;
    const float shift = d_shift ? (float)*d_shift : 0.0f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = (int64_t)blockIdx.x * 1024 + r * 256 + threadIdx.x;
        if (i >= n) break;
        const float x = xc[i];
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        hc[i] = part ? __float2bfloat16_rn(x - __bfloat162float(hi)) : hi;
        if (y_mode == 1) yc[i] = shift * x;
        else if (y_mode == 2) yc[i] = fmaf(shift, x, yc[i]);
    }
}

__device__ __forceinline__ float lo_part(float v)
{
    return v - __bfloat162float(__float2bfloat16_rn(v));
}

// BF16 image A' of the block upper triangle of A (see the top of this file).
// Block: 64 rows x 64 columns of one tile, 16 threads per row; a thread
// converts 4 consecutive entries (one float4 of A) in each of 4 rows 16
// apart, its four loads issued together, into halves of 16-byte chunks of
// the swizzled rows.  grid.x: 64-column tiles J, grid.y: 64-row chunks;
// tiles left of the diagonal block exit at once.  part 1 writes the low
// parts bf16(a - bf16(a)) instead (the split-BF16 form's second image).
__global__ void __launch_bounds__(256)
pack_upper_bf16_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                       uint16_t *__restrict__ Ab, int nbc, int vec, int part, int64_t nblocks)
{
    constexpr int RPT = 4;                            // rows per thread
    // grid-strided over the (tile column J, 64-row chunk) blocks
    for (int64_t bid = blockIdx.x; bid < nblocks; bid += gridDim.x) {
    const int J = (int)(bid % nbc);
    const int64_t chunk = bid / nbc;
    const int I = (int)((chunk * 64) / BM);
    if (J < R * I) continue;                          // uniform across the block
    const int64_t rbase = chunk * 64 + (threadIdx.x >> 4);
    const int64_t c0 = (int64_t)J * BN + 4 * (threadIdx.x & 15);
    float v[RPT][4];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int64_t r = rbase + 16 * u;
        if (r < n && vec && c0 + 4 <= n) {
            const float4 a = __ldcs(reinterpret_cast<const float4 *>(A + r * lda + c0));
            v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
        } else {
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) v[u][qq] = (r < n && c0 + qq < n) ? A[r * lda + c0 + qq] : 0.0f;
        }
    }
    const bool diagblk = J < R * (I + 1);
    const int k = (threadIdx.x & 15) >> 1;             // 16-byte chunk of the row
    const int64_t t = psd_tile_row_start(I, nbc) + (J - R * I);
    uint8_t *tile = reinterpret_cast<uint8_t *>(Ab + t * PSD_TILE_ELEMS);
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int64_t r = rbase + 16 * u;
        if (diagblk) {
            // diagonal block: keep the strict upper part, halve the diagonal
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int64_t c = c0 + qq;
                v[u][qq] = c > r ? v[u][qq] : (c == r ? 0.5f * v[u][qq] : 0.0f);
            }
        }
        if (part) {
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) v[u][qq] = lo_part(v[u][qq]);
        }
        uint2 o;
        o.x = pack_bf16(v[u][0], v[u][1]);
        o.y = pack_bf16(v[u][2], v[u][3]);
        const int rt = (int)(r - (int64_t)I * BM);     // row within the tile
        *reinterpret_cast<uint2 *>(tile + rt * 128 + ((k ^ (rt & 7)) << 4) + 8 * (threadIdx.x & 1)) = o;
    }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() { return tensor_map_encoder(); }

}  // namespace

cudaError_t launch_pack_bf16(cudaStream_t s, const float *A, int64_t n, int64_t lda, uint16_t *Ab,
                             int part)
{
    if ((reinterpret_cast<uintptr_t>(Ab) & 15) != 0) return cudaErrorInvalidValue;
    const int nbr = (int)((n + BM - 1) / BM);
    const int nbc = nbr * R;
    const int vec = (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    const int64_t nblocks = (int64_t)nbc * nbr * (BM / 64);
    // A in host memory (read over the host link): a few blocks per SM keep
    // the link busy without taking every SM from the other streams' kernels
    cudaPointerAttributes pa;
    const bool host = cudaPointerGetAttributes(&pa, A) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    if (!host) cudaGetLastError();
    int64_t grid = nblocks;
    if (host && grid > 152 * 2) grid = 152 * 2;
    if (grid > 0x7fffffff) grid = 0x7fffffff;
    pack_upper_bf16_kernel<<<(unsigned)grid, 256, 0, s>>>(A, n, lda, Ab, nbc, vec, part, nblocks);
    return cudaGetLastError();
}

cudaError_t launch_sym_pass_tc(cudaStream_t s, int sm_count, const uint16_t *Ab,
                               int64_t n, const float *X, int64_t ldx, int m,
                               const double *d_shift, float *Y, int64_t ldy, uint16_t *Xh,
                               int64_t ldh, int *d_status, int x_part, int accumulate)
{
    if (m < 1 || m > 128) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(Ab) & 15) != 0) return cudaErrorNotSupported;
    if ((ldh % 8) != 0 || (reinterpret_cast<uintptr_t>(Xh) & 15) != 0 || ldh < n)
        return cudaErrorNotSupported;
    auto encode = get_encode();
    if (!encode) return cudaErrorNotSupported;

    // BF16 image of X (rows n, columns m; TMA fills the rest with zeros);
    // Y starts at shift X (accumulate = 0) or gains it (accumulate = 1)
    if (n > 0) {
        const int y_mode = accumulate ? (d_shift ? 2 : 0) : 1;
        const dim3 grid((unsigned)((n + 1023) / 1024), (unsigned)m);
        to_bf16_kernel<<<grid, 256, 0, s>>>(X, ldx, n, reinterpret_cast<__nv_bfloat16 *>(Xh), ldh, x_part, Y, ldy,
                                            d_shift, y_mode);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    CUtensorMap tmX;
    {
        cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
        cuuint64_t strides[1] = {(cuuint64_t)ldh * 2};
        cuuint32_t box[2] = {64, 128};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Xh, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    Params P;
    P.n = n;
    P.m = m;
    P.nbr = (int)((n + BM - 1) / BM);
    P.nbc = P.nbr * R;
    P.tiles = psd_tile_count(n);
    P.Y = Y;
    P.ldy = ldy;
    P.d_status = d_status;
    P.tma_y = ((ldy % 4) == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0);
    CUtensorMap tmY;
    memset(&tmY, 0, sizeof(tmY));
    if (P.tma_y) {
        cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
        cuuint64_t strides[1] = {(cuuint64_t)ldy * 4};
        cuuint32_t box[2] = {32, 32};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&tmY, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Y, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            P.tma_y = 0;
    }

    cudaError_t e = cudaFuncSetAttribute(sym_pass_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int grid = sm_count > 0 ? sm_count : 148;
    if ((int64_t)grid > P.tiles) grid = (int)P.tiles;
    sym_pass_bf16_kernel<<<grid, NT, SMEM_BYTES, s>>>(Ab, tmX, tmY, P);
    return cudaGetLastError();
}
