// Symmetric pass Y = A X + shift X on the 5th-generation tensor cores
// (tcgen05, sm_103a): the sketch and power products of the range finder
// (Alg. 1) and the core product Z = A Q of Alg. 2, in BF16 with FP32
// accumulation.
//
// The pass reads a BF16 image A' of A written once per projection by
// pack_upper_bf16_kernel: the tiles (I, J) of BM = 256 rows x 64 columns with
// J >= 4 I (the block upper triangle), where the 256 x 256 blocks on the
// diagonal hold a_ij for j > i, a_ii / 2 on the diagonal and 0 below it, so
// that A = A' + A'^T exactly.  The image is padded with zeros to a multiple
// of 256 in both directions.  Every later pass over A then streams 2 bytes
// per upper-triangle entry instead of 4, and needs no masking.
//
// Each tile is loaded by TMA (128-byte swizzle, four stages in flight) and
// feeds two products straight from shared memory:
//   P1  D1^T (m x BM) += X_J^T (m x 64) . A'_IJ^T   (B operand K-major)
//   P2  D2^T (m x 64)   = X_I^T (m x BM) . A'_IJ    (B operand MN-major)
// with M = 128 rows of X^T (m <= 128; rows m..127 are zero).  D1^T
// accumulates over the run of tiles a CTA owns in one block row and is
// flushed once (with the shift term when the run holds the diagonal block);
// D2^T is double-buffered in TMEM and added to Y with red.global.add.v4.f32
// after every tile.
//
// Warp roles (256 threads, one CTA per SM, persistent over an equal share of
// the tiles in row-major order): warp 0 issues TMA, warp 1 owns TMEM and
// issues tcgen05.mma from one thread, warps 4-7 drain TMEM.  Every mbarrier
// wait is bounded; on a timeout the CTA records PSDPROJ_ETIMEOUT, unwinds and
// frees its TMEM.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "ctx.h"
#include "tc_common.cuh"

namespace {

using namespace tc;

constexpr int BN = 64;
constexpr int BM = 256;
constexpr int R = BM / BN;                       // column tiles per block-row step
constexpr int NSTAGE = 4;
constexpr uint32_t A_STAGE = BM * BN * 2;        // BF16 tile
constexpr uint32_t XJ_BYTES = 128 * BN * 2;      // 16 KB
constexpr uint32_t XI_BYTES = 128 * BM * 2;      // 64 KB
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_XJ = NSTAGE * A_STAGE;
constexpr uint32_t OFF_XI = OFF_XJ + 2 * XJ_BYTES;
constexpr uint32_t OFF_BAR = OFF_XI + XI_BYTES;
constexpr uint32_t SMEM_BYTES = OFF_BAR + 256;
constexpr uint32_t D1_COL = 0, D2_COL = BM;      // TMEM columns: D1 256, D2 2 x 64
constexpr uint32_t TMEM_COLS = 512;
constexpr int NT = 256;
constexpr long long WAIT_LIMIT = 4000000000LL;  // ~2 s at 2 GHz
static_assert(SMEM_BYTES <= 232448, "shared memory");

struct Bars {
    uint64_t fullA[NSTAGE], emptyA[NSTAGE];
    uint64_t fullXJ[2], emptyXJ[2];
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
    const float *X;
    int64_t ldx;
    float *Y;
    int64_t ldy;
    const double *d_shift;
    int *d_status;
    int vec_ok;
};

// tiles of block row I are J = R I .. nbc - 1; rows 0..I-1 hold
// sum_i (nbc - R i) = I nbc - R I (I - 1) / 2 of them
__device__ __forceinline__ int64_t row_start(int I, int nbc)
{
    return (int64_t)I * nbc - (int64_t)R * I * (I - 1) / 2;
}

__device__ __forceinline__ void tile_of(int64_t t, int nbc, int nbr, int &I, int &J)
{
    int lo = 0, hi = nbr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_start(mid, nbc) <= t) lo = mid; else hi = mid - 1;
    }
    I = lo;
    J = R * lo + (int)(t - row_start(lo, nbc));
}

// last tile of a run inside one block row
__device__ __forceinline__ bool last_in_row_run(int64_t t, int64_t t1, int I, const Params &P)
{
    return (t + 1 == t1) || (I + 1 < P.nbr && t + 1 == row_start(I + 1, P.nbc));
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

__global__ void __launch_bounds__(NT, 1)
sym_pass_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                     const Params P)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    Bars &B = *reinterpret_cast<Bars *>(sm + OFF_BAR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t0 = P.tiles * blockIdx.x / gridDim.x;
    const int64_t t1 = P.tiles * (blockIdx.x + 1) / gridDim.x;
    if ((smem_u32(sm) & 1023u) != 0u) {
        if (threadIdx.x == 0) psd_set_status(P.d_status, PSDPROJ_ECUDA);
        return;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&B.fullA[s], 1);
            mbar_init(&B.emptyA[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B.fullXJ[b], 1);
            mbar_init(&B.emptyXJ[b], 1);
            mbar_init(&B.d2full[b], 1);
            mbar_init(&B.d2empty[b], 4);
        }
        mbar_init(&B.fullXI, 1);
        mbar_init(&B.emptyXI, 1);
        mbar_init(&B.d1full, 1);
        mbar_init(&B.d1empty, 4);
        mbar_init(&B.mmadone, 1);
        B.abort = 0;
        fence_proxy_async_smem();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmX);
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

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            int curI = -1, xi_uses = 0;
            int64_t it = 0;
            for (int64_t t = t0; t < t1; ++t, ++it) {
                int I, J;
                tile_of(t, P.nbc, P.nbr, I, J);
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
                if (!mbar_wait(&B.emptyA[s], (us & 1) ^ 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                mbar_arrive_expect_tx(&B.fullA[s], A_STAGE);
                tma_load_2d(sm + OFF_A + s * A_STAGE, &tmA, BN * J, BM * I, &B.fullA[s]);
                const int b = (int)(it & 1);
                const uint32_t ub = (uint32_t)(it >> 1);
                if (!mbar_wait(&B.emptyXJ[b], (ub & 1) ^ 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                mbar_arrive_expect_tx(&B.fullXJ[b], XJ_BYTES);
                tma_load_2d(sm + OFF_XJ + b * XJ_BYTES, &tmX, BN * J, 0, &B.fullXJ[b]);
            }
            // wait (bounded) for the copies still in flight to land
            const int64_t n_it = it;
            for (int64_t k = (n_it > NSTAGE ? n_it - NSTAGE : 0); k < n_it; ++k)
                mbar_wait(&B.fullA[k % NSTAGE], (uint32_t)((k / NSTAGE) & 1), abort, WAIT_LIMIT);
            for (int64_t k = (n_it > 2 ? n_it - 2 : 0); k < n_it; ++k)
                mbar_wait(&B.fullXJ[k & 1], (uint32_t)((k >> 1) & 1), abort, WAIT_LIMIT);
            if (xi_uses > 0) mbar_wait(&B.fullXI, (uint32_t)((xi_uses - 1) & 1), abort, WAIT_LIMIT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            const uint32_t id1 = idesc_bf16(128, BM, 0, 0);
            const uint32_t id2 = idesc_bf16(128, BN, 0, 1);
            int curI = -1, seg = 0;
            int64_t it = 0;
            bool issued = false;
            for (int64_t t = t0; t < t1; ++t, ++it) {
                int I, J;
                tile_of(t, P.nbc, P.nbr, I, J);
                const bool first = (I != curI);
                const bool last = last_in_row_run(t, t1, I, P);
                if (first) {
                    if (!mbar_wait(&B.fullXI, seg & 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                    if (!mbar_wait(&B.d1empty, (seg & 1) ^ 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                    curI = I;
                }
                const int s = (int)(it % NSTAGE);
                const uint32_t us = (uint32_t)(it / NSTAGE);
                const int b = (int)(it & 1);
                const uint32_t ub = (uint32_t)(it >> 1);
                if (!mbar_wait(&B.fullA[s], us & 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                if (!mbar_wait(&B.fullXJ[b], ub & 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                if (!mbar_wait(&B.d2empty[b], (ub & 1) ^ 1, abort, WAIT_LIMIT)) { fail(B, P.d_status); break; }
                tc_fence_after();
                const uint32_t a_tile = smem_u32(sm + OFF_A + s * A_STAGE);
                const uint32_t xj = smem_u32(sm + OFF_XJ + b * XJ_BYTES);
                const uint32_t xi = smem_u32(sm + OFF_XI);
                // P1: D1^T += X_J^T A_IJ^T   (K = 64 tile columns)
#pragma unroll
                for (int kk = 0; kk < BN / 16; ++kk) {
                    const uint64_t ad = sdesc_sw128(xj + kk * 32, 16, 1024);
                    const uint64_t bd = sdesc_sw128(a_tile + kk * 32, 16, 1024);
                    mma_bf16_ss(tmem + D1_COL, ad, bd, id1, (!first || kk > 0) ? 1u : 0u);
                }
                // P2: D2^T = X_I^T A_IJ   (K = 256 tile rows)
#pragma unroll
                for (int kk = 0; kk < BM / 16; ++kk) {
                    const uint64_t ad = sdesc_sw128(xi + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024);
                    const uint64_t bd = sdesc_sw128(a_tile + kk * 2048, 16384, 1024);
                    mma_bf16_ss(tmem + D2_COL + BN * b, ad, bd, id2, kk > 0 ? 1u : 0u);
                }
                issued = true;
                mma_commit(&B.emptyA[s]);
                mma_commit(&B.emptyXJ[b]);
                mma_commit(&B.d2full[b]);
                if (last) {
                    mma_commit(&B.d1full);
                    mma_commit(&B.emptyXI);
                    ++seg;
                }
            }
            if (issued) {
                // all MMAs of this CTA complete before TMEM is released
                mma_commit(&B.mmadone);
                mbar_wait(&B.mmadone, 0, abort, WAIT_LIMIT);
            }
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------- epilogue
        const int q = warp & 3;                // TMEM lane quarter of this warp
        const int c = 32 * q + lane;           // column of X / Y held by this thread
        const bool cok = c < P.m;
        const double shift = P.d_shift ? *P.d_shift : 0.0;
        int curI = -1, seg = 0;
        bool has_diag = false;
        int64_t it = 0;
        float *ycol = P.Y + (int64_t)c * P.ldy;
        for (int64_t t = t0; t < t1; ++t, ++it) {
            int I, J;
            tile_of(t, P.nbc, P.nbr, I, J);
            if (I != curI) {
                curI = I;
                has_diag = (J == R * I);
            }
            const bool last = last_in_row_run(t, t1, I, P);
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
            if (cok) {
                const int64_t r0 = (int64_t)BN * J;
#pragma unroll
                for (int j = 0; j < 64; j += 4) {
                    const float *src = j < 32 ? v0 + j : v1 + (j - 32);
                    const int64_t r = r0 + j;
                    if (P.vec_ok && r + 3 < P.n) {
                        red_add_v4(ycol + r, src[0], src[1], src[2], src[3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (r + e < P.n) atomicAdd(ycol + r + e, src[e]);
                    }
                }
            }
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
                    if (cok) {
                        const int64_t rb = r0 + 32 * ch;
                        if (has_diag && shift != 0.0) {
                            const float *xc = P.X + (int64_t)c * P.ldx;
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                if (rb + e < P.n) v[e] = fmaf((float)shift, xc[rb + e], v[e]);
                        }
#pragma unroll
                        for (int e = 0; e < 32; e += 4) {
                            const int64_t r = rb + e;
                            if (P.vec_ok && r + 3 < P.n) {
                                red_add_v4(ycol + r, v[e], v[e + 1], v[e + 2], v[e + 3]);
                            } else {
#pragma unroll
                                for (int f = 0; f < 4; ++f)
                                    if (r + f < P.n) atomicAdd(ycol + r + f, v[e + f]);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&B.d1empty);
                ++seg;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// X (FP32, column-major) -> BF16 image used by the TMA loads of the pass
__global__ void to_bf16_kernel(const float *__restrict__ X, int64_t ldx, int64_t n, int m,
                               __nv_bfloat16 *__restrict__ H, int64_t ldh)
{
    const int64_t total = n * (int64_t)m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        H[c * ldh + i] = __float2bfloat16_rn(X[c * ldx + i]);
    }
}

// BF16 image A' of the block upper triangle of A (see the top of this file).
// Block: 16 rows x 64 columns, 16 threads per row, one float4 of A and one
// 8-byte store of A' per thread.  grid.x: 64-column tiles, grid.y: 16-row
// chunks; tiles left of the diagonal 256 x 256 block exit at once.
__global__ void __launch_bounds__(256)
pack_upper_bf16_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                       uint16_t *__restrict__ Ab, int64_t ldb, int vec)
{
    const int64_t r = (int64_t)blockIdx.y * 16 + (threadIdx.x >> 4);
    const int64_t cbase = (int64_t)blockIdx.x * BN;
    const int64_t blk0 = (r / BM) * BM;               // first column of the diagonal block
    if (cbase + BN <= blk0) return;                   // uniform across the block
    const int64_t c0 = cbase + 4 * (threadIdx.x & 15);
    float v[4];
    if (r < n && vec && c0 + 4 <= n) {
        const float4 a = __ldcs(reinterpret_cast<const float4 *>(A + r * lda + c0));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (r < n && c0 + q < n) ? A[r * lda + c0 + q] : 0.0f;
    }
    if (cbase < blk0 + BM) {
        // diagonal block: keep the strict upper part, halve the diagonal
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t c = c0 + q;
            v[q] = c > r ? v[q] : (c == r ? 0.5f * v[q] : 0.0f);
        }
    }
    uint2 o;
    o.x = pack_bf16(v[0], v[1]);
    o.y = pack_bf16(v[2], v[3]);
    *reinterpret_cast<uint2 *>(Ab + r * ldb + c0) = o;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

int64_t psd_bf16_image_pad(int64_t n) { return psd_round_up(n, BM); }

cudaError_t launch_pack_bf16(cudaStream_t s, const float *A, int64_t n, int64_t lda, uint16_t *Ab,
                             int64_t ldb)
{
    const int64_t npad = psd_bf16_image_pad(n);
    if (ldb < npad || (ldb % 8) != 0 || (reinterpret_cast<uintptr_t>(Ab) & 15) != 0)
        return cudaErrorInvalidValue;
    const int vec = (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    dim3 grid((unsigned)(npad / BN), (unsigned)(npad / 16));
    pack_upper_bf16_kernel<<<grid, 256, 0, s>>>(A, n, lda, Ab, ldb, vec);
    return cudaGetLastError();
}

cudaError_t launch_sym_pass_tc(cudaStream_t s, int sm_count, const uint16_t *Ab, int64_t ldb,
                               int64_t n, const float *X, int64_t ldx, int m,
                               const double *d_shift, float *Y, int64_t ldy, uint16_t *Xh,
                               int64_t ldh, int *d_status)
{
    const int64_t npad = psd_bf16_image_pad(n);
    if (m < 1 || m > 128) return cudaErrorNotSupported;
    if (ldb < npad || (ldb % 8) != 0 || (reinterpret_cast<uintptr_t>(Ab) & 15) != 0)
        return cudaErrorNotSupported;
    if ((ldh % 8) != 0 || (reinterpret_cast<uintptr_t>(Xh) & 15) != 0 || ldh < n)
        return cudaErrorNotSupported;
    auto encode = get_encode();
    if (!encode) return cudaErrorNotSupported;

    // BF16 image of X (rows n, columns m; TMA fills the rest with zeros)
    {
        const int64_t total = n * (int64_t)m;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        to_bf16_kernel<<<blocks, 256, 0, s>>>(X, ldx, n, m, reinterpret_cast<__nv_bfloat16 *>(Xh), ldh);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    CUtensorMap tmA, tmX;
    {
        cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)npad};
        cuuint64_t strides[1] = {(cuuint64_t)ldb * 2};
        cuuint32_t box[2] = {(cuuint32_t)BN, (cuuint32_t)BM};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(Ab), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
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
    P.nbr = (int)(npad / BM);
    P.nbc = (int)(npad / BN);
    P.tiles = (int64_t)P.nbr * P.nbc - (int64_t)R * P.nbr * (P.nbr - 1) / 2;
    P.X = X;
    P.ldx = ldx;
    P.Y = Y;
    P.ldy = ldy;
    P.d_shift = d_shift;
    P.d_status = d_status;
    P.vec_ok = ((ldy % 4) == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0);

    cudaError_t e = cudaMemset2DAsync(Y, (size_t)ldy * sizeof(float), 0, (size_t)n * sizeof(float),
                                      (size_t)m, s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sym_pass_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int grid = sm_count > 0 ? sm_count : 148;
    if ((int64_t)grid > P.tiles) grid = (int)P.tiles;
    sym_pass_bf16_kernel<<<grid, NT, SMEM_BYTES, s>>>(tmA, tmX, P);
    return cudaGetLastError();
}
