// Symmetric pass Y = A X + shift X in TF32 on the 5th-generation tensor cores
// (tcgen05 kind::tf32, sm_103a): the TF32 form of the sketch, power and core
// products of Alg. 1 / Alg. 2.
//
// The BF16 pass uses every stored upper-triangle tile twice (A_IJ X_J and
// A_IJ^T X_I), the second product with an MN-major B operand.  kind::tf32
// gave zero for that MN-major product on this GPU, so the TF32 form keeps to
// K-major operands only: pack_full_tf32_kernel writes a TF32 image of the
// FULL symmetric matrix (the lower triangle mirrored from the upper one,
// which alone is read), and every tile feeds one product
//   D^T (m x 256) += X_J^T (m x 32) . A_IJ^T,   i.e.  Y_I += A_IJ X_J,
// with M = 128 rows of X^T (m <= 128).  A pass therefore reads n^2 x 4 bytes
// of image (twice the upper triangle's FP32 bytes), in exchange for a
// four-stage pipeline with no resident X_I panel.
//
// Image: tile (I, J) of 256 rows x 32 columns at index I * nbc + J (nbc = 8
// nbr), 32 KB each, row r at r * 128 bytes, its 16-byte chunk k (columns
// 4k..4k+3) at position k ^ (r & 7): the 128-byte-swizzled K-major layout of
// a UMMA operand, so a stage is one bulk copy.  Entries are rounded to TF32
// (nearest, ties away from zero) and padded with zeros past row / column n.
//
// Warp roles (256 threads, one CTA per SM, persistent over an equal share of
// the tiles in row-major order): warp 0 issues the copies, warp 1 owns TMEM
// and issues tcgen05.mma from one thread, warps 4-7 drain TMEM.  The
// accumulator of a run of tiles in one block row is double-buffered in TMEM
// (2 x 256 columns) and added to Y by TMA bulk reduce-add (scalar atomics when
// Y is not 16-byte aligned with ld % 4 == 0).  The sweep that rounds X to
// TF32 starts Y at shift X, so the pass itself has no shift term.  Every mbarrier wait is
// bounded; on a timeout the CTA records PSDPROJ_ETIMEOUT, unwinds and frees
// its TMEM.
#include <cstring>
#include <cudaTypedefs.h>

#include "ctx.h"
#include "tc_common.cuh"

namespace {

using namespace tc;

constexpr int BM = PSD_TILE_M;                   // 256 tile rows
constexpr int BN = PSD_TILE32_N;                 // 32 tile columns (128 bytes)
constexpr int KSTEP = 8;                         // K of one kind::tf32 MMA
constexpr int NSTAGE = 4;
constexpr uint32_t A_BYTES = (uint32_t)PSD_TILE_BYTES;
constexpr uint32_t XJ_BYTES = 128 * BN * 4;      // X_J^T rows 0..127 (16 KB)
constexpr uint32_t STAGE = A_BYTES + XJ_BYTES;
constexpr uint32_t STG_BYTES = 32 * 32 * 4;      // epilogue staging box per warp
constexpr uint32_t OFF_STG = NSTAGE * STAGE;
constexpr uint32_t OFF_BAR = OFF_STG + 4 * STG_BYTES;
constexpr uint32_t SMEM_BYTES = OFF_BAR + 256;
constexpr uint32_t TMEM_COLS = 512;              // two 256-column accumulators
constexpr int NT = 256;
constexpr long long WAIT_LIMIT = 4000000000LL;  // ~2 s at 2 GHz
static_assert(SMEM_BYTES <= 232448, "shared memory");
static_assert(STAGE % 1024 == 0 && OFF_STG % 1024 == 0, "swizzle atoms");
static_assert(BN * 4 == 128 && BN / KSTEP == 4, "a tile row is one 128-byte swizzle row");

// tcgen05 instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B
// TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 (17-22), M >> 4 (24-28)
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BM >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_tf32_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}

struct Bars {
    uint64_t full[NSTAGE], empty[NSTAGE];
    uint64_t dfull[2], dempty[2];
    uint64_t mmadone;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(Bars) <= 256, "barrier block");

struct Params {
    int64_t n;
    int m;
    int nbc;
    int64_t tiles;
    float *Y;
    int64_t ldy;
    int *d_status;
    long long wait_limit;   // cycles a pipeline wait may spin (opts.spin_limit; 0: WAIT_LIMIT)
    int tma_y;
};

__device__ __forceinline__ void fail(Bars &B, int *st)
{
    B.abort = 1;
    psd_set_status(st, PSDPROJ_ETIMEOUT);
}

// FP32 -> TF32, round to nearest with ties away from zero (low 13 mantissa
// bits zero)
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Add 32 rows (r0 .. r0+31) of Y column c = 32 q + lane, held in v.  With
// TMA: stage a swizzled 32 x 32 box (chunk j of column c at
// c * 128 + ((j ^ (c & 7)) << 4)) and reduce-add it after the previous
// reduce from this box has been read.
__device__ __forceinline__ void flush32(const Params &P, const CUtensorMap *tmY, uint8_t *stg, int q,
                                        int lane, int64_t r0, const float (&v)[32])
{
    const int c = 32 * q + lane;
    if (P.tma_y) {
        if (r0 >= P.n || 32 * q >= P.m) return;
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
sym_pass_tf32_kernel(const uint8_t *__restrict__ At, const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmY, const Params P)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const long long WL = P.wait_limit > 0 ? P.wait_limit : WAIT_LIMIT;
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
            mbar_init(&B.full[s], 1);
            mbar_init(&B.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B.dfull[b], 1);
            mbar_init(&B.dempty[b], 4);
        }
        mbar_init(&B.mmadone, 1);
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

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            int64_t it = 0;
            for (int64_t t = t0; t < t1; ++t, ++it) {
                const int J = (int)(t % P.nbc);
                const int s = (int)(it % NSTAGE);
                const uint32_t us = (uint32_t)(it / NSTAGE);
                if (!mbar_wait(&B.empty[s], (us & 1) ^ 1, abort, WL)) { fail(B, P.d_status); break; }
                mbar_arrive_expect_tx(&B.full[s], STAGE);
                bulk_load(sm + s * STAGE, At + t * PSD_TILE_BYTES, A_BYTES, &B.full[s]);
                tma_load_2d(sm + s * STAGE + A_BYTES, &tmX, BN * J, 0, &B.full[s]);
            }
            // wait (bounded) for the copies still in flight to land
            for (int64_t k = (it > NSTAGE ? it - NSTAGE : 0); k < it; ++k)
                mbar_wait_drain(&B.full[k % NSTAGE], (uint32_t)((k / NSTAGE) & 1), WAIT_LIMIT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            int seg = 0;
            int64_t it = 0;
            for (int64_t t = t0; t < t1; ++t, ++it) {
                const int J = (int)(t % P.nbc);
                const bool first = (t == t0) || (J == 0);
                const bool last = (J == P.nbc - 1) || (t + 1 == t1);
                const int b = seg & 1;
                if (first && !mbar_wait(&B.dempty[b], ((uint32_t)(seg >> 1) & 1) ^ 1, abort, WL)) {
                    fail(B, P.d_status);
                    break;
                }
                const int s = (int)(it % NSTAGE);
                const uint32_t us = (uint32_t)(it / NSTAGE);
                if (!mbar_wait(&B.full[s], us & 1, abort, WL)) { fail(B, P.d_status); break; }
                tc_fence_after();
                const uint32_t a_tile = smem_u32(sm + s * STAGE);
                const uint32_t xj = a_tile + A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BN / KSTEP; ++kk) {
                    const uint64_t ad = sdesc_sw128(xj + kk * 32, 16, 1024);
                    const uint64_t bd = sdesc_sw128(a_tile + kk * 32, 16, 1024);
                    mma_tf32_ss(tmem + (uint32_t)(BM * b), ad, bd, (!first || kk > 0) ? 1u : 0u);
                }
                mma_commit(&B.empty[s]);
                if (last) {
                    mma_commit(&B.dfull[b]);
                    ++seg;
                }
            }
            // every MMA of this CTA completes before TMEM is released, also
            // when the CTA gave up (a commit with none pending arrives at once)
            mma_commit(&B.mmadone);
            mbar_wait_drain(&B.mmadone, 0, WAIT_LIMIT);
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------- epilogue
        const int q = warp & 3;                // TMEM lane quarter of this warp
        uint8_t *stg = sm + OFF_STG + q * STG_BYTES;
        int seg = 0;
        for (int64_t t = t0; t < t1; ++seg) {
            const int64_t I = t / P.nbc;
            const int64_t row_end = (I + 1) * P.nbc;
            const int b = seg & 1;
            {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&B.dfull[b], (uint32_t)(seg >> 1) & 1, abort, WL) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { if (lane == 0) fail(B, P.d_status); break; }
            }
            tc_fence_after();
            const int64_t r0 = (int64_t)BM * I;
#pragma unroll 1
            for (int ch = 0; ch < BM / 32; ++ch) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(BM * b + 32 * ch), v);
                flush32(P, &tmY, stg, q, lane, r0 + 32 * ch, v);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.dempty[b]);
            t = row_end < t1 ? row_end : t1;
        }
        if (lane == 0 && P.tma_y) bulk_wait_all();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// X (FP32, column-major) -> X rounded to TF32 in the aligned buffer that the
// pass loads by TMA; Y (a different buffer) starts at shift X in the same
// sweep (shift = *d_shift, 0 when d_shift is NULL).  Grid: x over 1024-row
// chunks, y over the m columns.
__global__ void __launch_bounds__(256)
to_tf32_kernel(const float *__restrict__ X, int64_t ldx, int64_t n, float *__restrict__ Xf, int64_t ldf,
               float *__restrict__ Y, int64_t ldy, const double *__restrict__ d_shift)
{
    const int c = blockIdx.y;
    const float shift = d_shift ? (float)*d_shift : 0.0f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = (int64_t)blockIdx.x * 1024 + r * 256 + threadIdx.x;
        if (i >= n) break;
        const float x = X[(int64_t)c * ldx + i];
        Xf[(int64_t)c * ldf + i] = tf32_rna(x);
        Y[(int64_t)c * ldy + i] = shift * x;
    }
}

// byte offset of the 16-byte chunk holding columns C..C+3 (C % 4 == 0) of
// row R in the full TF32 image
__device__ __forceinline__ int64_t image_off(int64_t R, int64_t C, int nbc)
{
    const int64_t I = R >> 8, J = C >> 5;
    const int rt = (int)(R & 255), k = (int)((C & 31) >> 2);
    return (I * nbc + J) * PSD_TILE_BYTES + rt * 128 + ((k ^ (rt & 7)) << 4);
}

// Full TF32 image from the upper triangle of A.  Block: one 64 x 64 block
// (by, bx) with bx >= by of the padded matrix, staged in shared memory (row
// stride 65 words); it is written at (by, bx) and, off the diagonal, its
// transpose at (bx, by).  In a diagonal block the entries below the diagonal
// are taken from their mirror images above it.  Each thread moves four
// float4 chunks (rows 16 apart) in each direction.
__global__ void __launch_bounds__(256)
pack_full_tf32_kernel(const float *__restrict__ A, int64_t n, int64_t lda, uint8_t *__restrict__ At,
                      int nbc, int vec)
{
    const int bx = blockIdx.x, by = blockIdx.y;
    if (bx < by) return;                              // uniform across the block
    __shared__ float S[64][65];
    const int64_t r0 = (int64_t)by * 64, c0 = (int64_t)bx * 64;
    const int k = threadIdx.x & 15;                   // float4 chunk within a 64-wide row
    const bool diag = bx == by;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = (threadIdx.x >> 4) + 16 * u;
        const int64_t r = r0 + i, cc = c0 + 4 * k;
        float v[4];
        if (r < n && vec && cc + 4 <= n && !diag) {
            const float4 a = __ldcs(reinterpret_cast<const float4 *>(A + r * lda + cc));
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t c = cc + j;
                // the upper triangle only (c >= r); the rest is filled below
                v[j] = (r < n && c < n && c >= r) ? A[r * lda + c] : 0.0f;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) S[i][4 * k + j] = v[j];
    }
    __syncthreads();
    if (diag) {
        // mirror the strict upper part into the lower one
        for (int e = threadIdx.x; e < 64 * 64; e += 256) {
            const int i = e >> 6, j = e & 63;
            if (j < i) S[i][j] = S[j][i];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = (threadIdx.x >> 4) + 16 * u;
        // block (by, bx): row r0 + i, columns c0 + 4k .. + 3
        float4 o = make_float4(tf32_rna(S[i][4 * k]), tf32_rna(S[i][4 * k + 1]), tf32_rna(S[i][4 * k + 2]),
                               tf32_rna(S[i][4 * k + 3]));
        *reinterpret_cast<float4 *>(At + image_off(r0 + i, c0 + 4 * k, nbc)) = o;
        if (!diag) {
            // block (bx, by): row c0 + i, columns r0 + 4k .. + 3 = column i of S
            o = make_float4(tf32_rna(S[4 * k][i]), tf32_rna(S[4 * k + 1][i]), tf32_rna(S[4 * k + 2][i]),
                            tf32_rna(S[4 * k + 3][i]));
            *reinterpret_cast<float4 *>(At + image_off(c0 + i, r0 + 4 * k, nbc)) = o;
        }
    }
}

bool encode_tall(CUtensorMap *tm, const float *base, int64_t n, int m, int64_t ld, int box_rows,
                 int box_cols)
{
    auto encode = tensor_map_encoder();
    if (!encode) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    cuuint32_t estr[2] = {1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_pack_tf32(cudaStream_t s, const float *A, int64_t n, int64_t lda, float *At)
{
    if ((reinterpret_cast<uintptr_t>(At) & 15) != 0) return cudaErrorInvalidValue;
    const int nbr = (int)((n + BM - 1) / BM);
    const int nb64 = nbr * (BM / 64);
    const int vec = (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    dim3 grid((unsigned)nb64, (unsigned)nb64);
    pack_full_tf32_kernel<<<grid, 256, 0, s>>>(A, n, lda, reinterpret_cast<uint8_t *>(At),
                                               nbr * (BM / BN), vec);
    return cudaGetLastError();
}

cudaError_t launch_sym_pass_tf32(cudaStream_t s, int sm_count, const float *At, int64_t n,
                                 const float *X, int64_t ldx, int m, const double *d_shift,
                                 float *Y, int64_t ldy, float *Xf, int64_t ldf, int *d_status,
                                 long long wait_limit)
{
    if (m < 1 || m > 128) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(At) & 15) != 0) return cudaErrorNotSupported;
    if ((ldf % 4) != 0 || (reinterpret_cast<uintptr_t>(Xf) & 15) != 0 || ldf < n) return cudaErrorNotSupported;
    if (!tensor_map_encoder()) return cudaErrorNotSupported;

    if (n > 0)
        to_tf32_kernel<<<dim3((unsigned)((n + 1023) / 1024), (unsigned)m), 256, 0, s>>>(X, ldx, n, Xf, ldf, Y, ldy,
                                                                                  d_shift);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // X_J^T: 32 rows of X (128 bytes) x 128 columns; columns >= m read as zero
    CUtensorMap tmX;
    if (!encode_tall(&tmX, Xf, n, m, ldf, BN, 128)) return cudaErrorInvalidValue;

    Params P;
    P.n = n;
    P.m = m;
    P.nbc = (int)((n + BM - 1) / BM) * (BM / BN);
    P.tiles = psd_tile32_count(n);
    P.Y = Y;
    P.ldy = ldy;
    P.d_status = d_status;
    P.wait_limit = wait_limit;
    P.tma_y = ((ldy % 4) == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0);
    CUtensorMap tmY;
    memset(&tmY, 0, sizeof(tmY));
    if (P.tma_y) {
        auto encode = tensor_map_encoder();
        cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
        cuuint64_t strides[1] = {(cuuint64_t)ldy * 4};
        cuuint32_t box[2] = {32, 32};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&tmY, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Y, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            P.tma_y = 0;
    }
    e = cudaFuncSetAttribute(sym_pass_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int grid = sm_count > 0 ? sm_count : 148;
    if ((int64_t)grid > P.tiles) grid = (int)P.tiles;
    sym_pass_tf32_kernel<<<grid, NT, SMEM_BYTES, s>>>(reinterpret_cast<const uint8_t *>(At), tmX, tmY, P);
    return cudaGetLastError();
}
