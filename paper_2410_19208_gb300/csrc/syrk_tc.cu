// Reconstruction P = W W^T (last line of Alg. 2) on the tcgen05 tensor cores.
//
// W (n x r, column-major FP32; r = r+ read on the device) is split once into
// BF16 images W = W_hi + W_lo; each 128 x 128 tile of P over the upper block
// triangle is D = W_I W_J^T = hi.hi^T + hi.lo^T + lo.hi^T (split BF16,
// FP32 accumulation in TMEM; ~2^-16 relative error per entry).  Both
// operands are MN-major (W is column-major) and TMA-loaded with the 128-byte
// swizzle: atoms of 64 rows x 8 columns of W, two atoms along M (and N).
// The kernel is store-bound (1.6 GB of P at n = 20000): D is double-buffered
// in TMEM so the MMAs of the next tile overlap the stores of this one; eight
// epilogue warps write the tile and, off the diagonal, its mirror by TMA
// tensor stores of 32 x 32 boxes staged in shared memory (128-byte swizzle,
// one 4 KB staging box per warp), so P is written in whole lines.  Diagonal
// tiles of the upper-only mode and P without 16-byte aligned rows take
// per-thread streaming stores.
// Warp roles (384 threads): warp 0 TMA, warp 1 TMEM owner + MMA issuer,
// warps 4-11 epilogue.  Every mbarrier wait is bounded.
#include <cuda_bf16.h>
#include <cstring>
#include <cudaTypedefs.h>

#include "ctx.h"
#include "tc_common.cuh"

namespace {

using namespace tc;

constexpr int TS = 128;                      // output tile side
constexpr int KMAX = 128;                    // largest r (W columns)
constexpr uint32_t OP_BYTES = TS * KMAX * 2; // one BF16 operand image (32 KB)
constexpr uint32_t ATOM_COL = 64 * 2 * KMAX; // bytes of one 64-row atom column (16 KB)
constexpr uint32_t OFF_WI = 0;               // hi, lo
constexpr uint32_t OFF_WJ = 2 * OP_BYTES;    // [2 buffers][hi, lo]
constexpr uint32_t STG_BYTES = 32 * 32 * 4;  // epilogue staging box per warp
constexpr uint32_t OFF_STG = OFF_WJ + 4 * OP_BYTES;
constexpr uint32_t OFF_BAR = OFF_STG + 8 * STG_BYTES;
constexpr uint32_t SMEM_BYTES = OFF_BAR + 256;
static_assert(SMEM_BYTES <= 232448, "shared memory");
static_assert(OFF_STG % 1024 == 0, "swizzle atoms");
constexpr int NT = 384;
constexpr uint32_t TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 4000000000LL;

struct Bars {
    uint64_t fullWI, emptyWI;
    uint64_t fullWJ[2], emptyWJ[2];
    uint64_t dfull[2], dempty[2];
    uint64_t mmadone;
    uint32_t tmem_base;
    int abort;
};

struct Params {
    int64_t n;
    int nb;
    int64_t tiles;
    const int *d_rank;
    int m;
    float *P;
    int64_t ldp;
    int upper_only;
    int nprod;        // 3: split BF16, 1: BF16 hi only
    int *d_status;
    long long wait_limit;   // cycles a pipeline wait may spin (opts.spin_limit; 0: WAIT_LIMIT)
    int vec_ok;
    int tma_p;        // P written by TMA stores (16-byte aligned rows)
};

__device__ __forceinline__ int64_t row_start(int I, int nb)
{
    // tiles of block rows 0..I-1: sum (nb - i)
    return (int64_t)I * nb - (int64_t)I * (I - 1) / 2;
}

__device__ __forceinline__ void tile_of(int64_t t, int nb, int &I, int &J)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_start(mid, nb) <= t) lo = mid; else hi = mid - 1;
    }
    I = lo;
    J = lo + (int)(t - row_start(lo, nb));
}

__device__ __forceinline__ void fail(Bars &B, int *st)
{
    B.abort = 1;
    psd_set_status(st, PSDPROJ_ETIMEOUT);
}

__device__ __forceinline__ void st_cs(float *p, float v)
{
    asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cs4(float *p, float a, float b, float c, float d)
{
    asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

__global__ void __launch_bounds__(NT, 1)
syrk_bf16x3_kernel(const __grid_constant__ CUtensorMap tmHi, const __grid_constant__ CUtensorMap tmLo,
                   const __grid_constant__ CUtensorMap tmP, const Params P)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const long long WL = P.wait_limit > 0 ? P.wait_limit : WAIT_LIMIT;
    Bars &B = *reinterpret_cast<Bars *>(sm + OFF_BAR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles dealt round-robin (tile t to CTA t % grid): CTAs running at the
    // same time write neighbouring 128-column blocks of the same 128 rows
    const int64_t t0 = blockIdx.x, t1 = P.tiles, tstep = gridDim.x;
    if ((smem_u32(sm) & 1023u) != 0u) {
        if (threadIdx.x == 0) psd_set_status(P.d_status, PSDPROJ_ECUDA);
        return;
    }
    int r = P.d_rank ? *P.d_rank : P.m;
    r = max(0, min(r, min(P.m, KMAX)));
    const int ksteps = (r + 15) / 16;
    const uint32_t op_tx = OP_BYTES;  // a box always lands whole (OOB columns zero-filled)

    if (threadIdx.x == 0) {
        mbar_init(&B.fullWI, 1);
        mbar_init(&B.emptyWI, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B.fullWJ[b], 1);
            mbar_init(&B.emptyWJ[b], 1);
            mbar_init(&B.dfull[b], 1);
            mbar_init(&B.dempty[b], 8);
        }
        mbar_init(&B.mmadone, 1);
        B.abort = 0;
        fence_proxy_async_smem();
        prefetch_tmap(&tmHi);
        prefetch_tmap(&tmLo);
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
    const bool lo_too = P.nprod == 3;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            int curI = -1, wi_uses = 0;
            int64_t it = 0;
            for (int64_t t = t0; t < t1; t += tstep, ++it) {
                int I, J;
                tile_of(t, P.nb, I, J);
                if (I != curI) {
                    if (!mbar_wait(&B.emptyWI, (wi_uses & 1) ^ 1, abort, WL)) { fail(B, P.d_status); break; }
                    mbar_arrive_expect_tx(&B.fullWI, op_tx * (lo_too ? 2u : 1u));
                    for (int a = 0; a < 2; ++a) {
                        tma_load_2d(sm + OFF_WI + a * ATOM_COL, &tmHi, TS * I + 64 * a, 0, &B.fullWI);
                        if (lo_too)
                            tma_load_2d(sm + OFF_WI + OP_BYTES + a * ATOM_COL, &tmLo, TS * I + 64 * a, 0, &B.fullWI);
                    }
                    ++wi_uses;
                    curI = I;
                }
                const int b = (int)(it & 1);
                const uint32_t ub = (uint32_t)(it >> 1);
                if (!mbar_wait(&B.emptyWJ[b], (ub & 1) ^ 1, abort, WL)) { fail(B, P.d_status); break; }
                mbar_arrive_expect_tx(&B.fullWJ[b], op_tx * (lo_too ? 2u : 1u));
                uint8_t *dst = sm + OFF_WJ + b * 2 * OP_BYTES;
                for (int a = 0; a < 2; ++a) {
                    tma_load_2d(dst + a * ATOM_COL, &tmHi, TS * J + 64 * a, 0, &B.fullWJ[b]);
                    if (lo_too) tma_load_2d(dst + OP_BYTES + a * ATOM_COL, &tmLo, TS * J + 64 * a, 0, &B.fullWJ[b]);
                }
            }
            const int64_t n_it = it;
            for (int64_t k = (n_it > 2 ? n_it - 2 : 0); k < n_it; ++k)
                mbar_wait_drain(&B.fullWJ[k & 1], (uint32_t)((k >> 1) & 1), WAIT_LIMIT);
            if (wi_uses > 0) mbar_wait_drain(&B.fullWI, (uint32_t)((wi_uses - 1) & 1), WAIT_LIMIT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            const uint32_t id = idesc_bf16(TS, TS, 1, 1);
            int curI = -1, seg = 0;
            int64_t it = 0;
            for (int64_t t = t0; t < t1; t += tstep, ++it) {
                int I, J;
                tile_of(t, P.nb, I, J);
                // the CTA's next tile is in another block row (or there is none)
                const bool last = (t + tstep >= t1) || (I + 1 < P.nb && t + tstep >= row_start(I + 1, P.nb));
                if (I != curI) {
                    if (!mbar_wait(&B.fullWI, seg & 1, abort, WL)) { fail(B, P.d_status); break; }
                    curI = I;
                }
                const int b = (int)(it & 1);
                const uint32_t ub = (uint32_t)(it >> 1);
                if (!mbar_wait(&B.fullWJ[b], ub & 1, abort, WL)) { fail(B, P.d_status); break; }
                if (!mbar_wait(&B.dempty[b], (ub & 1) ^ 1, abort, WL)) { fail(B, P.d_status); break; }
                tc_fence_after();
                const uint32_t ahi = smem_u32(sm + OFF_WI), alo = ahi + OP_BYTES;
                const uint32_t bhi = smem_u32(sm + OFF_WJ + b * 2 * OP_BYTES), blo = bhi + OP_BYTES;
                const uint32_t d = tmem + TS * b;
                uint32_t acc = 0;
                for (int kk = 0; kk < ksteps; ++kk) {
                    // MN-major: 16 columns of W = 16 rows of 128 bytes per atom column;
                    // LBO = stride between the two 64-row atom columns, SBO = 8 rows
                    const uint32_t off = kk * 16 * 128;
                    mma_bf16_ss(d, sdesc_sw128(ahi + off, ATOM_COL, 1024), sdesc_sw128(bhi + off, ATOM_COL, 1024), id, acc);
                    acc = 1;
                    if (lo_too) {
                        mma_bf16_ss(d, sdesc_sw128(ahi + off, ATOM_COL, 1024), sdesc_sw128(blo + off, ATOM_COL, 1024), id, 1);
                        mma_bf16_ss(d, sdesc_sw128(alo + off, ATOM_COL, 1024), sdesc_sw128(bhi + off, ATOM_COL, 1024), id, 1);
                    }
                }
                mma_commit(&B.emptyWJ[b]);
                mma_commit(&B.dfull[b]);
                if (last) {
                    mma_commit(&B.emptyWI);
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
        const int q = warp & 3;               // TMEM lane quarter
        const int g = (warp - 4) >> 2;        // column half of the tile
        int64_t it = 0;
        for (int64_t t = t0; t < t1; t += tstep, ++it) {
            int I, J;
            tile_of(t, P.nb, I, J);
            const int b = (int)(it & 1);
            const uint32_t ub = (uint32_t)(it >> 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&B.dfull[b], ub & 1, abort, WL) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) { if (lane == 0) fail(B, P.d_status); break; }
            tc_fence_after();
            float v[64];
            {
                float v0[32], v1[32];
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + TS * b + 64 * g;
                if (ksteps > 0) {
                    tmem_ld32(ta, v0);
                    tmem_ld32(ta + 32, v1);
                } else {
#pragma unroll
                    for (int e = 0; e < 32; ++e) { v0[e] = 0.0f; v1[e] = 0.0f; }
                }
#pragma unroll
                for (int e = 0; e < 32; ++e) { v[e] = v0[e]; v[32 + e] = v1[e]; }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.dempty[b]);
            const int64_t gi = (int64_t)TS * I + 32 * q + lane;   // row of P
            const int64_t gj0 = (int64_t)TS * J + 64 * g;          // first column
            const bool diag = (I == J);
            if (P.tma_p && !(diag && P.upper_only)) {
                // 32 x 32 boxes: rows 32q.. of the tile, columns gj0 + 32c ..; the
                // mirror box holds the same entries transposed
                uint8_t *stg = sm + OFF_STG + (warp - 4) * STG_BYTES;
                const int64_t i0 = (int64_t)TS * I + 32 * q;
                for (int c = 0; c < 2; ++c) {
                    const int64_t j0 = gj0 + 32 * c;
                    if (j0 >= P.n || i0 >= P.n) continue;           // box outside P
                    if (lane == 0) bulk_wait_read();
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        *reinterpret_cast<float4 *>(stg + lane * 128 + ((k ^ (lane & 7)) << 4)) =
                            make_float4(v[32 * c + 4 * k], v[32 * c + 4 * k + 1], v[32 * c + 4 * k + 2],
                                        v[32 * c + 4 * k + 3]);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&tmP, (int)j0, (int)i0, stg);
                        bulk_commit();
                    }
                    if (diag || P.upper_only) continue;      // no mirror: diagonal tile or upper only
                    if (lane == 0) bulk_wait_read();
                    __syncwarp();
                    // mirror: row e of the box is column j0 + e of the tile; this
                    // lane's entry goes to its column (lane) of every row
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        *reinterpret_cast<float *>(stg + e * 128 + (((lane >> 2) ^ (e & 7)) << 4) + 4 * (lane & 3)) =
                            v[32 * c + e];
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&tmP, (int)i0, (int)j0, stg);
                        bulk_commit();
                    }
                }
                continue;
            }
            if (gi < P.n) {
                float *row = P.P + gi * P.ldp;
#pragma unroll
                for (int e = 0; e < 64; e += 4) {
                    const int64_t j = gj0 + e;
                    const bool full = P.vec_ok && j + 3 < P.n && (!diag || !P.upper_only || j >= gi);
                    if (full) {
                        st_cs4(row + j, v[e], v[e + 1], v[e + 2], v[e + 3]);
                    } else {
#pragma unroll
                        for (int f = 0; f < 4; ++f)
                            if (j + f < P.n && (!diag || !P.upper_only || j + f >= gi)) st_cs(row + j + f, v[e + f]);
                    }
                }
            }
            if (!diag && !P.upper_only && gi < P.n) {
                // mirror: P[j][gi] for the 64 columns j; lanes write consecutive gi
#pragma unroll
                for (int e = 0; e < 64; ++e) {
                    const int64_t j = gj0 + e;
                    if (j < P.n) st_cs(P.P + j * P.ldp + gi, v[e]);
                }
            }
        }
    }

    if (warp >= 4 && lane == 0 && P.tma_p) bulk_wait_all();

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// W (FP32, column-major) -> BF16 hi and lo images, rows n, columns m
__global__ void split_bf16_kernel(const float *__restrict__ W, int64_t ldw, int64_t n, int m,
                                  __nv_bfloat16 *__restrict__ H, __nv_bfloat16 *__restrict__ L,
                                  int64_t ldh)
{
    const int64_t total = n * (int64_t)m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        const float w = W[c * ldw + i];
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        H[c * ldh + i] = h;
        L[c * ldh + i] = __float2bfloat16_rn(w - __bfloat162float(h));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() { return tensor_map_encoder(); }

bool encode_w(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap *map, void *base, int64_t n,
              int m, int64_t ldh)
{
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)ldh * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)KMAX};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_syrk_tc(cudaStream_t s, int sm_count, const float *W, int64_t ldw, int64_t n,
                           int m, const int *d_rank, float *P, int64_t ldp, int upper_only,
                           uint16_t *Whi, uint16_t *Wlo, int64_t ldh, int *d_status, long long wait_limit,
                           int prepared)
{
    if (m < 1 || m > KMAX) return cudaErrorNotSupported;
    if ((ldh % 8) != 0 || ldh < n || (reinterpret_cast<uintptr_t>(Whi) & 15) ||
        (reinterpret_cast<uintptr_t>(Wlo) & 15))
        return cudaErrorNotSupported;
    auto enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    if (!prepared) {
        const int64_t total = n * (int64_t)m;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        split_bf16_kernel<<<blocks, 256, 0, s>>>(W, ldw, n, m, reinterpret_cast<__nv_bfloat16 *>(Whi),
                                                 reinterpret_cast<__nv_bfloat16 *>(Wlo), ldh);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    CUtensorMap tmHi, tmLo;
    if (!encode_w(enc, &tmHi, Whi, n, m, ldh) || !encode_w(enc, &tmLo, Wlo, n, m, ldh))
        return cudaErrorInvalidValue;
    Params p;
    p.n = n;
    p.nb = (int)((n + TS - 1) / TS);
    p.tiles = (int64_t)p.nb * (p.nb + 1) / 2;
    p.d_rank = d_rank;
    p.m = m;
    p.P = P;
    p.ldp = ldp;
    p.upper_only = upper_only;
    p.nprod = 3;
    p.d_status = d_status;
    p.wait_limit = wait_limit;
    p.vec_ok = ((ldp % 4) == 0) && ((reinterpret_cast<uintptr_t>(P) & 15) == 0);
    p.tma_p = p.vec_ok;
    CUtensorMap tmP;
    memset(&tmP, 0, sizeof(tmP));
    if (p.tma_p) {
        cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
        cuuint64_t strides[1] = {(cuuint64_t)ldp * 4};
        cuuint32_t box[2] = {32, 32};
        cuuint32_t estr[2] = {1, 1};
        if (enc(&tmP, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, P, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            p.tma_p = 0;
    }
    cudaError_t e = cudaFuncSetAttribute(syrk_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int grid = sm_count > 0 ? sm_count : 148;
    if ((int64_t)grid > p.tiles) grid = (int)p.tiles;
    syrk_bf16x3_kernel<<<grid, NT, SMEM_BYTES, s>>>(tmHi, tmLo, tmP, p);
    return cudaGetLastError();
}
