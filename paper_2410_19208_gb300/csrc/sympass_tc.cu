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
// Each tile (with the X_J tile loaded by TMA beside it, two to four stages
// in flight) feeds two products:
//   P1  D1^T (m x BM) += X_J^T (m x 64) . A'_IJ^T   (B operand K-major)
//   P2  D2^T (m x 64)   = X_I^T (m x BM) . A'_IJ    (B operand MN-major)
// with M = 128 rows of X^T.  The A operand of P1 and both B operands are
// read from shared memory; X_I^T, the A operand of P2, is copied into TMEM
// once per block row (shared-memory bandwidth, not the tensor pipe, bounds
// the pass, and P2 would otherwise read X_I from shared memory sixteen
// times per tile).  Only MR = 64, 112 or 128 rows of X^T (m <= MR)
// are staged, which leaves shared memory for the stages and eight staging
// boxes; accumulator lanes >= m are never stored.  D1^T accumulates over the
// run of tiles a CTA owns in one block row and is flushed once; D2^T is
// double-buffered in TMEM and added to Y after every tile.  The shift term
// is not in the pass: the sweep that converts X to BF16 starts Y at shift X
// (or adds it), so a run that holds a diagonal block drains D1 without extra
// global reads.  Both are added by TMA bulk reduce-add from a swizzled
// 32 x 32 staging box per epilogue warp (scalar atomics when Y is not
// 16-byte aligned with ld % 4 == 0).
//
// Warp roles (384 threads, one CTA per SM, persistent over a cost-balanced
// range of the tiles in row-major order): warp 0 issues the copies, warp 1
// owns TMEM and issues every tcgen05 operation (one thread), warps 4-11
// drain TMEM, two per TMEM lane quarter, so that every epilogue warp stages
// and reduces one 32 x 32 box of D2 per tile.  Every mbarrier wait is bounded; on a timeout the CTA records
// PSDPROJ_ETIMEOUT, unwinds and frees its TMEM.
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
constexpr uint32_t A_BYTES = BM * BN * 2;        // BF16 tile of A' (32 KB)
constexpr uint32_t STG_BYTES = 32 * 32 * 4;      // epilogue staging box per warp
constexpr int NEPI = 8;                          // epilogue warps (two per TMEM lane quarter)
constexpr int NT = 32 * (4 + NEPI);
// TMEM columns: D1^T 256, D2^T 128 (a group of two tiles), X_I^T (the A
// operand of P2, K = 256 BF16 values per lane) 128
constexpr uint32_t D1_COL = 0, D2_COL = BM, XI_COL = BM + 2 * BN;
constexpr uint32_t TMEM_COLS = 512;
static_assert(XI_COL + BM / 2 == TMEM_COLS, "tensor memory");
constexpr long long WAIT_LIMIT = 4000000000LL;  // ~2 s at 2 GHz
constexpr int MAX_GRID = 160;                    // CTAs a launch may have (tile ranges in the parameters)
// A block-row start costs about SEGC tiles (D1 drained, X_I reloaded into
// TMEM, the pipelines refilled): CTAs whose range crosses many short rows
// near the end of the triangle get fewer tiles.
constexpr int64_t SEGC = 2;

// Shared-memory layout for MR staged rows of X^T (the sketch width m <= MR,
// MR a multiple of 8): a ring of NA tiles of A' and a ring of NX slots of
// X^T (64 rows of X each: an X_J operand, or one of the four 64-row chunks
// of X_I on their way into TMEM), then the staging boxes.  A slot holds the
// 128 rows that the UMMA A operand (M = 128) reads; the copy fills rows
// 0..MR-1 and rows MR..127 stay zero (written once at the start), so no
// operand read reaches memory that a copy is writing.
template <int MR>
struct Lay {
    static constexpr int NA = 4;
    static constexpr int NX = 4;
    static constexpr uint32_t XB = MR * 128;                  // bytes a copy fills: MR rows x 64 bf16
    static constexpr uint32_t XS = 128 * 128;                 // slot stride: 128 rows
    static constexpr uint32_t OFF_X = NA * A_BYTES;
    static constexpr uint32_t OFF_STG = OFF_X + NX * XS;
    static constexpr uint32_t OFF_BAR = OFF_STG + NEPI * STG_BYTES;
    static constexpr uint32_t SMEM = OFF_BAR + 256;
    static_assert(MR % 8 == 0 && MR <= 128, "staged rows");
    static_assert(SMEM <= 232448, "shared memory");
    static_assert(XB % 1024 == 0 && OFF_X % 1024 == 0 && OFF_STG % 1024 == 0, "swizzle atoms");
};

struct Bars {
    uint64_t fullG[2], emptyG[2];   // the A' tiles of a group (ring slots 2 gs, 2 gs + 1)
    uint64_t fullX[4], emptyX[4];
    uint64_t d2full, d2empty;
    uint64_t d1full, d1empty;
    uint64_t xidone;     // the issuer's MMAs so far (X_I in TMEM may be overwritten) are complete
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
    long long wait_limit;   // cycles a pipeline wait may spin (opts.spin_limit; 0: WAIT_LIMIT)
    int tma_y;                  // Y reduced by TMA (aligned Y); else scalar atomics
    int64_t tstart[MAX_GRID + 1];  // CTA b owns tiles tstart[b] .. tstart[b + 1] - 1
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

// The X ring carries, in production order, the four X_I chunks of every
// block row the CTA enters, then the X_J box of every tile; each consumer
// (P2 for the chunks, P1 for the boxes) counts the items the same way.
struct XSeq {
    int64_t item = 0;
    __device__ __forceinline__ int slot(int nx) const { return (int)(item % nx); }
    __device__ __forceinline__ uint32_t phase(int nx) const { return (uint32_t)((item / nx) & 1); }
};

// Tiles are taken in groups of one or two consecutive tiles of one block row
// (two when the range's next tile is in the same row): the group's
// transposed product is one MMA chain of N = 64 per tile.  Group g holds the
// A' ring slots 2 (g % 2) and 2 (g % 2) + 1, so the two tiles of a pair sit
// one slot (32 KB, the descriptor's leading byte offset) apart.  Every role
// walks the same groups.
struct Groups {
    int64_t t, t1;
    int I, J, nbc, curI = -1;
    int sz = 1;
    bool first = false, last = false;
    __device__ Groups(int64_t a, int64_t b, int I0, int J0, int nbc_) : t(a), t1(b), I(I0), J(J0), nbc(nbc_) {}
    __device__ bool more() const { return t < t1; }
    __device__ void fill()
    {
        sz = (t + 1 < t1 && J + 1 < nbc) ? 2 : 1;
        first = (I != curI);
        last = (J + sz == nbc) || (t + sz == t1);
    }
    __device__ void next()
    {
        curI = I;
        t += sz;
        J += sz;
        if (J == nbc) {
            ++I;
            J = R * I;
        }
    }
};

template <int MR>
__global__ void __launch_bounds__(NT, 1)
sym_pass_bf16_kernel(const uint16_t *__restrict__ Ab, const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmY, const __grid_constant__ Params P)
{
    using L = Lay<MR>;
    constexpr int NX = L::NX;
    extern __shared__ __align__(1024) uint8_t sm[];
    Bars &B = *reinterpret_cast<Bars *>(sm + L::OFF_BAR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t0 = P.tstart[blockIdx.x], t1 = P.tstart[blockIdx.x + 1];
    const long long WL = P.wait_limit > 0 ? P.wait_limit : WAIT_LIMIT;
    if ((smem_u32(sm) & 1023u) != 0u) {
        if (threadIdx.x == 0) psd_set_status(P.d_status, PSDPROJ_ECUDA);
        return;
    }
    // rows MR..127 of every X slot: zero, written once (the copies fill rows
    // 0..MR-1 only); visible to the tensor core's reads through the fence below
    if constexpr (MR < 128) {
        constexpr int PADV = (128 - MR) * 128 / 16;          // 16-byte words per slot
        for (int e = threadIdx.x; e < NX * PADV; e += NT) {
            const int slot = e / PADV, w = e % PADV;
            *reinterpret_cast<uint4 *>(sm + L::OFF_X + slot * L::XS + L::XB + 16 * w) = make_uint4(0, 0, 0, 0);
        }
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&B.fullG[s], 1);
            mbar_init(&B.emptyG[s], 1);   // the MMA issuer
        }
        for (int s = 0; s < NX; ++s) {
            mbar_init(&B.fullX[s], 1);
            mbar_init(&B.emptyX[s], 1);   // the one consumer of the item
        }
        mbar_init(&B.d2full, 1);
        mbar_init(&B.d2empty, NEPI);
        mbar_init(&B.d1full, 1);
        mbar_init(&B.d1empty, NEPI);
        mbar_init(&B.xidone, 1);
        mbar_init(&B.mmadone, 1);
        B.abort = 0;
    }
    fence_proxy_async_smem();
    if (threadIdx.x == 0) {
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
            Groups gr(t0, t1, I0, J0, P.nbc);
            int64_t g = 0;          // groups whose copies were issued
            XSeq xs;                // X boxes whose copy was issued
            bool ok = true;
            auto push_x = [&](int x) -> bool {      // one 64-row box of X^T at row x
                const int sl = xs.slot(NX);
                if (!mbar_wait(&B.emptyX[sl], xs.phase(NX) ^ 1, abort, WL)) return false;
                mbar_arrive_expect_tx(&B.fullX[sl], L::XB);
                tma_load_2d(sm + L::OFF_X + sl * L::XS, &tmX, x, 0, &B.fullX[sl]);
                ++xs.item;
                return true;
            };
            for (; gr.more() && ok; gr.next()) {
                gr.fill();
                if (gr.first)
                    for (int kk = 0; kk < BM / 64 && ok; ++kk) ok = push_x(BM * gr.I + 64 * kk);
                if (!ok) break;
                const int gs = (int)(g & 1);
                if (!mbar_wait(&B.emptyG[gs], (uint32_t)((g >> 1) & 1) ^ 1, abort, WL)) { ok = false; break; }
                mbar_arrive_expect_tx(&B.fullG[gs], A_BYTES * (uint32_t)gr.sz);
                for (int u = 0; u < gr.sz; ++u)
                    bulk_load(sm + (2 * gs + u) * A_BYTES, Ab + (gr.t + u) * PSD_TILE_ELEMS, A_BYTES, &B.fullG[gs]);
                ++g;
                for (int u = 0; u < gr.sz && ok; ++u) ok = push_x(BN * (gr.J + u));
            }
            if (!ok) fail(B, P.d_status);
            // wait (bounded, also after giving up) for the copies in flight to land
            for (int64_t k = (g > 2 ? g - 2 : 0); k < g; ++k)
                mbar_wait_drain(&B.fullG[k & 1], (uint32_t)((k >> 1) & 1), WAIT_LIMIT);
            for (int64_t k = (xs.item > NX ? xs.item - NX : 0); k < xs.item; ++k)
                mbar_wait_drain(&B.fullX[k % NX], (uint32_t)((k / NX) & 1), WAIT_LIMIT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        // One issuing thread (it also owns TMEM), per group of one or two
        // tiles: the transposed product (P2, sixteen MMAs of N = 64 per tile
        // of the group, into D2), then the row products of its tiles (P1,
        // four N = 256 MMAs each, into D1); at a block-row start the four
        // chunks of X_I^T are first copied into TMEM, after the thread's own
        // earlier MMAs (readers of the previous X_I) are complete.  Every
        // tcgen05 operation is issued by this thread, in program order.
        // Descriptors: one per operand base, advanced by constants (the
        // start-address field holds addr >> 4 in its low 14 bits, and every
        // shared-memory address here is below 2^18, so adding never carries).
        if (lane == 0) {
            constexpr uint32_t id1 = idesc_bf16(128, BM, 0, 0);
            constexpr uint32_t id2a = idesc_bf16(128, BN, 0, 1);        // one tile
            constexpr uint32_t id2b = idesc_bf16(128, 2 * BN, 0, 1);    // a pair
            const uint64_t dA0 = sdesc_sw128(smem_u32(sm), 16, 1024);              // A' tile, K-major (P1)
            // A' tiles, MN-major (P2): the pair's second tile is the next
            // 64-column atom, one slot (A_BYTES) further
            const uint64_t dAmn0 = sdesc_sw128(smem_u32(sm), A_BYTES, 1024);
            const uint64_t dX0 = sdesc_sw128(smem_u32(sm + L::OFF_X), 16, 1024);   // X^T slot, K-major
            Groups gr(t0, t1, I0, J0, P.nbc);
            int64_t g = 0;
            int seg = 0;
            XSeq xs;
            bool ok = true;
            for (; gr.more(); gr.next(), ++g) {
                gr.fill();
                if (gr.first) {
                    if (seg > 0) {
                        // the previous row's MMAs read X_I in TMEM: let them complete
                        mma_commit(&B.xidone);
                        ok = mbar_wait(&B.xidone, (seg - 1) & 1, abort, WL);
                    }
                    for (int kk = 0; kk < BM / 64 && ok; ++kk) {
                        const int sl = xs.slot(NX);
                        ok = mbar_wait(&B.fullX[sl], xs.phase(NX), abort, WL);
                        if (!ok) break;
                        tc_fence_after();
                        const uint64_t xd = dX0 + (uint64_t)((sl * L::XS) >> 4);
#pragma unroll
                        for (int k2 = 0; k2 < 4; ++k2)
                            tmem_cp_128x256b(tmem + XI_COL + 8 * (4 * kk + k2), xd + 2 * k2);
                        mma_commit(&B.emptyX[sl]);
                        ++xs.item;
                    }
                    if (!ok) break;
                }
                const int gs = (int)(g & 1);
                const uint64_t goff = (uint64_t)((2 * gs * A_BYTES) >> 4);
                if (!mbar_wait(&B.fullG[gs], (uint32_t)((g >> 1) & 1), abort, WL)) { ok = false; break; }
                // P2: D2^T = X_I^T [A_IJ | A_I,J+1]   (K = 256 tile rows; X_I^T from TMEM)
                if (!mbar_wait(&B.d2empty, (uint32_t)(g & 1) ^ 1, abort, WL)) { ok = false; break; }
                tc_fence_after();
                {
                    const uint64_t bd = dAmn0 + goff;
                    const uint32_t id2 = gr.sz == 2 ? id2b : id2a;
#pragma unroll
                    for (int kk = 0; kk < BM / 16; ++kk)
                        mma_bf16_ts(tmem + D2_COL, tmem + XI_COL + 8 * kk, bd + (uint64_t)((kk * 2048) >> 4), id2,
                                    kk > 0 ? 1u : 0u);
                    mma_commit(&B.d2full);
                }
                // P1: D1^T += X_J^T A_IJ^T per tile (K = 64 tile columns); D1
                // drained by the epilogue before a block row's first group
                if (gr.first && !mbar_wait(&B.d1empty, (seg & 1) ^ 1, abort, WL)) { ok = false; break; }
                for (int u = 0; u < gr.sz; ++u) {
                    const int sl = xs.slot(NX);
                    if (!mbar_wait(&B.fullX[sl], xs.phase(NX), abort, WL)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t ad = dX0 + (uint64_t)((sl * L::XS) >> 4);
                    const uint64_t bd = dA0 + goff + (uint64_t)((u * A_BYTES) >> 4);
#pragma unroll
                    for (int kk = 0; kk < BN / 16; ++kk)
                        mma_bf16_ss(tmem + D1_COL, ad + 2 * kk, bd + 2 * kk, id1,
                                    (!gr.first || u > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&B.emptyX[sl]);
                    ++xs.item;
                }
                if (!ok) break;
                mma_commit(&B.emptyG[gs]);
                if (gr.last) {
                    mma_commit(&B.d1full);
                    ++seg;
                }
            }
            if (!ok) fail(B, P.d_status);
            // every tcgen05 operation of this CTA completes before TMEM is
            // released, also when the CTA gave up
            mma_commit(&B.mmadone);
            mbar_wait_drain(&B.mmadone, 0, WAIT_LIMIT);
        }
    } else if (warp >= 4) {
        // ------------------------------------------------------- epilogue
        // two warps per TMEM lane quarter q (a warp reads only its own
        // quarter): half h drains its half of D2 after every group (32
        // columns of a single tile, 64 of a pair) and the 32-column chunks
        // h, h + 2, ... of D1 after a block row
        const int q = warp & 3;
        const int h = (warp - 4) >> 2;
        uint8_t *stg = sm + L::OFF_STG + (warp - 4) * STG_BYTES;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        Groups gr(t0, t1, I0, J0, P.nbc);
        int64_t g = 0;
        int seg = 0;
        for (; gr.more(); gr.next(), ++g) {
            gr.fill();
            {
                // lane 0 waits (bounded); the warp leaves together
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&B.d2full, (uint32_t)(g & 1), abort, WL) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { if (lane == 0) fail(B, P.d_status); break; }
            }
            tc_fence_after();
            const int w = 32 * gr.sz;                   // D2 columns of this half
            float v0[32], v1[32];
            tmem_ld32(tmem + lane_base + D2_COL + w * h, v0);
            if (gr.sz == 2) tmem_ld32(tmem + lane_base + D2_COL + w * h + 32, v1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.d2empty);
            const int64_t r0 = (int64_t)BN * gr.J + w * h;
            flush32(P, &tmY, stg, q, lane, r0, v0);
            if (gr.sz == 2) flush32(P, &tmY, stg, q, lane, r0 + 32, v1);
            if (gr.last) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&B.d1full, seg & 1, abort, WL) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { if (lane == 0) fail(B, P.d_status); break; }
                tc_fence_after();
                const int64_t rr = (int64_t)BM * gr.I;
#pragma unroll 1
                for (int ch = h; ch < BM / 32; ch += 2) {
                    float wv[32];
                    tmem_ld32(tmem + lane_base + D1_COL + 32 * ch, wv);
                    flush32(P, &tmY, stg, q, lane, rr + 32 * ch, wv);
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
// tiles left of the diagonal block exit at once (pack_block: block bid of
// the (tile column, 64-row chunk) blocks of one image).  part 1 writes the low
// parts bf16(a - bf16(a)) instead (the split-BF16 form's second image).
__device__ __forceinline__ void pack_block(const float *__restrict__ A, int64_t n, int64_t lda,
                                           uint16_t *__restrict__ Ab, int nbc, int vec, int part, int64_t bid)
{
    constexpr int RPT = 4;                            // rows per thread
    const int J = (int)(bid % nbc);
    const int64_t chunk = bid / nbc;
    const int I = (int)((chunk * 64) / BM);
    if (J < R * I) return;                            // uniform across the block
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

__global__ void __launch_bounds__(256)
pack_upper_bf16_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                       uint16_t *__restrict__ Ab, int nbc, int vec, int part, int64_t nblocks)
{
    // grid-strided over the (tile column J, 64-row chunk) blocks
    for (int64_t bid = blockIdx.x; bid < nblocks; bid += gridDim.x) pack_block(A, n, lda, Ab, nbc, vec, part, bid);
}

// many images in one launch: block b packs block bmap[b].y of entry bmap[b].x
__global__ void __launch_bounds__(256)
pack_upper_bf16_grouped_kernel(const psd_g_pack *__restrict__ tab, const int2 *__restrict__ bmap, int part)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_pack a = tab[b.x];
    pack_block(a.A, a.n, a.lda, a.Ab, a.nbc, a.vec, part, b.y);
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

cudaError_t launch_pack_grouped(cudaStream_t s, const psd_g_pack *tab, const int2 *bmap, int nb, int part)
{
    if (nb < 1) return cudaErrorInvalidValue;
    pack_upper_bf16_grouped_kernel<<<(unsigned)nb, 256, 0, s>>>(tab, bmap, part);
    return cudaGetLastError();
}

cudaError_t launch_sym_pass_tc(cudaStream_t s, int sm_count, const uint16_t *Ab,
                               int64_t n, const float *X, int64_t ldx, int m,
                               const double *d_shift, float *Y, int64_t ldy, uint16_t *Xh,
                               int64_t ldh, int *d_status, int x_part, int accumulate, int prepared,
                               long long wait_limit)
{
    if (m < 1 || m > 128) return cudaErrorNotSupported;
    if (prepared && (x_part != 0 || accumulate != 0)) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(Ab) & 15) != 0) return cudaErrorNotSupported;
    if ((ldh % 8) != 0 || (reinterpret_cast<uintptr_t>(Xh) & 15) != 0 || ldh < n)
        return cudaErrorNotSupported;
    auto encode = get_encode();
    if (!encode) return cudaErrorNotSupported;
    // rows of X^T staged in shared memory: the sketch width rounded up
    const int mr = m <= 64 ? 64 : (m <= 112 ? 112 : 128);

    // BF16 image of X (rows n, columns m; TMA fills the rest with zeros);
    // Y starts at shift X (accumulate = 0) or gains it (accumulate = 1),
    // unless the producer of X wrote both already
    if (n > 0 && !prepared) {
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
        cuuint32_t box[2] = {64, (cuuint32_t)mr};
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
    P.wait_limit = wait_limit;
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
    int grid = sm_count > 0 ? sm_count : 148;
    if (grid > MAX_GRID) grid = MAX_GRID;
    if ((int64_t)grid > P.tiles) grid = (int)P.tiles;
    // contiguous tile ranges of equal cost(t) = t + SEGC * (block row of t):
    // CTA b starts at the smallest t with cost(t) >= total cost * b / grid
    {
        const int64_t total = P.tiles + SEGC * P.nbr;
        int b = 0, I = 0;
        P.tstart[0] = 0;
        for (int64_t t = 0; t < P.tiles && b + 1 < grid; ++t) {
            while (I + 1 < P.nbr && psd_tile_row_start(I + 1, P.nbc) <= t) ++I;
            while (b + 1 < grid && t + SEGC * I >= total * (b + 1) / grid) P.tstart[++b] = t;
        }
        while (b + 1 < grid) P.tstart[++b] = P.tiles;
        P.tstart[grid] = P.tiles;
    }
    auto go = [&](auto kern, uint32_t smem) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, NT, smem, s>>>(Ab, tmX, tmY, P);
        return cudaGetLastError();
    };
    if (mr == 64) return go(sym_pass_bf16_kernel<64>, Lay<64>::SMEM);
    if (mr == 112) return go(sym_pass_bf16_kernel<112>, Lay<112>::SMEM);
    return go(sym_pass_bf16_kernel<128>, Lay<128>::SMEM);
}
