// Gram products of the small-matrix steps:
//   G = Y^T Y           (CholeskyQR2, the QR 'econ' of Alg. 1)
//   C = (Q^T Z + Z^T Q)/2 with Z = A Q  (the projected core Q^T A Q of Alg. 2)
// Each thread block forms the FP32 partial product of one chunk of 64 rows
// (register micro-tiles); a second kernel sums the chunk partials in FP64 in
// a fixed order (deterministic, no atomics).
#include "ctx.h"

namespace {

constexpr int CH = 64;    // rows per chunk (PSD_GRAM_CHUNK)
constexpr int RS = 32;    // rows staged in shared memory at a time
constexpr int NT = 256;

__global__ void __launch_bounds__(NT)
gram_partial_kernel(const float *__restrict__ X, int64_t ldx, const float *__restrict__ Z,
                    int64_t ldz, int64_t n, int m, int mp, int upper_only,
                    float *__restrict__ gpart)
{
    extern __shared__ float sm[];
    float *Xs = sm;              // RS x mp
    float *Zs = sm + RS * mp;    // RS x mp
    const int64_t row0 = (int64_t)blockIdx.x * CH;
    const int nbt = mp / 8;      // micro-tiles per side
    const int ntiles = upper_only ? nbt * (nbt + 1) / 2 : nbt * nbt;
    float *out = gpart + (int64_t)blockIdx.x * mp * mp;
    const bool same = (X == Z) && (ldx == ldz);

    for (int pass = 0; pass * NT < ntiles; ++pass) {
        const int tile = pass * NT + threadIdx.x;
        int bi = 0, bj = 0;
        const bool active = tile < ntiles;
        if (active) {
            if (upper_only) {
                // tile -> (bi <= bj), row-major over the upper triangle
                int t = tile;
                bi = 0;
                while (t >= nbt - bi) { t -= nbt - bi; ++bi; }
                bj = bi + t;
            } else {
                bi = tile / nbt;
                bj = tile % nbt;
            }
        }
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
        for (int rs = 0; rs < CH; rs += RS) {
            __syncthreads();
            for (int e = threadIdx.x; e < RS * mp; e += NT) {
                const int a = e / RS, k = e % RS;
                const int64_t r = row0 + rs + k;
                const bool ok = r < n && a < m;
                Xs[k * mp + a] = ok ? X[(int64_t)a * ldx + r] : 0.0f;
                if (!same) Zs[k * mp + a] = ok ? Z[(int64_t)a * ldz + r] : 0.0f;
            }
            __syncthreads();
            const float *Zsrc = same ? Xs : Zs;
            if (active) {
#pragma unroll 2
                for (int k = 0; k < RS; ++k) {
                    float x[8], z[8];
                    const float4 *xp = reinterpret_cast<const float4 *>(Xs + k * mp + 8 * bi);
                    const float4 *zp = reinterpret_cast<const float4 *>(Zsrc + k * mp + 8 * bj);
                    float4 x0 = xp[0], x1 = xp[1], z0 = zp[0], z1 = zp[1];
                    x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w;
                    x[4] = x1.x; x[5] = x1.y; x[6] = x1.z; x[7] = x1.w;
                    z[0] = z0.x; z[1] = z0.y; z[2] = z0.z; z[3] = z0.w;
                    z[4] = z1.x; z[5] = z1.y; z[6] = z1.z; z[7] = z1.w;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(x[i], z[j], acc[i][j]);
                }
            }
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) out[(8 * bi + i) * mp + 8 * bj + j] = acc[i][j];
        }
    }
}

// The same partial products for m <= 128 with every thread busy: a 16 x 16
// thread grid covers the whole mp x mp square (thread (tx, ty) owns rows
// ty T .. ty T + T-1 and columns tx T .. tx T + T-1, T = ceil(mp / 16), so
// 16 T >= m), reading the staged rows with stride T (conflict-free for odd
// T).  Symmetric products are formed in full; the reduction reads the half
// it needs.
template <int T>
__global__ void __launch_bounds__(NT)
gram_partial_sq_kernel(const float *__restrict__ X, int64_t ldx, const float *__restrict__ Z,
                       int64_t ldz, int64_t n, int m, int mp, float *__restrict__ gpart)
{
    constexpr int S = 16 * T;
    __shared__ float Xs[RS][S + 1];
    __shared__ float Zs[RS][S + 1];
    const int64_t row0 = (int64_t)blockIdx.x * CH;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const bool same = (X == Z) && (ldx == ldz);
    float acc[T][T];
#pragma unroll
    for (int u = 0; u < T; ++u)
#pragma unroll
        for (int v = 0; v < T; ++v) acc[u][v] = 0.0f;
    // the next RS rows are read into registers while the current ones are
    // multiplied (fixed trip counts, so a thread's loads are in flight together)
    constexpr int NE = RS * S / NT;
    static_assert(RS * S % NT == 0, "staging split");
    float rx[NE], rz[NE];
    auto fetch = [&](int rs) {
#pragma unroll
        for (int i = 0; i < NE; ++i) {
            const int e = i * NT + threadIdx.x;
            const int a = e / RS, k = e % RS;
            const int64_t r = row0 + rs + k;
            const bool ok = r < n && a < m;
            rx[i] = ok ? X[(int64_t)a * ldx + r] : 0.0f;
            if (!same) rz[i] = ok ? Z[(int64_t)a * ldz + r] : 0.0f;
        }
    };
    fetch(0);
    for (int rs = 0; rs < CH; rs += RS) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NE; ++i) {
            const int e = i * NT + threadIdx.x;
            Xs[e % RS][e / RS] = rx[i];
            if (!same) Zs[e % RS][e / RS] = rz[i];
        }
        __syncthreads();
        if (rs + RS < CH) fetch(rs + RS);
        const float (*Zsrc)[S + 1] = same ? Xs : Zs;
#pragma unroll 4
        for (int k = 0; k < RS; ++k) {
            float x[T], z[T];
#pragma unroll
            for (int u = 0; u < T; ++u) {
                x[u] = Xs[k][ty * T + u];
                z[u] = Zsrc[k][tx * T + u];
            }
#pragma unroll
            for (int u = 0; u < T; ++u)
#pragma unroll
                for (int v = 0; v < T; ++v) acc[u][v] = fmaf(x[u], z[v], acc[u][v]);
        }
    }
    float *out = gpart + (int64_t)blockIdx.x * mp * mp;
#pragma unroll
    for (int u = 0; u < T; ++u) {
        const int a = ty * T + u;
#pragma unroll
        for (int v = 0; v < T; ++v) {
            const int b = tx * T + v;
            if (a < m && b < m) out[a * mp + b] = acc[u][v];
        }
    }
}

// Sum of two unevaluated FP32 pairs hi + lo (Knuth's two-sum on the high
// parts, about 48 significant bits): the chunk sums below in FP32
// arithmetic, off the FP64 pipe (a few operations per SM and clock here).
struct fsum {
    float hi, lo;
};
__device__ __forceinline__ fsum fsum_add(fsum a, fsum b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float lo = ((a.hi - (s - bb)) + (b.hi - bb)) + a.lo + b.lo;
    const float h = s + lo;
    return {h, lo - (h - s)};
}

// G[a + b*m] = sum over chunks of gpart (double-float, then FP64); mode 0:
// full product, mode 1: upper-only symmetric Gram (mirror), mode 2:
// symmetrise (S+S^T)/2.  Eight lanes share one entry of the partials
// (coalesced over the entry index) and split the chunk sum in a fixed order.
__global__ void gram_reduce_kernel(const float *__restrict__ gpart, int nchunk, int m, int mp,
                                   int mode, double *__restrict__ G, float2 *__restrict__ Gdf)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int f = (int)(tid >> 3), sub = (int)(tid & 7);
    const bool act = f < mp * mp;
    const int ia = act ? f / mp : 0, ib = act ? f - (f / mp) * mp : 0;
    fsum acc = {0.0f, 0.0f};
    if (act && ia < m && ib < m && (mode != 1 || ia <= ib)) {
#pragma unroll 4
        for (int c = sub; c < nchunk; c += 8) acc = fsum_add(acc, {gpart[(int64_t)c * mp * mp + f], 0.0f});
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
        acc = fsum_add(acc, {__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)});
    const double s = (double)acc.hi + (double)acc.lo;
    if (!act || sub != 0 || ia >= m || ib >= m) return;
    if (mode == 0) {
        G[(int64_t)ib * m + ia] = s;
        if (Gdf) Gdf[(int64_t)ib * m + ia] = make_float2(acc.hi, acc.lo);
    } else if (mode == 1) {
        if (ia <= ib) {
            G[(int64_t)ib * m + ia] = s;
            G[(int64_t)ia * m + ib] = s;
            if (Gdf) {
                Gdf[(int64_t)ib * m + ia] = make_float2(acc.hi, acc.lo);
                Gdf[(int64_t)ia * m + ib] = make_float2(acc.hi, acc.lo);
            }
        }
    } else {
        // (S + S^T)/2: entry (ia, ib) contributes half to both positions
        atomicAdd(&G[(int64_t)ib * m + ia], 0.5 * s);
        atomicAdd(&G[(int64_t)ia * m + ib], 0.5 * s);
    }
}

// The symmetric products for m <= 128 (G = X^T X, or S = (X^T Z + Z^T X)/2)
// on the upper triangle only: 2 blocks per SM, block b owning rows
// [b R, (b + 1) R) (R = rows, a multiple of 8), staged SR rows at a time;
// thread t owns the t-th 8 x 8 tile (bi <= bj) of the upper triangle (64
// FMAs per four 16-byte shared loads; twice that for the two-sided form)
// and writes one FP32 partial per block, tile-major.
constexpr int SR = 64;            // rows staged at a time
constexpr int NTU = 160;          // >= tiles of the upper triangle for m <= 128 (136)

template <bool TWO>
__device__ __forceinline__ void gram_upper_body(const float *__restrict__ X, int64_t ldx,
                                                const float *__restrict__ Z, int64_t ldz, int64_t n, int m,
                                                int mp, int rows, float *__restrict__ gpart, int bid)
{
    extern __shared__ __align__(16) float sgu[];
    const int ld = mp + 4;
    float *Xs = sgu;                       // SR x ld
    float *Zs = sgu + SR * ld;             // (two-sided form)
    const int tid = threadIdx.x;
    const int nt8 = mp / 8, ntiles = nt8 * (nt8 + 1) / 2;
    int bi = 0, bj = 0;
    {
        int t = tid < ntiles ? tid : 0;
        while (t >= nt8 - bi) {
            t -= nt8 - bi;
            ++bi;
        }
        bj = bi + t;
    }
    const bool act = tid < ntiles;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    const int64_t rbeg = (int64_t)bid * rows;
    const int64_t rend = min(rbeg + rows, n);
    for (int64_t r0 = rbeg; r0 < rend; r0 += SR) {
        const int nr = (int)min((int64_t)SR, rend - r0);
        __syncthreads();
        // stage rows r0 .. r0 + nr - 1: element e = (column e / SR, row e % SR),
        // consecutive threads on consecutive rows (coalesced), a batch of
        // loads in flight per thread before their stores
        constexpr int BT = TWO ? 8 : 16;
        for (int base = 0; base < mp * SR; base += NTU * BT) {
            float vx[BT], vz[BT];
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                const int e = base + tid + NTU * u;
                const int c = e / SR, r = e % SR;
                const bool ok = e < mp * SR && r < nr && c < m;
                vx[u] = ok ? X[(int64_t)c * ldx + r0 + r] : 0.0f;
                if (TWO) vz[u] = ok ? Z[(int64_t)c * ldz + r0 + r] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < BT; ++u) {
                const int e = base + tid + NTU * u;
                if (e < mp * SR) {
                    Xs[(e % SR) * ld + e / SR] = vx[u];
                    if (TWO) Zs[(e % SR) * ld + e / SR] = vz[u];
                }
            }
        }
        __syncthreads();
        if (act) {
#pragma unroll 2
            for (int r = 0; r < nr; ++r) {
                const float4 *xi = reinterpret_cast<const float4 *>(Xs + r * ld + 8 * bi);
                const float4 *xj = reinterpret_cast<const float4 *>(Xs + r * ld + 8 * bj);
                const float4 a0 = xi[0], a1 = xi[1], b0 = xj[0], b1 = xj[1];
                const float x[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float y[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                if (TWO) {
                    const float4 *zi = reinterpret_cast<const float4 *>(Zs + r * ld + 8 * bi);
                    const float4 *zj = reinterpret_cast<const float4 *>(Zs + r * ld + 8 * bj);
                    const float4 c0 = zi[0], c1 = zi[1], d0 = zj[0], d1 = zj[1];
                    const float zi8[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
                    const float zj8[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(x[i], zj8[j], fmaf(zi8[i], y[j], acc[i][j]));
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(x[i], y[j], acc[i][j]);
                }
            }
        }
    }
    if (act) {
        float *out = gpart + ((int64_t)bid * ntiles + tid) * 64;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            reinterpret_cast<float4 *>(out + 8 * i)[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            reinterpret_cast<float4 *>(out + 8 * i)[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
        }
    }
}

template <bool TWO>
__global__ void __launch_bounds__(NTU)
gram_upper_kernel(const float *__restrict__ X, int64_t ldx, const float *__restrict__ Z, int64_t ldz, int64_t n,
                  int m, int mp, int rows, float *__restrict__ gpart)
{
    gram_upper_body<TWO>(X, ldx, Z, ldz, n, m, mp, rows, gpart, blockIdx.x);
}

// many problems in one launch: block b runs block bmap[b].y of entry bmap[b].x
// (two blocks per SM: each block's rows are few when the problems are small)
template <bool TWO>
__global__ void __launch_bounds__(NTU, 2)
gram_upper_grouped_kernel(const psd_g_gram *__restrict__ tab, const int2 *__restrict__ bmap)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_gram a = tab[b.x];
    gram_upper_body<TWO>(a.X, a.ldx, TWO ? a.Z : a.X, TWO ? a.ldz : a.ldx, a.n, a.m, a.mp, a.rows, a.gpart, b.y);
}

// G from the per-block partials of gram_upper_kernel: a block takes 32
// consecutive positions q of the tile-major partial (lane = position, so the
// loads are coalesced) and its 8 warps split the block partials (warp g:
// partials g, g + 8, ...), each summing in double-float; the 8 sums are
// added in a fixed order (deterministic).  Both (a, b) and (b, a) are
// written (scale: 1 for X^T X, 1/2 for the two-sided form).
// position q of the tile-major partials (tile q / 64, entry (i, j) of its
// 8 x 8 block) stored as entries (a, b) and (b, a) of G (and Gdf), scaled
__device__ __forceinline__ void gram_reduce_store(fsum acc, int q, int nt8, int m, float scale,
                                                  double *__restrict__ G, float2 *__restrict__ Gdf)
{
    const int t = q >> 6, ij = q & 63, i = ij >> 3, j = ij & 7;
    int bi = 0, tt = t;
    while (tt >= nt8 - bi) {
        tt -= nt8 - bi;
        ++bi;
    }
    const int bj = bi + tt;
    const int ia = 8 * bi + i, ib = 8 * bj + j;
    if (ia >= m || ib >= m || (bi == bj && i > j)) return;
    acc.hi *= scale;          // exact: scale is a power of two
    acc.lo *= scale;
    const double sv = (double)acc.hi + (double)acc.lo;
    G[(int64_t)ib * m + ia] = sv;
    G[(int64_t)ia * m + ib] = sv;
    if (Gdf) {
        Gdf[(int64_t)ib * m + ia] = make_float2(acc.hi, acc.lo);
        Gdf[(int64_t)ia * m + ib] = make_float2(acc.hi, acc.lo);
    }
}

__device__ __forceinline__ void gram_upper_reduce_body(const float *__restrict__ gpart, int nblk, int m, int mp,
                                                       float scale, double *__restrict__ G,
                                                       float2 *__restrict__ Gdf, int bid)
{
    __shared__ fsum part[8][32];
    const int nt8 = mp / 8, ntiles = nt8 * (nt8 + 1) / 2;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int q = bid * 32 + lane;
    const bool inr = q < ntiles * 64;
    fsum acc = {0.0f, 0.0f};
    if (inr) {
#pragma unroll 4
        for (int b = g; b < nblk; b += 8) acc = fsum_add(acc, {gpart[(int64_t)b * ntiles * 64 + q], 0.0f});
    }
    part[g][lane] = acc;
    __syncthreads();
    if (g != 0 || !inr) return;
#pragma unroll
    for (int w = 1; w < 8; ++w) acc = fsum_add(acc, part[w][lane]);
    gram_reduce_store(acc, q, nt8, m, scale, G, Gdf);
}

// The same sums with a thread per position (256 per block), each adding its
// position's partials in order: a problem of a grouped batch with at most
// PSD_GRAM_RED_SEQ partials would leave most warps of the form above idle
// in its many blocks
__device__ __forceinline__ void gram_upper_reduce_seq_body(const float *__restrict__ gpart, int nblk, int m, int mp,
                                                           float scale, double *__restrict__ G,
                                                           float2 *__restrict__ Gdf, int bid)
{
    const int nt8 = mp / 8, ntiles = nt8 * (nt8 + 1) / 2;
    const int q = bid * 256 + threadIdx.x;
    if (q >= ntiles * 64) return;
    fsum acc = {0.0f, 0.0f};
#pragma unroll 4
    for (int b = 0; b < nblk; ++b) acc = fsum_add(acc, {gpart[(int64_t)b * ntiles * 64 + q], 0.0f});
    gram_reduce_store(acc, q, nt8, m, scale, G, Gdf);
}

__global__ void __launch_bounds__(256)
gram_upper_reduce_kernel(const float *__restrict__ gpart, int nblk, int m, int mp, float scale,
                         double *__restrict__ G, float2 *__restrict__ Gdf)
{
    gram_upper_reduce_body(gpart, nblk, m, mp, scale, G, Gdf, blockIdx.x);
}

__global__ void __launch_bounds__(256)
gram_upper_reduce_grouped_kernel(const psd_g_gram *__restrict__ tab, const int2 *__restrict__ bmap, float scale)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_gram a = tab[b.x];
    if (a.nblk <= PSD_GRAM_RED_SEQ)          // uniform across the block
        gram_upper_reduce_seq_body(a.gpart, a.nblk, a.m, a.mp, scale, a.G, a.Gdf, b.y);
    else
        gram_upper_reduce_body(a.gpart, a.nblk, a.m, a.mp, scale, a.G, a.Gdf, b.y);
}

}  // namespace

// symmetrize: 0 = G = X^T Z as is; 1 = X == Z (upper computed, mirrored);
// 2 = (X^T Z + Z^T X)/2.
cudaError_t launch_gram(cudaStream_t s, const float *X, int64_t ldx, const float *Z,
                        int64_t ldz, int64_t n, int m, float *gpart, double *G, int symmetrize, float *Gdf,
                        int sm_count)
{
    if (Gdf && symmetrize == 0) return cudaErrorInvalidValue;
    if (symmetrize != 0 && m <= 128 && n > 0) {
        // rows per block: at least PSD_GRAM_CHUNK (so that the blocks' partials
        // fit the workspace sized for ceil(n / PSD_GRAM_CHUNK) chunks of mp^2),
        // about two blocks per SM
        const int mp = (int)psd_round_up(m, 8);
        const int64_t rows = psd_gram_rows(n, sm_count);
        const int nblk = psd_gram_blocks(n, sm_count);
        const bool two = symmetrize == 2;
        const size_t smem = sizeof(float) * (size_t)SR * (mp + 4) * (two ? 2 : 1);
        if (two) {
            // the attribute is process-wide: the largest size (m = 128)
            cudaError_t ea = cudaFuncSetAttribute(gram_upper_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)(sizeof(float) * SR * (128 + 4) * 2));
            if (ea != cudaSuccess) return ea;
        }
        if (two)
            gram_upper_kernel<true><<<nblk, NTU, smem, s>>>(X, ldx, Z, ldz, n, m, mp, (int)rows, gpart);
        else
            gram_upper_kernel<false><<<nblk, NTU, smem, s>>>(X, ldx, X, ldx, n, m, mp, (int)rows, gpart);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        gram_upper_reduce_kernel<<<(unsigned)psd_gram_reduce_blocks(m), 256, 0, s>>>(
            gpart, nblk, m, mp, two ? 0.5f : 1.0f, G, reinterpret_cast<float2 *>(Gdf));
        return cudaGetLastError();
    }
    if (Gdf && symmetrize == 2) return cudaErrorInvalidValue;
    const int mp = (int)psd_round_up(m, 8);
    const int nchunk = (int)((n + CH - 1) / CH);
    const size_t smem = sizeof(float) * 2 * RS * (size_t)mp;
    cudaError_t e = cudaSuccess;
    const int T = (mp + 15) / 16;
    switch (T) {
    case 1: gram_partial_sq_kernel<1><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    case 2: gram_partial_sq_kernel<2><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    case 3: gram_partial_sq_kernel<3><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    case 4: gram_partial_sq_kernel<4><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    case 5: gram_partial_sq_kernel<5><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    case 6: gram_partial_sq_kernel<6><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    case 7: gram_partial_sq_kernel<7><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    case 8: gram_partial_sq_kernel<8><<<nchunk, NT, 0, s>>>(X, ldx, Z, ldz, n, m, mp, gpart); break;
    default:
        // process-wide attribute: the largest size (m = PSD_MAX_M)
        e = cudaFuncSetAttribute(gram_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * 2 * RS * (size_t)psd_round_up(PSD_MAX_M, 8)));
        if (e != cudaSuccess) return e;
        gram_partial_kernel<<<nchunk, NT, smem, s>>>(X, ldx, Z, ldz, n, m, mp, symmetrize == 1,
                                                     gpart);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (symmetrize == 2) {
        e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)m * m, s);
        if (e != cudaSuccess) return e;
    }
    const int64_t threads = (int64_t)mp * mp * 8;
    gram_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(gpart, nchunk, m, mp, symmetrize, G,
                                                                          reinterpret_cast<float2 *>(Gdf));
    return cudaGetLastError();
}

cudaError_t launch_gram_grouped(cudaStream_t s, const psd_g_gram *tab, int two, const int2 *bmap, int nb,
                                const int2 *bmap_red, int nb_red, int mp_max)
{
    if (nb < 1 || nb_red < 1 || mp_max < 8 || mp_max > 128) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (size_t)SR * (mp_max + 4) * (two ? 2 : 1);
    // process-wide attributes: the largest size (m = 128)
    const int smax = (int)(sizeof(float) * SR * (128 + 4) * (two ? 2 : 1));
    cudaError_t e = two ? cudaFuncSetAttribute(gram_upper_grouped_kernel<true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smax)
                        : cudaFuncSetAttribute(gram_upper_grouped_kernel<false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (e != cudaSuccess) return e;
    if (two)
        gram_upper_grouped_kernel<true><<<(unsigned)nb, NTU, smem, s>>>(tab, bmap);
    else
        gram_upper_grouped_kernel<false><<<(unsigned)nb, NTU, smem, s>>>(tab, bmap);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gram_upper_reduce_grouped_kernel<<<(unsigned)nb_red, 256, 0, s>>>(tab, bmap_red, two ? 0.5f : 1.0f);
    return cudaGetLastError();
}
