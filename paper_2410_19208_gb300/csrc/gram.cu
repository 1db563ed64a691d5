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

}  // namespace

// symmetrize: 0 = G = X^T Z as is; 1 = X == Z (upper computed, mirrored);
// 2 = (X^T Z + Z^T X)/2.
cudaError_t launch_gram(cudaStream_t s, const float *X, int64_t ldx, const float *Z,
                        int64_t ldz, int64_t n, int m, float *gpart, double *G, int symmetrize, float *Gdf)
{
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
