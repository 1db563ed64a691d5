// Test matrix of the randomized range finder (Alg. 1, "Omega = randn"), its
// structured SRHT alternative, and the start vectors of power_iteration
// (Alg. 4).
//
// Element (i, c) of random stream s is keyed by the Philox4x32-10 counter
// (i, c, s, 0) with key (seed lo, seed hi) (Salmon, Moraes, Dror, Shaw, SC'11),
// and mapped to N(0,1) by the Box-Muller cosine branch on output words 0 and 1
// with u = (x + 1/2) 2^-32.  The keying makes Omega independent of the sketch
// width and of the launch shape.  The transform runs in FP32 with CUDA's logf,
// log1pf and cospif; -2 ln u is taken through log1p when u >= 1/2 so that no
// cancellation occurs.
#include <cuda_bf16.h>

#include "ctx.h"

namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                              uint32_t c3, uint32_t k0, uint32_t k1,
                                              uint32_t &o0, uint32_t &o1)
{
    // Philox round: multiply words 0 and 2 by the round multipliers, mix the
    // high halves with words 1 and 3 and the key; bump the key by the Weyl
    // increments between rounds.
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    o0 = c0;
    o1 = c1;
}

__device__ __forceinline__ float box_muller(uint32_t w0, uint32_t w1)
{
    float m2lnu;
    if (w0 >= 0x80000000u) {
        // u - 1 = -((2^32 - 1 - w0) + 1/2) 2^-32, exact enough in FP32
        const float t = -((float)(~w0) + 0.5f) * 2.3283064365386963e-10f;
        m2lnu = -2.0f * log1pf(t);
    } else {
        const float u = ((float)w0 + 0.5f) * 2.3283064365386963e-10f;
        m2lnu = -2.0f * logf(u);
    }
    const float two_u2 = ((float)w1 + 0.5f) * 4.6566128730773926e-10f;  // 2 u2
    return sqrtf(m2lnu) * cospif(two_u2);
}

__device__ __forceinline__ void gaussian_body(uint64_t seed, uint32_t stream_id, int64_t n, int m, int mpad,
                                              int64_t rows_pad, float *__restrict__ X, int64_t ldx,
                                              psd_bf16_side side, int bid, int nb)
{
    const float shift = side.d_shift ? (float)*side.d_shift : 0.0f;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
    const uint32_t k1 = (uint32_t)(seed >> 32);
    const int64_t total = rows_pad * (int64_t)mpad;
    for (int64_t idx = bid * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)nb * blockDim.x) {
        const int c = (int)(idx / rows_pad);
        const int64_t i = idx - (int64_t)c * rows_pad;
        float v = 0.0f;
        if (i < n && c < m) {
            uint32_t w0, w1;
            philox4x32_10((uint32_t)i, (uint32_t)c, stream_id, 0u, k0, k1, w0, w1);
            v = box_muller(w0, w1);
            if (side.Xh) side.Xh[(int64_t)c * side.ldh + i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
            if (side.Y) side.Y[(int64_t)c * side.ldy + i] = shift * v;
        }
        X[(int64_t)c * ldx + i] = v;
    }
}

__global__ void gaussian_kernel(uint64_t seed, uint32_t stream_id, int64_t n, int m,
                                int mpad, int64_t rows_pad, float *__restrict__ X,
                                int64_t ldx, psd_bf16_side side)
{
    gaussian_body(seed, stream_id, n, m, mpad, rows_pad, X, ldx, side, blockIdx.x, gridDim.x);
}

// many test matrices in one launch: block b runs block bmap[b].y of entry
// bmap[b].x's nb (each entry as its own launch_gaussian)
__global__ void __launch_bounds__(256)
gaussian_grouped_kernel(const psd_g_gauss *__restrict__ tab, const int2 *__restrict__ bmap, uint32_t stream_id)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_gauss a = tab[b.x];
    gaussian_body(a.seed, stream_id, a.n, a.m, a.mpad, a.rows_pad, a.X, a.ldx, a.side, b.y, a.nb);
}

// The starts of many power iterations (as launch_gaussian of the start
// vector v0 with n rows and one column, then launch_pi_init): block b runs
// block bmap[b].y of entry bmap[b].x's nb
__global__ void __launch_bounds__(256)
pi_start_grouped_kernel(const psd_g_pi *__restrict__ tab, const int2 *__restrict__ bmap, uint32_t stream_id)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_pi a = tab[b.x];
    const psd_bf16_side none = {nullptr, 0, nullptr, 0, nullptr};
    gaussian_body(a.seed, stream_id, a.n, 1, 1, a.n, a.v0, a.n, none, b.y, a.nb);
    if (b.y == 0 && threadIdx.x == 0) {
        a.scal[0] = 1.0;
        a.scal[1] = 0.0;
    }
    for (int64_t i = b.y * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)a.nb * blockDim.x)
        a.v1[i] = 0.0f;
}

// SRHT test matrix (the real counterpart of the subsampled randomized
// Fourier transform named in the footnote to Alg. 1): with N the power of two
// >= n, Omega = D H_N S restricted to rows 0..n-1, i.e.
//   Omega[i, c] = d_i (-1)^popcount(i & s_c),
// D = diag(d) random signs, H_N the Sylvester-Hadamard matrix (entries +-1),
// S the columns s_0..s_{m-1} of H_N drawn without replacement.
//   d_i = -1 when bit 0 of word 0 of Philox(i, 0, PSD_SRHT_SIGNS, 0) is 1;
//   s_c = the first draw (word 0 of Philox(c, t, PSD_SRHT_PICKS, 0)) mod N,
//         t = 0, 1, ..., not already taken by a column before c.
// The picks run in one thread (m <= 256 draws, each checked against the
// earlier ones); an exhausted bound on t sets PSDPROJ_ETIMEOUT.
__global__ void srht_pick_kernel(uint64_t seed, int m, uint32_t nmask, int *__restrict__ picks,
                                 int *d_status)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int c = 0; c < m; ++c) {
        int got = -1;
        for (uint32_t t = 0; t < (1u << 20) && got < 0; ++t) {
            uint32_t w0, w1;
            philox4x32_10((uint32_t)c, t, PSD_SRHT_PICKS, 0u, k0, k1, w0, w1);
            const int x = (int)(w0 & nmask);
            bool dup = false;
            for (int j = 0; j < c && !dup; ++j) dup = picks[j] == x;
            if (!dup) got = x;
        }
        if (got < 0) {
            psd_set_status(d_status, PSDPROJ_ETIMEOUT);
            got = 0;
        }
        picks[c] = got;
    }
}

__global__ void srht_fill_kernel(uint64_t seed, int64_t n, int m, int mpad, int64_t rows_pad,
                                 const int *__restrict__ picks, float *__restrict__ X, int64_t ldx)
{
    __shared__ int sp[PSD_MAX_M];
    for (int c = threadIdx.x; c < m; c += blockDim.x) sp[c] = picks[c];
    __syncthreads();
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    const int64_t total = rows_pad * (int64_t)mpad;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / rows_pad);
        const int64_t i = idx - (int64_t)c * rows_pad;
        float v = 0.0f;
        if (i < n && c < m) {
            uint32_t w0, w1;
            philox4x32_10((uint32_t)i, 0u, PSD_SRHT_SIGNS, 0u, k0, k1, w0, w1);
            const int par = (__popc((uint32_t)i & (uint32_t)sp[c]) + (int)(w0 & 1u)) & 1;
            v = par ? -1.0f : 1.0f;
        }
        X[(int64_t)c * ldx + i] = v;
    }
}

}  // namespace

cudaError_t launch_srht(cudaStream_t s, uint64_t seed, int64_t n, int m, int mpad, int64_t rows_pad,
                        int *picks, int *d_status, float *X, int64_t ldx)
{
    if (m < 1 || m > PSD_MAX_M || n < m || n > (int64_t)1 << 30) return cudaErrorInvalidValue;
    uint32_t N = 1;
    while ((int64_t)N < n) N <<= 1;
    srht_pick_kernel<<<1, 32, 0, s>>>(seed, m, N - 1, picks, d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = rows_pad * (int64_t)mpad;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    srht_fill_kernel<<<blocks, 256, 0, s>>>(seed, n, m, mpad, rows_pad, picks, X, ldx);
    return cudaGetLastError();
}

// Writes rows [0, rows_pad) x columns [0, mpad); entries with i >= n or
// c >= m are zero (padding of context-owned buffers).
cudaError_t launch_gaussian_grouped(cudaStream_t s, const psd_g_gauss *tab, const int2 *bmap, int nb,
                                    uint32_t stream_id)
{
    if (nb < 1) return cudaErrorInvalidValue;
    gaussian_grouped_kernel<<<(unsigned)nb, 256, 0, s>>>(tab, bmap, stream_id);
    return cudaGetLastError();
}

cudaError_t launch_pi_start_grouped(cudaStream_t s, const psd_g_pi *tab, const int2 *bmap, int nb,
                                   uint32_t stream_id)
{
    if (nb < 1) return cudaErrorInvalidValue;
    pi_start_grouped_kernel<<<(unsigned)nb, 256, 0, s>>>(tab, bmap, stream_id);
    return cudaGetLastError();
}

cudaError_t launch_gaussian(cudaStream_t s, uint64_t seed, uint32_t stream_id, int64_t n,
                            int m, int mpad, int64_t rows_pad, float *X, int64_t ldx,
                            const psd_bf16_side *side)
{
    const psd_bf16_side none = {nullptr, 0, nullptr, 0, nullptr};
    const int64_t total = rows_pad * (int64_t)mpad;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    gaussian_kernel<<<blocks, 256, 0, s>>>(seed, stream_id, n, m, mpad, rows_pad, X, ldx, side ? *side : none);
    return cudaGetLastError();
}
