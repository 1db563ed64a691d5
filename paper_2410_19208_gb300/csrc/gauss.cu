// Test matrix of the randomized range finder (Alg. 1, "Omega = randn") and the
// start vectors of power_iteration (Alg. 4).
//
// Element (i, c) of random stream s is keyed by the Philox4x32-10 counter
// (i, c, s, 0) with key (seed lo, seed hi) (Salmon, Moraes, Dror, Shaw, SC'11),
// and mapped to N(0,1) by the Box-Muller cosine branch on output words 0 and 1
// with u = (x + 1/2) 2^-32.  The keying makes Omega independent of the sketch
// width and of the launch shape.  The transform runs in FP32 with CUDA's logf,
// log1pf and cospif; -2 ln u is taken through log1p when u >= 1/2 so that no
// cancellation occurs.
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

__global__ void gaussian_kernel(uint64_t seed, uint32_t stream_id, int64_t n, int m,
                                int mpad, int64_t rows_pad, float *__restrict__ X,
                                int64_t ldx)
{
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu);
    const uint32_t k1 = (uint32_t)(seed >> 32);
    const int64_t total = rows_pad * (int64_t)mpad;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / rows_pad);
        const int64_t i = idx - (int64_t)c * rows_pad;
        float v = 0.0f;
        if (i < n && c < m) {
            uint32_t w0, w1;
            philox4x32_10((uint32_t)i, (uint32_t)c, stream_id, 0u, k0, k1, w0, w1);
            v = box_muller(w0, w1);
        }
        X[(int64_t)c * ldx + i] = v;
    }
}

}  // namespace

// Writes rows [0, rows_pad) x columns [0, mpad); entries with i >= n or
// c >= m are zero (padding of context-owned buffers).
cudaError_t launch_gaussian(cudaStream_t s, uint64_t seed, uint32_t stream_id, int64_t n,
                            int m, int mpad, int64_t rows_pad, float *X, int64_t ldx)
{
    const int64_t total = rows_pad * (int64_t)mpad;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    gaussian_kernel<<<blocks, 256, 0, s>>>(seed, stream_id, n, m, mpad, rows_pad, X, ldx);
    return cudaGetLastError();
}
