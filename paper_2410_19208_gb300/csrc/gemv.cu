// power_iteration (Alg. 4) and min_eig (Alg. 5) on the device.
//
// One launch per product w = (A + shift I) (s * v): A is streamed once, upper
// triangle only, in 32 x 128 tiles.  A thread block owns a segment of one
// block row: the row sums accumulate in registers, the transposed
// contributions of each tile are summed over the block's 8 warps and added
// with atomics.  The last block to finish (atomic ticket) forms ||w|| in
// FP64, stores the scale 1/||w|| that the next product applies on load,
// clears the other vector for the next product, and resets the ticket.
// sigma = ||A v|| after the N normalised steps is written to *d_sigma.
#include "ctx.h"

namespace {

constexpr int TRW = 32;    // rows per tile
constexpr int TCW = 128;   // columns per tile
constexpr int SEGW = 8;    // tiles per block
constexpr int NTW = 256;

// scal[0]: scale of the input vector; scal[1]: norm of the last output;
// scal[2]: the shift applied (A + shift I).
__global__ void __launch_bounds__(NTW)
sym_gemv_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                const float *__restrict__ x, float *__restrict__ y, float *__restrict__ other,
                double *scal, unsigned *counter, const double *d_shift_neg, double *d_sigma,
                int nb, int vec)
{
    __shared__ float colsum[8][TCW];
    __shared__ double red[NTW / 32];
    __shared__ bool s_last;
    int64_t idx = blockIdx.x;
    int I = 0;
    for (; I < nb; ++I) {
        const int64_t row0 = (int64_t)I * TRW;
        const int tiles = (int)((n - row0 + TCW - 1) / TCW);
        const int cnt = (tiles + SEGW - 1) / SEGW;
        if (idx < cnt) break;
        idx -= cnt;
    }
    const int64_t row0 = (int64_t)I * TRW;
    const int tiles = (int)((n - row0 + TCW - 1) / TCW);
    const int t0 = (int)idx * SEGW, t1 = min(tiles, t0 + SEGW);
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
    for (int t = t0; t < t1; ++t) {
        const int64_t c0 = row0 + (int64_t)t * TCW + lane * 4;
        float xc[4];
        float colacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 4; ++j) xc[j] = (c0 + j < n) ? x[c0 + j] * sc : 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t gr = row0 + warp * 4 + i;
            if (gr >= n) continue;
            float a[4];
            if (vec && c0 + 3 < n && c0 >= gr) {
                const float4 v4 = *reinterpret_cast<const float4 *>(A + gr * lda + c0);
                a[0] = v4.x; a[1] = v4.y; a[2] = v4.z; a[3] = v4.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    a[j] = (c0 + j < n && c0 + j >= gr) ? A[gr * lda + c0 + j] : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                rowacc[i] = fmaf(a[j], xc[j], rowacc[i]);
                if (c0 + j > gr) colacc[j] = fmaf(a[j], xr[i], colacc[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) colsum[warp][lane * 4 + j] = colacc[j];
        __syncthreads();
        if (threadIdx.x < TCW) {
            float s = 0.0f;
#pragma unroll
            for (int w = 0; w < 8; ++w) s += colsum[w][threadIdx.x];
            const int64_t gc = row0 + (int64_t)t * TCW + threadIdx.x;
            if (gc < n && s != 0.0f) atomicAdd(&y[gc], s);
        }
        __syncthreads();
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

    // ticket: the last block finishes the product
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NTW) {
        const double v = (double)__ldcg(&y[i]);
        acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NTW / 32; ++w) s += red[w];
        const double nrm = sqrt(s);
        scal[1] = nrm;
        scal[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
        if (d_sigma) *d_sigma = nrm;
        *counter = 0u;
    }
    for (int64_t i = threadIdx.x; i < n; i += NTW) other[i] = 0.0f;
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

}  // namespace

cudaError_t launch_power_iteration(cudaStream_t s, const float *A, int64_t n, int64_t lda, int N,
                                   uint64_t seed, uint32_t stream_id, const double *d_shift_neg,
                                   float *v0, float *v1, double *scal, unsigned *counter,
                                   double *d_sigma)
{
    cudaError_t e = launch_gaussian(s, seed, stream_id, n, 1, 1, n, v0, n);
    if (e != cudaSuccess) return e;
    pi_init_kernel<<<64, 256, 0, s>>>(scal, v1, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = (int)((n + TRW - 1) / TRW);
    int64_t blocks = 0;
    for (int I = 0; I < nb; ++I) {
        const int tiles = (int)((n - (int64_t)I * TRW + TCW - 1) / TCW);
        blocks += (tiles + SEGW - 1) / SEGW;
    }
    const int vec = ((lda % 4) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    float *in = v0, *out = v1;
    for (int it = 0; it <= N; ++it) {
        sym_gemv_kernel<<<(unsigned)blocks, NTW, 0, s>>>(A, n, lda, in, out, in, scal, counter,
                                                         d_shift_neg, it == N ? d_sigma : nullptr,
                                                         nb, vec);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float *t = in; in = out; out = t;
    }
    return cudaSuccess;
}

cudaError_t launch_alpha_finish(cudaStream_t s, const double *d_s1, const double *d_s2,
                                double alpha_in, double *d_alpha, double *d_shift, int *d_info)
{
    alpha_finish_kernel<<<1, 1, 0, s>>>(d_s1, d_s2, alpha_in, d_alpha, d_shift, d_info);
    return cudaGetLastError();
}
