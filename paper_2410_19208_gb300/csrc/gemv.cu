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

// scal[0]: scale of the input vector; scal[1]: norm of the last output.
// A block owns a segment of SEGW tiles (32 rows x 128 columns each) of one
// block row.  Warp w holds rows 4w..4w+3, lane l columns 4l..4l+3 of every
// tile; the loads of the whole segment are independent, and the column
// partial sums stay in registers until the segment ends (one barrier).
__global__ void __launch_bounds__(NTW, 2)
sym_gemv_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                const float *__restrict__ x, float *__restrict__ y, float *__restrict__ other,
                double *scal, unsigned *counter, const double *d_shift_neg, double *d_sigma,
                int nb, int vec)
{
    __shared__ float colsum[8][SEGW * TCW];
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
    const int t0 = (int)idx * SEGW;
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
    // two batches of four tiles: the 16 float4 loads of a batch are issued
    // together (predicated, no branches), then consumed
#pragma unroll 1
    for (int b = 0; b < SEGW; b += 4) {
        float4 va[4][4];
        float colacc[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int tt = t0 + b + t;
            const int64_t c0 = row0 + (int64_t)tt * TCW + lane * 4;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t gr = row0 + warp * 4 + i;
                const bool ok = vec && tt < tiles && gr < n && c0 + 3 < n;
                const float4 *src = reinterpret_cast<const float4 *>(A + (ok ? gr * lda + c0 : 0));
                va[t][i] = ok ? __ldcs(src) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int tt = t0 + b + t;
            const int64_t c0 = row0 + (int64_t)tt * TCW + lane * 4;
            float xc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                colacc[t][j] = 0.0f;
                xc[j] = (tt < tiles && c0 + j < n) ? x[c0 + j] * sc : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t gr = row0 + warp * 4 + i;
                float a[4] = {va[t][i].x, va[t][i].y, va[t][i].z, va[t][i].w};
                if (tt < tiles && gr < n && (!vec || c0 + 3 >= n) && c0 < n) {
                    // ragged right edge or unaligned rows: scalar loads
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        a[j] = (c0 + j < n && c0 + j >= gr) ? A[gr * lda + c0 + j] : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // strictly-lower entries of the diagonal tile are discarded
                    const float aj = (c0 + j >= gr) ? a[j] : 0.0f;
                    rowacc[i] = fmaf(aj, xc[j], rowacc[i]);
                    colacc[t][j] = fmaf((c0 + j > gr) ? aj : 0.0f, xr[i], colacc[t][j]);
                }
            }
        }
        // this thread's column partials of the batch (one owner per slot)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int j = 0; j < 4; ++j) colsum[warp][(b + t) * TCW + lane * 4 + j] = colacc[t][j];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < SEGW * TCW; c += NTW) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += colsum[w][c];
        const int64_t gc = row0 + (int64_t)t0 * TCW + c;
        if (gc < n && s != 0.0f) atomicAdd(&y[gc], s);
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
