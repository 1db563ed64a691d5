// Kernels of the dual gradient descent for the semidefinite least-squares
// problem (Alg. 6): forming X = C / rho + sum_i y_i A_i, the gradient terms
// <A_i, W W^T> = sum_c w_c^T (A_i w_c), and the warm-started test matrix;
// and the upper-triangle gather of the host-buffer calls.
#include "ctx.h"

namespace {

// X[r, j] = C[r, j] / rho + sum_i y_i A_i[r, j] for j >= r (upper triangle,
// row-major, leading dimensions ld of the inputs and ldx of X); FP64 sums.
// grid.y = row r, grid.x x blockDim.x covers the columns r .. n-1.
__global__ void sdls_combine_kernel(const float *__restrict__ C, const float *const *__restrict__ A, int mc,
                                    const double *__restrict__ y, double inv_rho, int64_t n, int64_t ld,
                                    float *__restrict__ X, int64_t ldx)
{
    const int64_t r = blockIdx.y;
    for (int64_t j = r + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double v = inv_rho * (double)C[r * ld + j];
        for (int i = 0; i < mc; ++i) v += y[i] * (double)A[i][r * ld + j];
        X[r * ldx + j] = (float)v;
    }
}

// g[idx] += sum over i < n, c < m of W[c*ld + i] * Z[c*ld + i] (FP64)
__global__ void sdls_dot_kernel(const float *__restrict__ W, const float *__restrict__ Z, int64_t n, int m,
                                int64_t ld, double *g)
{
    __shared__ double part[32];
    double acc = 0.0;
    const int64_t total = n * (int64_t)m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        acc += (double)W[c * ld + i] * (double)Z[c * ld + i];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(g, v);
    }
}

// Omega[:, c] = Q[:, c] for the columns the orthonormalisation kept
// (dead[c] == 0); the others keep the fresh Gaussian column already there
__global__ void sdls_warm_omega_kernel(float *__restrict__ Om, const float *__restrict__ Q,
                                       const int *__restrict__ dead, int64_t n, int m, int64_t ld)
{
    const int64_t total = n * (int64_t)m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        if (!dead[c]) Om[c * ld + i] = Q[c * ld + i];
    }
}

// D[i*ldd + j] = S[i*lds + j], j >= i: one block per row, float4 where both
// rows allow it (16-byte aligned starts)
__global__ void copy_upper_kernel(const float *__restrict__ S, int64_t n, int64_t lds, float *__restrict__ D,
                                  int64_t ldd, int vec)
{
    const int64_t i = blockIdx.x;
    const float *src = S + i * lds;
    float *dst = D + i * ldd;
    int64_t j0 = i;
    if (vec) {
        const int64_t a = (i + 3) & ~(int64_t)3;                 // first 4-aligned column >= i
        for (int64_t j = i + threadIdx.x; j < a && j < n; j += blockDim.x) dst[j] = src[j];
        const int64_t nv = (n - a) >> 2;
        for (int64_t v = threadIdx.x; v < nv; v += blockDim.x)
            reinterpret_cast<float4 *>(dst + a)[v] = __ldcs(reinterpret_cast<const float4 *>(src + a) + v);
        j0 = a + 4 * (nv > 0 ? nv : 0);
        if (j0 < a) j0 = a;
    }
    for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) dst[j] = src[j];
}

unsigned blocks_for(int64_t total, int64_t cap)
{
    int64_t b = (total + 255) / 256;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_sdls_combine(cudaStream_t s, const float *C, const float *const *dA, int mc, const double *y,
                                double rho, int64_t n, int64_t ld, float *X, int64_t ldx)
{
    if (n > 65535) return cudaErrorInvalidValue;       // one grid row per matrix row
    const unsigned bx = (unsigned)((n + 255) / 256 < 8 ? (n + 255) / 256 : 8);
    sdls_combine_kernel<<<dim3(bx, (unsigned)n), 256, 0, s>>>(C, dA, mc, y, 1.0 / rho, n, ld, X, ldx);
    return cudaGetLastError();
}

cudaError_t launch_sdls_dot(cudaStream_t s, const float *W, const float *Z, int64_t n, int m, int64_t ld,
                            double *g)
{
    sdls_dot_kernel<<<blocks_for(n * (int64_t)m, 152 * 4), 256, 0, s>>>(W, Z, n, m, ld, g);
    return cudaGetLastError();
}

cudaError_t launch_sdls_warm_omega(cudaStream_t s, float *Om, const float *Q, const int *dead, int64_t n,
                                   int m, int64_t ld)
{
    sdls_warm_omega_kernel<<<blocks_for(n * (int64_t)m, 152 * 8), 256, 0, s>>>(Om, Q, dead, n, m, ld);
    return cudaGetLastError();
}

cudaError_t launch_copy_upper(cudaStream_t s, const float *S, int64_t n, int64_t lds, float *D, int64_t ldd)
{
    if (n > 0x7fffffff) return cudaErrorInvalidValue;
    const int vec = (lds % 4) == 0 && (ldd % 4) == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(D) & 15) == 0;
    copy_upper_kernel<<<(unsigned)n, 256, 0, s>>>(S, n, lds, D, ldd, vec);
    return cudaGetLastError();
}
