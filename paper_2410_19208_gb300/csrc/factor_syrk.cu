// Last line of Alg. 2 (and, through Lemma 4, of Alg. 3):
//   X+_hat = Q V D+ V^T Q^T = W W^T with W = Q V sqrt(max(D, 0)).
// factor_prep forms M = V sqrt(max(D,0)) (eigenpairs sorted decreasingly, so
// the r+ positive ones come first) and r+; W = Q M is a tall x small product
// (cholesky.cu); the SIMT SYRK below writes P = W W^T.
#include "ctx.h"

namespace {

// M = V diag(sqrt(max(d, 0))) and the count of positive eigenvalues; one
// root per column (FP64 roots are slow on this GPU), then the scaling
__device__ __forceinline__ void factor_prep_body(const float *__restrict__ V, const double *__restrict__ d, int m,
                                                 float *__restrict__ M, int *__restrict__ d_rank,
                                                 int *__restrict__ d_rank_out)
{
    __shared__ int s_r;
    __shared__ float s_g[PSD_MAX_M];
    if (threadIdx.x == 0) s_r = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double dj = d[j];
        if (dj > 0.0) atomicAdd(&s_r, 1);
        s_g[j] = dj > 0.0 ? sqrtf((float)dj) : 0.0f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) M[e] = V[e] * s_g[e / m];
    if (threadIdx.x == 0 && d_rank) *d_rank = s_r;
    if (threadIdx.x == 0 && d_rank_out) *d_rank_out = s_r;
}

__global__ void factor_prep_kernel(const float *__restrict__ V, const double *__restrict__ d,
                                   int m, float *__restrict__ M, int *__restrict__ d_rank)
{
    factor_prep_body(V, d, m, M, d_rank, nullptr);
}

// many problems in one launch: block b prepares entry b
__global__ void factor_prep_grouped_kernel(const psd_g_factor *__restrict__ tab)
{
    const psd_g_factor a = tab[blockIdx.x];
    factor_prep_body(a.V, a.d, a.m, a.M, a.d_rank, a.d_rank_out);
}

// P tile (I, J), I <= J, 128 x 128, 256 threads, 8 x 8 micro-tiles.
constexpr int TS = 128, KC = 16;

__global__ void __launch_bounds__(256)
syrk_simt_kernel(const float *__restrict__ W, int64_t ldw, int64_t n, int m,
                 const int *__restrict__ d_rank, float *__restrict__ P, int64_t ldp,
                 int upper_only, int nb)
{
    __shared__ float Wi[KC][TS + 4];
    __shared__ float Wj[KC][TS + 4];
    // blockIdx.x -> (I <= J) over the upper triangle of tiles
    int t = blockIdx.x, I = 0;
    while (t >= nb - I) { t -= nb - I; ++I; }
    const int J = I + t;
    const int64_t r0 = (int64_t)I * TS, c0 = (int64_t)J * TS;
    const int r = d_rank ? min(*d_rank, m) : m;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < r; k0 += KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < KC * TS; e += 256) {
            const int k = e / TS, rr = e % TS;
            const bool kok = k0 + k < r;
            const int64_t gi = r0 + rr, gj = c0 + rr;
            Wi[k][rr] = (kok && gi < n) ? W[(int64_t)(k0 + k) * ldw + gi] : 0.0f;
            Wj[k][rr] = (kok && gj < n) ? W[(int64_t)(k0 + k) * ldw + gj] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            float a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = Wi[k][ty * 8 + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Wj[k][tx * 8 + j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
    }
    const bool diag = (I == J);
    // direct tile
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gr = r0 + ty * 8 + i;
        if (gr >= n) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t gc = c0 + tx * 8 + j;
            if (gc < n && (!diag || !upper_only || gc >= gr)) P[gr * ldp + gc] = acc[i][j];
        }
    }
    // mirrored tile (full output, off-diagonal tiles)
    if (!diag && !upper_only) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t gr = c0 + tx * 8 + j;
            if (gr >= n) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t gc = r0 + ty * 8 + i;
                if (gc < n) P[gr * ldp + gc] = acc[i][j];
            }
        }
    }
}

__global__ void copy_tall_kernel(const float *__restrict__ X, int64_t ldx, int64_t n, int m,
                                 float *__restrict__ Y, int64_t ldy)
{
    const int64_t total = n * (int64_t)m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - (e / n) * n;
        Y[c * ldy + i] = X[c * ldx + i];
    }
}

}  // namespace

cudaError_t launch_factor_prep(cudaStream_t s, const float *V, const double *d, int m, float *M,
                               int *d_rank)
{
    factor_prep_kernel<<<1, 1024, 0, s>>>(V, d, m, M, d_rank);
    return cudaGetLastError();
}

cudaError_t launch_factor_prep_grouped(cudaStream_t s, const psd_g_factor *tab, int count)
{
    if (count < 1) return cudaErrorInvalidValue;
    factor_prep_grouped_kernel<<<(unsigned)count, 1024, 0, s>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_syrk_simt(cudaStream_t s, const float *W, int64_t ldw, int64_t n, int m,
                             const int *d_rank, float *P, int64_t ldp, int upper_only)
{
    const int nb = (int)((n + TS - 1) / TS);
    const int64_t tiles = (int64_t)nb * (nb + 1) / 2;
    syrk_simt_kernel<<<(unsigned)tiles, 256, 0, s>>>(W, ldw, n, m, d_rank, P, ldp, upper_only, nb);
    return cudaGetLastError();
}

cudaError_t launch_copy_tall(cudaStream_t s, const float *X, int64_t ldx, int64_t n, int m,
                             float *Y, int64_t ldy)
{
    const int64_t total = n * (int64_t)m;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    copy_tall_kernel<<<blocks, 256, 0, s>>>(X, ldx, n, m, Y, ldy);
    return cudaGetLastError();
}
