// CholeskyQR steps of the orthonormalisation (QR 'econ' in Alg. 1):
//   R = chol(G) in FP64 with the dependent-column rule, R^-1 in FP32, and
//   Q = Y R^-1 (a tall x small product on the CUDA cores).
//
// Dependent-column rule: column j is dependent when its pivot (the squared
// norm of y_j after removing the earlier columns) is <= tau * max_i G_ii, or
// is not a number.  Its row of R becomes e_j^T, so it feeds no other column,
// and its column of Q is written as zero (it then adds nothing to Q^T A Q).
#include "ctx.h"

namespace {

constexpr int NT = 1024;
constexpr int SMEM_M = 128;  // largest m kept in shared memory

__global__ void __launch_bounds__(NT)
cholesky_kernel(const double *__restrict__ G, int m, double *R, float *Rinv,
                int *__restrict__ dead, int *__restrict__ d_qrank, double tau, double *gU,
                int *d_status)
{
    extern __shared__ double smd[];
    const bool in_smem = m <= SMEM_M;
    const int ldu = in_smem ? (m + 1) : m;
    double *U = in_smem ? smd : gU;                                  // m x ldu, row-major
    float *X = in_smem ? reinterpret_cast<float *>(smd + m * (m + 1)) : Rinv;  // R^-1
    const int ldx = in_smem ? (m + 1) : m;
    __shared__ double s_gmax;
    __shared__ int s_dead[PSD_MAX_M];
    __shared__ int s_bad;
    const int tid = threadIdx.x;

    // U = upper(G) (row-major: U[i*ldu + k] = G(i,k), k >= i)
    for (int e = tid; e < m * m; e += NT) {
        const int i = e / m, k = e % m;
        if (k >= i) U[i * ldu + k] = G[(int64_t)k * m + i];
    }
    if (tid == 0) {
        double g = 0.0;
        int bad = 0;
        for (int i = 0; i < m; ++i) {
            const double v = G[(int64_t)i * m + i];
            if (!isfinite(v)) bad = 1;
            else if (v > g) g = v;
        }
        s_gmax = g;
        s_bad = bad;
    }
    __syncthreads();
    if (s_bad) psd_set_status(d_status, PSDPROJ_ENOTFINITE);
    const double thr = tau * s_gmax;

    for (int j = 0; j < m; ++j) {
        const double piv = U[j * ldu + j];
        __syncthreads();  // every thread holds piv before row j is rewritten
        const bool dj = !(piv > thr) || !(s_gmax > 0.0);
        if (dj) {
            for (int k = j + 1 + tid; k < m; k += NT) U[j * ldu + k] = 0.0;
            if (tid == 0) { U[j * ldu + j] = 1.0; s_dead[j] = 1; }
            __syncthreads();
            continue;
        }
        const double r = sqrt(piv);
        const double inv = 1.0 / r;
        for (int k = j + 1 + tid; k < m; k += NT) U[j * ldu + k] *= inv;
        if (tid == 0) { U[j * ldu + j] = r; s_dead[j] = 0; }
        __syncthreads();
        // trailing update of the upper triangle: U(i,k) -= R(j,i) R(j,k), j < i <= k
        const int t = m - j - 1;
        for (int e = tid; e < t * t; e += NT) {
            const int a = e / t, b = e - (e / t) * t;
            if (b < a) continue;
            const int i = j + 1 + a, k = j + 1 + b;
            U[i * ldu + k] -= U[j * ldu + i] * U[j * ldu + k];
        }
        __syncthreads();
    }

    // R^-1 (upper) in FP32, row by row from the bottom:
    //   X(i, j) = (delta_ij - sum_{i<k<=j} R(i,k) X(k,j)) / R(i,i),  j >= i.
    // Eight lanes share one output and split the sum.
    for (int e = tid; e < m * m; e += NT) {
        const int i = e / m, k = e % m;
        X[i * ldx + k] = 0.0f;
    }
    __syncthreads();
    const int grp = tid >> 3, lane8 = tid & 7;
    for (int i = m - 1; i >= 0; --i) {
        const float rii = (float)U[i * ldu + i];
        for (int j0 = i; j0 < m; j0 += NT / 8) {
            const int j = j0 + grp;
            float s = 0.0f;
            if (j < m)
                for (int k = i + 1 + lane8; k <= j; k += 8) s = fmaf((float)U[i * ldu + k], X[k * ldx + j], s);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            if (j < m && lane8 == 0) X[i * ldx + j] = ((i == j ? 1.0f : 0.0f) - s) / rii;
        }
        __syncthreads();
    }

    // outputs: R (column-major FP64), R^-1 (column-major FP32)
    if (in_smem) {
        for (int e = tid; e < m * m; e += NT) {
            const int i = e % m, k = e / m;  // (row i, column k)
            R[(int64_t)k * m + i] = (k >= i) ? U[i * ldu + k] : 0.0;
            Rinv[(int64_t)k * m + i] = X[i * ldx + k];
        }
    } else {
        // U (in R) and X (in Rinv) are row-major upper triangles: transpose
        // in place pairwise, zeroing the strict lower parts
        for (int e = tid; e < m * m; e += NT) {
            const int i = e / m, k = e % m;
            if (k > i) {
                const double u = R[(int64_t)i * m + k];
                R[(int64_t)k * m + i] = u;
                R[(int64_t)i * m + k] = 0.0;
                const float x = Rinv[(int64_t)i * m + k];
                Rinv[(int64_t)k * m + i] = x;
                Rinv[(int64_t)i * m + k] = 0.0f;
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < m; j += NT) dead[j] = s_dead[j];
    if (tid == 0 && d_qrank) {
        int r = 0;
        for (int j = 0; j < m; ++j) r += !s_dead[j];
        *d_qrank = r;
    }
}

// Z (n x c) = Y (n x m) * B (m x c, column-major ld m).  Block: 64 rows x 64
// output columns; 256 threads with 4 x 4 micro-tiles.
constexpr int TR = 64, TC = 64, KC = 64;

__global__ void __launch_bounds__(256)
tall_small_kernel(const float *__restrict__ Y, int64_t ldy, int64_t n, int m,
                  const float *__restrict__ B, int c, const int *__restrict__ colmask,
                  const int *__restrict__ d_cols, float *__restrict__ Z, int64_t ldz)
{
    __shared__ float Ys[KC][TR + 4];
    __shared__ float Bs[KC][TC + 4];
    const int64_t r0 = (int64_t)blockIdx.x * TR;
    const int c0 = blockIdx.y * TC;
    const int ncols = d_cols ? min(*d_cols, c) : c;
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < m; k0 += KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < KC * TR; e += 256) {
            const int k = e / TR, r = e % TR;
            const int64_t gr = r0 + r;
            Ys[k][r] = (gr < n && k0 + k < m) ? Y[(int64_t)(k0 + k) * ldy + gr] : 0.0f;
        }
        for (int e = threadIdx.x; e < KC * TC; e += 256) {
            const int cc = e / KC, k = e % KC;
            const int gc = c0 + cc;
            Bs[k][cc] = (gc < ncols && k0 + k < m) ? B[(int64_t)gc * m + k0 + k] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < KC; ++k) {
            float y[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) y[i] = Ys[k][tr * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(y[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gc = c0 + tc * 4 + j;
        if (gc >= c) continue;
        const bool zero = gc >= ncols || (colmask && colmask[gc]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t gr = r0 + tr * 4 + i;
            if (gr < n) Z[(int64_t)gc * ldz + gr] = zero ? 0.0f : acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_cholesky(cudaStream_t s, const double *G, int m, double *R, float *Rinv,
                            int *dead, int *d_qrank, double tau, int *d_status)
{
    // large m works in global memory: U in R, X in Rinv
    const size_t smem = m <= SMEM_M ? (sizeof(double) * m * (m + 1) + sizeof(float) * m * (m + 1)) : 0;
    cudaError_t e = cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cholesky_kernel<<<1, NT, smem, s>>>(G, m, R, Rinv, dead, d_qrank, tau, R, d_status);
    return cudaGetLastError();
}

cudaError_t launch_tall_small(cudaStream_t s, const float *Y, int64_t ldy, int64_t n, int m,
                              const float *B, int c, const int *colmask, const int *d_cols,
                              float *Z, int64_t ldz)
{
    dim3 grid((unsigned)((n + TR - 1) / TR), (unsigned)((c + TC - 1) / TC));
    tall_small_kernel<<<grid, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz);
    return cudaGetLastError();
}
