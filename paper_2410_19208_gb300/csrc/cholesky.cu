// CholeskyQR steps of the orthonormalisation (QR 'econ' in Alg. 1):
//   R = chol(G) (FP64 for the first pass of CholeskyQR2, FP32 for the second,
//   whose Gram is I + O(eps)) with the dependent-column rule, R^-1 in FP32,
//   and Q = Y R^-1 (a tall x small product on the CUDA cores).
// The factorization is right-looking with two block barriers per column;
// each thread owns a fixed set of upper-triangle entries.
//
// Dependent-column rule: column j is dependent when its pivot (the squared
// norm of y_j after removing the earlier columns) is <= tau * max_i G_ii, or
// is not a number.  Its row of R becomes e_j^T, so it feeds no other column,
// and its column of Q is written as zero (it then adds nothing to Q^T A Q).
#include "ctx.h"

namespace {

constexpr int NT = 1024;
constexpr int SMEM_M = 128;  // largest m kept in shared memory
constexpr int EPT = (SMEM_M * (SMEM_M + 1) / 2 + NT - 1) / NT;  // upper entries per thread

// T = double: the first CholeskyQR pass (the Gram of the raw sketch, which can
// be ill-conditioned); T = float: the second pass, whose Gram is I + O(eps).
template <typename T>
__global__ void __launch_bounds__(NT)
cholesky_kernel(const double *__restrict__ G, int m, double *R, float *Rinv,
                int *__restrict__ dead, int *__restrict__ d_qrank, double tau, T *gU, T *growj,
                int *d_status)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const bool in_smem = m <= SMEM_M;
    const int ldu = in_smem ? (m + 1) : m;
    T *U = in_smem ? reinterpret_cast<T *>(smraw) : gU;            // row-major upper triangle
    T *rowj = in_smem ? (U + m * (m + 1)) : growj;                  // scaled row j
    float *Rs = in_smem ? reinterpret_cast<float *>(rowj + m) : nullptr;  // FP32 R (row-major)
    __shared__ double s_gmax;
    __shared__ int s_dead[PSD_MAX_M];
    __shared__ int s_bad;
    __shared__ T s_r, s_inv;
    __shared__ int s_dj;
    const int tid = threadIdx.x;
    const int nup = m * (m + 1) / 2;

    // U = upper(G)
    for (int e = tid; e < m * m; e += NT) {
        const int i = e / m, k = e - (e / m) * m;
        if (k >= i) U[i * ldu + k] = (T)G[(int64_t)k * m + i];
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
    // this thread's upper-triangle entries (fixed for the whole factorization)
    int ei[EPT], ek[EPT];
#pragma unroll
    for (int c = 0; c < EPT; ++c) {
        const int e = tid + c * NT;
        ei[c] = -1;
        ek[c] = 0;
        if (in_smem && e < nup) {
            // e -> (i <= k), row-major over the upper triangle
            const float hb = 2.0f * m + 1.0f;
            int i = (int)((hb - sqrtf(fmaxf(hb * hb - 8.0f * e, 0.0f))) * 0.5f);
            i = max(0, min(i, m - 1));
            while (i > 0 && i * m - i * (i - 1) / 2 > e) --i;
            while (i + 1 < m && (i + 1) * m - (i + 1) * i / 2 <= e) ++i;
            ei[c] = i;
            ek[c] = i + (e - (i * m - i * (i - 1) / 2));
        }
    }
    __syncthreads();
    if (s_bad) psd_set_status(d_status, PSDPROJ_ENOTFINITE);
    const T thr = (T)(tau * s_gmax);
    const bool any = s_gmax > 0.0;

    for (int j = 0; j < m; ++j) {
        // phase A: pivot (one thread: FP64 sqrt and division are slow on
        // this GPU) and scaled row j
        if (tid == 0) {
            const T piv = U[j * ldu + j];
            const bool d0 = !(piv > thr) || !any;
            const T r0 = d0 ? (T)1 : (T)sqrt(piv);
            s_r = r0;
            s_inv = (T)1 / r0;
            s_dj = d0 ? 1 : 0;
        }
        __syncthreads();
        const bool dj = s_dj != 0;
        const T r = s_r, inv = s_inv;
        for (int k = j + tid; k < m; k += NT) {
            const T v = (k == j) ? r : (dj ? (T)0 : U[j * ldu + k] * inv);
            U[j * ldu + k] = v;
            rowj[k] = (k == j) ? (T)0 : v;
        }
        if (tid == 0) s_dead[j] = dj ? 1 : 0;
        __syncthreads();
        // phase B: trailing update U(i,k) -= R(j,i) R(j,k), j < i <= k
        if (!dj) {
            if (in_smem) {
#pragma unroll
                for (int c = 0; c < EPT; ++c) {
                    if (ei[c] > j) {
                        const int i = ei[c], k = ek[c];
                        U[i * ldu + k] -= rowj[i] * rowj[k];
                    }
                }
            } else {
                const int t = m - j - 1;
                for (int e = tid; e < t * t; e += NT) {
                    const int a = e / t, b = e - (e / t) * t;
                    if (b < a) continue;
                    const int i = j + 1 + a, k = j + 1 + b;
                    U[i * ldu + k] -= rowj[i] * rowj[k];
                }
            }
        }
        __syncthreads();
    }

    // R (column-major FP64) and an FP32 copy for the inverse
    for (int e = tid; e < m * m; e += NT) {
        const int i = e % m, k = e / m;  // (row i, column k)
        const T u = (k >= i) ? U[i * ldu + k] : (T)0;
        R[(int64_t)k * m + i] = (double)u;
        if (in_smem) Rs[i * ldu + k] = (float)u;
    }
    __syncthreads();
    // R^-1 (upper, FP32): one warp per column j, back substitution
    //   x_j = 1 / R_jj;  x_i = -(sum_{i<k<=j} R_ik x_k) / R_ii  (i = j-1 .. 0)
    // x is kept in the output column of Rinv (column-major, ld m).
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < m; j += NT / 32) {
        float *x = Rinv + (int64_t)j * m;
        for (int i = lane; i < m; i += 32) x[i] = 0.0f;
        __syncwarp();
        auto Rget = [&](int i, int k) -> float {
            return in_smem ? Rs[i * ldu + k] : (float)R[(int64_t)k * m + i];
        };
        if (lane == 0) x[j] = 1.0f / Rget(j, j);
        __syncwarp();
        for (int i = j - 1; i >= 0; --i) {
            float sacc = 0.0f;
            for (int k = i + 1 + lane; k <= j; k += 32) sacc = fmaf(Rget(i, k), x[k], sacc);
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            if (lane == 0) x[i] = -sacc / Rget(i, i);
            __syncwarp();
        }
    }
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
                            int *dead, int *d_qrank, double tau, int *d_status, int fp64,
                            double *gscratch)
{
    // large m works in global memory (gscratch: m*m + m doubles)
    if (fp64) {
        const size_t smem = m <= SMEM_M ? (sizeof(double) * (m * (m + 1) + m) + sizeof(float) * m * (m + 1)) : 0;
        cudaError_t e = cudaFuncSetAttribute(cholesky_kernel<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cholesky_kernel<double><<<1, NT, smem, s>>>(G, m, R, Rinv, dead, d_qrank, tau, gscratch,
                                                    gscratch + (size_t)m * m, d_status);
    } else {
        float *fs = reinterpret_cast<float *>(gscratch);
        const size_t smem = m <= SMEM_M ? (sizeof(float) * (m * (m + 1) + m) + sizeof(float) * m * (m + 1)) : 0;
        cudaError_t e = cudaFuncSetAttribute(cholesky_kernel<float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cholesky_kernel<float><<<1, NT, smem, s>>>(G, m, R, Rinv, dead, d_qrank, tau, fs,
                                                   fs + (size_t)m * m, d_status);
    }
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
