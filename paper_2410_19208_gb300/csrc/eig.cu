// Small symmetric eigensolver of Alg. 2 line 2 / Alg. 3 line 3 ("eig(Q^T X Q)"):
// parallel cyclic Jacobi in one thread block.
//
// The m x m core is held in shared memory in FP32 (GB300's FP64 pipe runs at
// about 2 FMA/clk/SM, so an FP64 Jacobi on 112 x 112 would take ~17 ms; the
// FP32 solve has backward error ~eps32 ||C||, and the PSD projection is
// non-expansive in the Frobenius norm (Prop. 1), so the output moves by at
// most that much).  Each sweep runs the m-1 rounds of the round-robin
// (circle) ordering; a round applies m/2 disjoint rotations at once: row
// update, then column update of C and V.  Rotations use the classical stable
// formula t = sign(tau) / (|tau| + sqrt(1 + tau^2)).  Sweeps stop when the
// off-diagonal Frobenius norm is <= 1e-6 ||C||_F.  Eigenpairs are returned
// sorted by decreasing eigenvalue.
#include "ctx.h"

namespace {

constexpr int NT = 1024;
constexpr int MAX_SWEEPS = 40;

__global__ void __launch_bounds__(NT)
eig_kernel(const double *__restrict__ C, int m, float *__restrict__ Vout,
           double *__restrict__ dout, float *gA, float *gV, int smem_A, int smem_V,
           int *d_status)
{
    extern __shared__ float sm[];
    const int mm = m + (m & 1);           // even size (ghost index when m is odd)
    const int ld = mm + 1;
    float *A = smem_A ? sm : gA;
    float *V = smem_V ? (sm + (smem_A ? mm * ld : 0)) : gV;
    __shared__ int rp[PSD_MAX_M / 2 + 1], rq[PSD_MAX_M / 2 + 1];
    __shared__ float rc[PSD_MAX_M / 2 + 1], rs[PSD_MAX_M / 2 + 1];
    __shared__ float red[NT / 32];
    __shared__ float s_off, s_fro;
    __shared__ int s_rank[PSD_MAX_M];
    const int tid = threadIdx.x;
    const int half = mm / 2;
    if (tid < half) rs[tid] = 0.0f;

    for (int e = tid; e < mm * mm; e += NT) {
        const int i = e / mm, j = e % mm;
        const float v = (i < m && j < m) ? (float)C[(int64_t)j * m + i] : 0.0f;
        A[i * ld + j] = v;
        V[i * ld + j] = (i == j) ? 1.0f : 0.0f;
    }
    __syncthreads();

    int sweep = 0;
    bool converged = false;
    for (; sweep <= MAX_SWEEPS; ++sweep) {
        // off-diagonal and full Frobenius norms
        float off = 0.0f, fro = 0.0f;
        for (int e = tid; e < mm * mm; e += NT) {
            const int i = e / mm, j = e % mm;
            const float v = A[i * ld + j];
            fro += v * v;
            if (i != j) off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            fro += __shfl_xor_sync(0xffffffffu, fro, o);
        }
        if ((tid & 31) == 0) red[tid >> 5] = off;
        __syncthreads();
        if (tid == 0) {
            float s = 0.0f;
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            s_off = s;
        }
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = fro;
        __syncthreads();
        if (tid == 0) {
            float s = 0.0f;
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            s_fro = s;
        }
        __syncthreads();
        if (!(s_off > 1e-12f * s_fro)) { converged = true; break; }
        if (!isfinite(s_fro)) break;
        if (sweep == MAX_SWEEPS) break;

        for (int r = 0; r < mm - 1; ++r) {
            if (tid < half) {
                // set the pair rotated in the previous round to an exact zero
                // (it is zero in exact arithmetic); no pair repeats in
                // consecutive rounds, so no other thread reads it now
                if ((sweep > 0 || r > 0) && rs[tid] != 0.0f) {
                    A[rp[tid] * ld + rq[tid]] = 0.0f;
                    A[rq[tid] * ld + rp[tid]] = 0.0f;
                }
                int p, q;
                if (tid == 0) { p = mm - 1; q = r; }
                else { p = (r + tid) % (mm - 1); q = (r - tid + mm - 1) % (mm - 1); }
                if (p > q) { const int t = p; p = q; q = t; }
                const float apq = A[p * ld + q];
                float c = 1.0f, s = 0.0f;
                if (apq != 0.0f) {
                    const float app = A[p * ld + p], aqq = A[q * ld + q];
                    const float tau = (aqq - app) / (2.0f * apq);
                    float t;
                    if (fabsf(tau) > 1e18f) t = 0.5f / tau;
                    else t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
                    c = rsqrtf(1.0f + t * t);
                    s = t * c;
                }
                rp[tid] = p; rq[tid] = q; rc[tid] = c; rs[tid] = s;
            }
            __syncthreads();
            // rows p, q of A
            for (int e = tid; e < half * mm; e += NT) {
                const int k = e / mm, col = e - (e / mm) * mm;
                const float c = rc[k], s = rs[k];
                if (s == 0.0f) continue;
                const int p = rp[k], q = rq[k];
                const float x = A[p * ld + col], y = A[q * ld + col];
                A[p * ld + col] = c * x - s * y;
                A[q * ld + col] = s * x + c * y;
            }
            __syncthreads();
            // columns p, q of A and V
            for (int e = tid; e < half * mm; e += NT) {
                const int k = e / mm, row = e - (e / mm) * mm;
                const float c = rc[k], s = rs[k];
                if (s == 0.0f) continue;
                const int p = rp[k], q = rq[k];
                const float x = A[row * ld + p], y = A[row * ld + q];
                A[row * ld + p] = c * x - s * y;
                A[row * ld + q] = s * x + c * y;
                const float vx = V[row * ld + p], vy = V[row * ld + q];
                V[row * ld + p] = c * vx - s * vy;
                V[row * ld + q] = s * vx + c * vy;
            }
            __syncthreads();
        }
    }
    if (!converged) psd_set_status(d_status, PSDPROJ_ENOCONV);

    // sort by decreasing eigenvalue (rank of each index; ties by index)
    for (int i = tid; i < m; i += NT) {
        const float di = A[i * ld + i];
        int rk = 0;
        for (int j = 0; j < m; ++j) {
            const float dj = A[j * ld + j];
            rk += (dj > di) || (dj == di && j < i);
        }
        s_rank[i] = rk;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += NT) {
        const int row = e % m, col = e / m;
        Vout[(int64_t)s_rank[col] * m + row] = V[row * ld + col];
    }
    for (int i = tid; i < m; i += NT) dout[s_rank[i]] = (double)A[i * ld + i];
}

}  // namespace

cudaError_t launch_eig(cudaStream_t s, const double *C, int m, float *V, double *d,
                       float *scratch, int *d_status)
{
    const int mm = m + (m & 1);
    const size_t mat = sizeof(float) * (size_t)mm * (mm + 1);
    int smem_A = 1, smem_V = 1;
    size_t smem = 2 * mat;
    if (smem > 200 * 1024) { smem_V = 0; smem = mat; }
    if (smem > 200 * 1024) { smem_A = 0; smem = 0; }
    float *gA = scratch;
    float *gV = scratch + (size_t)mm * (mm + 1);
    cudaError_t e = cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    eig_kernel<<<1, NT, smem, s>>>(C, m, V, d, gA, gV, smem_A, smem_V, d_status);
    return cudaGetLastError();
}
