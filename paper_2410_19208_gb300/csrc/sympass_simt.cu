// Symmetric pass Y = A X + shift X on the CUDA cores in plain FP32 (the
// products of the range finder, Alg. 1, and of the projected core, Alg. 2).
//
// A is read once, upper triangle only.  The upper triangle is cut into
// 64 x 64 tiles (I <= J).  Tile (I, J) feeds Y_I += A_IJ X_J and, off the
// diagonal, Y_J += A_IJ^T X_I.  One thread block owns a segment of up to
// SEG consecutive tiles of one block row I: the Y_I part accumulates in
// shared memory across the segment and is flushed once; the Y_J parts are
// added with atomics per tile.  Diagonal tiles load only j >= i and mirror
// the block in shared memory, so the strict lower triangle is never read.
#include "ctx.h"

namespace {

constexpr int BT = 64;     // tile side
constexpr int LC = 32;     // X columns per chunk
constexpr int SEG = 8;     // tiles per thread block
constexpr int NT = 256;    // threads

__global__ void __launch_bounds__(NT)
sym_pass_simt_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                     const float *__restrict__ X, int64_t ldx, int m, int mchunks,
                     const double *__restrict__ d_shift, float *__restrict__ Y, int64_t ldy,
                     int nb)
{
    extern __shared__ float smem[];
    float *As = smem;                       // BT x (BT+1)
    float *XJ = As + BT * (BT + 1);         // BT x (LC+1)
    float *XI = XJ + BT * (LC + 1);         // BT x (LC+1)
    float *Y1 = XI + BT * (LC + 1);         // BT x (mchunks*LC)
    const int mc = mchunks * LC;

    // map blockIdx -> (block row I, first tile J0)
    int64_t idx = blockIdx.x;
    int I = 0;
    for (; I < nb; ++I) {
        const int cnt = (nb - I + SEG - 1) / SEG;
        if (idx < cnt) break;
        idx -= cnt;
    }
    if (I >= nb) return;
    const int J0 = I + (int)idx * SEG;
    const int J1 = min(nb, J0 + SEG);
    const int tid = threadIdx.x;
    const float shift = d_shift ? (float)(*d_shift) : 0.0f;

    for (int e = tid; e < BT * mc; e += NT) Y1[e] = 0.0f;

    const int64_t r0 = (int64_t)I * BT;
    const bool p2 = tid >= 128;
    const int t = tid & 127;
    const int rr = t >> 3, cc = t & 7;

    for (int J = J0; J < J1; ++J) {
        const int64_t c0g = (int64_t)J * BT;
        const bool diag = (J == I);
        __syncthreads();
        for (int e = tid; e < BT * BT; e += NT) {
            const int r = e / BT, c = e % BT;
            const int64_t gi = r0 + r, gj = c0g + c;
            float v = 0.0f;
            if (gi < n && gj < n && (!diag || c >= r)) v = A[gi * lda + gj];
            As[r * (BT + 1) + c] = v;
        }
        if (diag) {
            __syncthreads();
            for (int e = tid; e < BT * BT; e += NT) {
                const int r = e / BT, c = e % BT;
                if (c < r) As[r * (BT + 1) + c] = As[c * (BT + 1) + r];
            }
        }
        for (int ch = 0; ch < mchunks; ++ch) {
            __syncthreads();
            for (int e = tid; e < BT * LC; e += NT) {
                const int k = e % BT, cl = e / BT;
                const int col = ch * LC + cl;
                const int64_t gj = c0g + k, gi = r0 + k;
                XJ[k * (LC + 1) + cl] = (gj < n && col < m) ? X[(int64_t)col * ldx + gj] : 0.0f;
                if (!diag)
                    XI[k * (LC + 1) + cl] = (gi < n && col < m) ? X[(int64_t)col * ldx + gi] : 0.0f;
            }
            __syncthreads();
            float acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
            if (!p2) {
                // Y_I chunk += A_IJ X_J
#pragma unroll 4
                for (int k = 0; k < BT; ++k) {
                    float a[4], x[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = As[(4 * rr + i) * (BT + 1) + k];
#pragma unroll
                    for (int j = 0; j < 4; ++j) x[j] = XJ[k * (LC + 1) + 4 * cc + j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], x[j], acc[i][j]);
                }
                if (diag) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            acc[i][j] = fmaf(shift, XJ[(4 * rr + i) * (LC + 1) + 4 * cc + j], acc[i][j]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) Y1[(4 * rr + i) * mc + ch * LC + 4 * cc + j] += acc[i][j];
            } else if (!diag) {
                // Y_J chunk += A_IJ^T X_I
#pragma unroll 4
                for (int k = 0; k < BT; ++k) {
                    float a[4], x[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = As[k * (BT + 1) + 4 * rr + i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) x[j] = XI[k * (LC + 1) + 4 * cc + j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], x[j], acc[i][j]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t gr = c0g + 4 * rr + i;
                    if (gr >= n) continue;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int col = ch * LC + 4 * cc + j;
                        if (col < m) atomicAdd(&Y[(int64_t)col * ldy + gr], acc[i][j]);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < BT * mc; e += NT) {
        const int r = e % BT, col = e / BT;
        const int64_t gr = r0 + r;
        if (gr < n && col < m) atomicAdd(&Y[(int64_t)col * ldy + gr], Y1[r * mc + col]);
    }
}

}  // namespace

cudaError_t launch_sym_pass_simt(cudaStream_t s, const float *A, int64_t n, int64_t lda,
                                 const float *X, int64_t ldx, int m, const double *d_shift,
                                 float *Y, int64_t ldy)
{
    const int nb = (int)((n + BT - 1) / BT);
    int64_t segs = 0;
    for (int I = 0; I < nb; ++I) segs += (nb - I + SEG - 1) / SEG;
    const int mchunks = (m + LC - 1) / LC;
    const size_t smem = sizeof(float) * ((size_t)BT * (BT + 1) + 2 * (size_t)BT * (LC + 1) +
                                         (size_t)BT * mchunks * LC);
    cudaError_t e = cudaMemset2DAsync(Y, (size_t)ldy * sizeof(float), 0, (size_t)n * sizeof(float),
                                      (size_t)m, s);
    if (e != cudaSuccess) return e;
    // process-wide attribute: the largest size (m = PSD_MAX_M) for every launch
    const int mchunks_max = (PSD_MAX_M + LC - 1) / LC;
    const size_t smem_max = sizeof(float) * ((size_t)BT * (BT + 1) + 2 * (size_t)BT * (LC + 1) +
                                             (size_t)BT * mchunks_max * LC);
    e = cudaFuncSetAttribute(sym_pass_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_max);
    if (e != cudaSuccess) return e;
    sym_pass_simt_kernel<<<(unsigned)segs, NT, smem, s>>>(A, n, lda, X, ldx, m, mchunks, d_shift,
                                                          Y, ldy, nb);
    return cudaGetLastError();
}
