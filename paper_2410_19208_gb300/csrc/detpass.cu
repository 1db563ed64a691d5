// Deterministic products with A: the FP32 symmetric pass Y = A X + shift X
// (the range finder's products, Alg. 1, and the core product of Alg. 2) and
// the power iteration of Algs. 4 and 5, summed in a fixed order so that a
// repeated call returns bitwise the same result (opts.deterministic).
//
// No atomics: the CTA (I, sp) of a grid (64-row blocks of Y, DSPLIT splits
// of the tile columns) sums block I of Y over the 64 x 64 tiles J of its
// split in increasing J, reading A(I, J) from the upper triangle only: the
// row panel A[i*lda + j] for J > I, the column panel A(J, I)^T for J < I,
// and for J = I the upper half of the diagonal tile, mirrored in shared
// memory.  Each upper-triangle entry is read twice (once from each side).
// A second kernel adds the DSPLIT partial sums in order and the shift term.
// DSPLIT depends on n only, so the order is a function of the problem.
#include "ctx.h"

namespace {

constexpr int DT = 64;        // tile side
constexpr int NTD = 256;

int det_splits(int64_t n)
{
    const int64_t nb = (n + DT - 1) / DT;
    int64_t sp = (304 + nb - 1) / nb;         // about two CTAs per SM at any n
    if (sp > 16) sp = 16;
    if (sp > nb) sp = nb;
    return (int)(sp < 1 ? 1 : sp);
}

// A(I, J) into T (64 x 65), from the upper triangle: direct for J > I,
// transposed from A(J, I) for J < I, mirrored within the tile for J = I.
// Entries past n are zero.
__device__ __forceinline__ void load_tile(const float *__restrict__ A, int64_t n, int64_t lda, int I, int J,
                                          float (*T)[DT + 1])
{
    const int64_t r0 = (int64_t)I * DT, c0 = (int64_t)J * DT;
    if (J > I) {
        for (int e = threadIdx.x; e < DT * DT; e += NTD) {
            const int rr = e / DT, cc = e % DT;
            const int64_t gi = r0 + rr, gj = c0 + cc;
            T[rr][cc] = (gi < n && gj < n) ? A[gi * lda + gj] : 0.0f;
        }
    } else if (J < I) {
        // A(I, J)[rr][cc] = A[(c0 + cc) * lda + r0 + rr]: consecutive threads
        // read consecutive rr (one row of the upper triangle)
        for (int e = threadIdx.x; e < DT * DT; e += NTD) {
            const int rr = e % DT, cc = e / DT;
            const int64_t gi = r0 + rr, gj = c0 + cc;
            T[rr][cc] = (gi < n && gj < n) ? A[gj * lda + gi] : 0.0f;
        }
    } else {
        for (int e = threadIdx.x; e < DT * DT; e += NTD) {
            const int rr = e / DT, cc = e % DT;
            const int64_t gi = r0 + rr, gj = c0 + cc;
            float v = 0.0f;
            if (gi < n && gj < n) v = cc >= rr ? A[gi * lda + gj] : A[gj * lda + gi];
            T[rr][cc] = v;
        }
    }
}

// Partial sums of Y_I over the tiles of split sp: thread (tr, tc) owns rows
// 4 tr .. 4 tr + 3 and columns tc + 16 c (c < MC) of block I.
template <int MC>
__global__ void __launch_bounds__(NTD)
det_pass_partial_kernel(const float *__restrict__ A, int64_t n, int64_t lda, const float *__restrict__ X,
                        int64_t ldx, int m, float *__restrict__ part, int64_t ldp, int nb, int splits)
{
    extern __shared__ float dsm[];
    float (*T)[DT + 1] = reinterpret_cast<float (*)[DT + 1]>(dsm);
    float *Xs = dsm + DT * (DT + 1);             // DT x (16 MC + 1)
    constexpr int XW = 16 * MC + 1;
    const int I = blockIdx.x, sp = blockIdx.y;
    const int J0 = (int)((int64_t)nb * sp / splits), J1 = (int)((int64_t)nb * (sp + 1) / splits);
    const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
    float acc[4][MC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[i][c] = 0.0f;
    for (int J = J0; J < J1; ++J) {
        __syncthreads();
        load_tile(A, n, lda, I, J, T);
        for (int e = threadIdx.x; e < DT * 16 * MC; e += NTD) {
            const int k = e % DT, c = e / DT;
            const int64_t gj = (int64_t)J * DT + k;
            Xs[k * XW + c] = (c < m && gj < n) ? X[(int64_t)c * ldx + gj] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < DT; ++k) {
            float a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = T[4 * tr + i][k];
#pragma unroll
            for (int c = 0; c < MC; ++c) {
                const float x = Xs[k * XW + tc + 16 * c];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][c] = fmaf(a[i], x, acc[i][c]);
            }
        }
    }
    float *ps = part + (int64_t)sp * m * ldp;
#pragma unroll
    for (int c = 0; c < MC; ++c) {
        const int col = tc + 16 * c;
        if (col >= m) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t gr = (int64_t)I * DT + 4 * tr + i;
            if (gr < n) ps[(int64_t)col * ldp + gr] = acc[i][c];
        }
    }
}

// Y = sum over sp (in order) of the partials + shift X.
__global__ void det_pass_reduce_kernel(const float *__restrict__ part, int64_t ldp, int splits,
                                       const float *__restrict__ X, int64_t ldx, int64_t n, int m,
                                       const double *__restrict__ d_shift, float *__restrict__ Y, int64_t ldy)
{
    const float shift = d_shift ? (float)*d_shift : 0.0f;
    const int64_t total = n * (int64_t)m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, i = e - c * n;
        float s = 0.0f;
        for (int sp = 0; sp < splits; ++sp) s += part[((int64_t)sp * m + c) * ldp + i];
        Y[c * ldy + i] = fmaf(shift, X[c * ldx + i], s);
    }
}

// The power iteration's product w = (A + shift I)(sc v), sc = scal[0],
// shift = -*d_shift_neg (0 when NULL): thread (r, kq) sums row r of block I
// over the columns kq, kq + 4, ... of each tile, the four partials of a row
// added by fixed shuffles at the end.
__global__ void __launch_bounds__(NTD)
det_gemv_partial_kernel(const float *__restrict__ A, int64_t n, int64_t lda, const float *__restrict__ x,
                        const double *__restrict__ scal, float *__restrict__ part, int nb, int splits)
{
    __shared__ float T[DT][DT + 1];
    __shared__ float xs[DT];
    const int I = blockIdx.x, sp = blockIdx.y;
    const int J0 = (int)((int64_t)nb * sp / splits), J1 = (int)((int64_t)nb * (sp + 1) / splits);
    const int r = threadIdx.x >> 2, kq = threadIdx.x & 3;
    const float sc = (float)scal[0];
    float acc = 0.0f;
    for (int J = J0; J < J1; ++J) {
        __syncthreads();
        load_tile(A, n, lda, I, J, T);
        if (threadIdx.x < DT) {
            const int64_t gj = (int64_t)J * DT + threadIdx.x;
            xs[threadIdx.x] = gj < n ? x[gj] * sc : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = kq; k < DT; k += 4) acc = fmaf(T[r][k], xs[k], acc);
    }
    acc += __shfl_down_sync(0xffffffffu, acc, 2, 4);
    acc += __shfl_down_sync(0xffffffffu, acc, 1, 4);
    const int64_t gr = (int64_t)I * DT + r;
    if (kq == 0 && gr < n) part[(int64_t)sp * n + gr] = acc;
}

__global__ void det_gemv_reduce_kernel(const float *__restrict__ part, int splits, const float *__restrict__ x,
                                       const double *__restrict__ scal, const double *__restrict__ d_shift_neg,
                                       int64_t n, float *__restrict__ y)
{
    const float sc = (float)scal[0];
    const float shift = d_shift_neg ? (float)(-(*d_shift_neg)) : 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int sp = 0; sp < splits; ++sp) s += part[(int64_t)sp * n + i];
        y[i] = fmaf(shift, x[i] * sc, s);
    }
}

size_t det_pass_smem(int mc) { return sizeof(float) * ((size_t)DT * (DT + 1) + (size_t)DT * (16 * mc + 1)); }

template <int MC>
cudaError_t go_det(cudaStream_t s, const float *A, int64_t n, int64_t lda, const float *X, int64_t ldx, int m,
                   float *part, int64_t ldp, int nb, int splits)
{
    const size_t smem = det_pass_smem(MC);
    cudaError_t e = cudaFuncSetAttribute(det_pass_partial_kernel<MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    det_pass_partial_kernel<MC><<<dim3((unsigned)nb, (unsigned)splits), NTD, smem, s>>>(A, n, lda, X, ldx, m, part,
                                                                                         ldp, nb, splits);
    return cudaGetLastError();
}

}  // namespace

int64_t psd_det_part_floats(int64_t n, int m)
{
    const int64_t ldp = (n + 3) / 4 * 4;
    return (int64_t)det_splits(n) * (m > 1 ? m : 1) * ldp;
}

cudaError_t launch_sym_pass_det(cudaStream_t s, const float *A, int64_t n, int64_t lda, const float *X,
                                int64_t ldx, int m, const double *d_shift, float *Y, int64_t ldy, float *part)
{
    if (m < 1 || m > PSD_MAX_M) return cudaErrorInvalidValue;
    const int nb = (int)((n + DT - 1) / DT);
    const int splits = det_splits(n);
    const int64_t ldp = (n + 3) / 4 * 4;
    cudaError_t e;
    switch ((m + 15) / 16) {
    case 1: e = go_det<1>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 2: e = go_det<2>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 3: e = go_det<3>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 4: e = go_det<4>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 5: e = go_det<5>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 6: e = go_det<6>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 7: e = go_det<7>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 8: e = go_det<8>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 9: e = go_det<9>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 10: e = go_det<10>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 11: e = go_det<11>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 12: e = go_det<12>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 13: e = go_det<13>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 14: e = go_det<14>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    case 15: e = go_det<15>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    default: e = go_det<16>(s, A, n, lda, X, ldx, m, part, ldp, nb, splits); break;
    }
    if (e != cudaSuccess) return e;
    int64_t blocks = (n * (int64_t)m + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    det_pass_reduce_kernel<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(part, ldp, splits, X, ldx, n, m,
                                                                               d_shift, Y, ldy);
    return cudaGetLastError();
}

cudaError_t launch_power_iteration_det(cudaStream_t s, const float *A, int64_t n, int64_t lda, int N,
                                       uint64_t seed, uint32_t stream_id, const double *d_shift_neg,
                                       float *v0, float *v1, double *scal, double *d_sigma, float *part)
{
    cudaError_t e = launch_gaussian(s, seed, stream_id, n, 1, 1, n, v0, n);
    if (e != cudaSuccess) return e;
    e = launch_pi_init(s, scal, v1, n);
    if (e != cudaSuccess) return e;
    const int nb = (int)((n + DT - 1) / DT);
    const int splits = det_splits(n);
    int64_t rblocks = (n + 255) / 256;
    if (rblocks > 152 * 4) rblocks = 152 * 4;
    float *in = v0, *out = v1;
    for (int it = 0; it <= N; ++it) {
        det_gemv_partial_kernel<<<dim3((unsigned)nb, (unsigned)splits), NTD, 0, s>>>(A, n, lda, in, scal, part, nb,
                                                                                     splits);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        det_gemv_reduce_kernel<<<(unsigned)rblocks, 256, 0, s>>>(part, splits, in, scal, d_shift_neg, n, out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_pi_norm(s, out, in, n, scal, it == N ? d_sigma : nullptr);
        if (e != cudaSuccess) return e;
        float *t = in; in = out; out = t;
    }
    return cudaSuccess;
}
