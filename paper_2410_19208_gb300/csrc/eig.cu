// Small symmetric eigensolver of Alg. 2 line 2 / Alg. 3 line 3 ("eig(Q^T X Q)"):
// parallel cyclic Jacobi in one thread block.  Used on its own
// (PSDPROJ_EIG_JACOBI) or as the fallback of the tridiagonal solver
// (eig_tridiag.cu), in which case it runs only when that solver's failure
// flag is set.
//
// The m x m core is held in shared memory in FP32 (GB300's FP64 pipe runs at
// about 2 FMA/clk/SM, so an FP64 Jacobi on 112 x 112 would take ~17 ms; the
// FP32 solve has backward error ~eps32 ||C||, and the PSD projection is
// non-expansive in the Frobenius norm (Prop. 1), so the output moves by at
// most that much).  Each sweep runs the m-1 rounds of the round-robin
// (circle) ordering; a round applies m/2 disjoint rotations J at once as
// C <- J^T C J.  Because C is symmetric, the update is done per 2 x 2 block
// between two rotation pairs (k, k'): B <- R_k^T B R_k', one thread per block
// of the upper block triangle, mirrored to the lower one; the rotated
// pair's own off-diagonal entry is set to an exact zero.  Eigenvectors are
// accumulated in V^T (row-major) so that each rotation updates two
// contiguous rows.  Rotations use the classical stable formula
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2) with
// correctly rounded square root and division (no approximate reciprocal
// square root: its bias would make every rotation slightly contractive).
// Sweeps stop when the off-diagonal Frobenius norm is <= 1e-6 ||C||_F.
// Eigenpairs are returned sorted by decreasing eigenvalue.
#include "ctx.h"

namespace {

constexpr int NT = 512;
constexpr int MAX_SWEEPS = 40;
constexpr int MAXH = PSD_MAX_M / 2;

__device__ __forceinline__ void eig_body(const double *__restrict__ C, int m, float *__restrict__ Vout,
                                         double *__restrict__ dout, float *gA, float *gV, int smem_A, int smem_V,
                                         int *d_status, const int *only_if)
{
    // fallback use: run only when the tridiagonal solver flagged a failure
    if (only_if && *only_if == 0) return;
    extern __shared__ float sm[];
    const int mm = m + (m & 1);           // even size (ghost index when m is odd)
    const int ld = mm + 1;
    const int ldv = mm + 4;               // V^T rows, 16-byte aligned
    float *A = smem_A ? sm : gA;
    float *Vt = smem_V ? (sm + (smem_A ? ((mm * ld + 3) & ~3) : 0)) : gV;
    __shared__ int rp[MAXH], rq[MAXH];
    __shared__ float rs[MAXH], rt[MAXH], rtau[MAXH];
    __shared__ int s_rot;
    __shared__ float s_fro;
    __shared__ float red[2][NT / 32];
    __shared__ int s_rank[PSD_MAX_M];
    __shared__ int s_done;
    const int tid = threadIdx.x;
    const int half = mm / 2;
    const int nblk = half * (half + 1) / 2;
    if (tid == 0) s_rot = 0;

    for (int e = tid; e < mm * mm; e += NT) {
        const int i = e / mm, j = e % mm;
        A[i * ld + j] = (i < m && j < m) ? (float)C[(int64_t)j * m + i] : 0.0f;
        Vt[i * ldv + j] = (i == j) ? 1.0f : 0.0f;
    }
    __syncthreads();

    bool converged = false;
    float abs_floor = 0.0f;
    for (int sweep = 0; sweep <= MAX_SWEEPS; ++sweep) {
        // off-diagonal and full Frobenius norms
        float off = 0.0f, fro = 0.0f;
        for (int e = tid; e < mm * mm; e += NT) {
            const int i = e / mm, j = e - (e / mm) * mm;
            const float v = A[i * ld + j];
            fro = fmaf(v, v, fro);
            if (i != j) off = fmaf(v, v, off);
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            fro += __shfl_xor_sync(0xffffffffu, fro, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = off;
            red[1][tid >> 5] = fro;
        }
        __syncthreads();
        if (tid == 0) {
            float so = 0.0f, sf = 0.0f;
            for (int w = 0; w < NT / 32; ++w) {
                so += red[0][w];
                sf += red[1][w];
            }
            // converged: off-diagonal mass below 1e-6 ||C||_F, or the last
            // sweep found no entry worth a rotation
            s_done = (!(so > 1e-12f * sf) || (sweep > 0 && s_rot == 0)) ? 1 : (!isfinite(sf) ? 2 : 0);
            s_rot = 0;
            s_fro = sf;
        }
        __syncthreads();
        if (s_done == 1) { converged = true; break; }
        if (s_done == 2 || sweep == MAX_SWEEPS) break;
        if (sweep == 0) abs_floor = 1e-10f * sqrtf(s_fro);

        for (int r = 0; r < mm - 1; ++r) {
            // the rotation of each pair of round r of the circle ordering
            if (tid < half) {
                int p, q;
                if (tid == 0) { p = mm - 1; q = r; }
                else { p = (r + tid) % (mm - 1); q = (r - tid + mm - 1) % (mm - 1); }
                if (p > q) { const int t = p; p = q; q = t; }
                const float apq = A[p * ld + q];
                const float app = A[p * ld + p], aqq = A[q * ld + q];
                float c = 1.0f, s = 0.0f, t = 0.0f;
                // entries below eps * sqrt(|a_pp a_qq|) (or an absolute floor
                // far below ||C||) change no eigenvalue: no rotation
                if (fabsf(apq) > fmaxf(5.96e-8f * sqrtf(fabsf(app * aqq)), abs_floor)) {
                    const float th = (aqq - app) / (2.0f * apq);
                    if (fabsf(th) > 1e18f) t = 0.5f / th;
                    else t = copysignf(1.0f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
                    c = 1.0f / sqrtf(fmaf(t, t, 1.0f));
                    s = t * c;
                    s_rot = 1;  // any rotation in this sweep (plain store: same value)
                }
                rp[tid] = p; rq[tid] = q; rs[tid] = s; rt[tid] = t;
                rtau[tid] = s / (1.0f + c);
            }
            __syncthreads();
            // 2 x 2 blocks (k <= k') of C and the two rows of V^T per pair
            for (int e = tid; e < nblk; e += NT) {
                // e -> (k, k'), row-major over the upper block triangle; row k
                // starts at k*half - k(k-1)/2
                const float hb = 2.0f * half + 1.0f;
                int k = (int)((hb - sqrtf(fmaxf(hb * hb - 8.0f * e, 0.0f))) * 0.5f);
                k = max(0, min(k, half - 1));
                while (k > 0 && k * half - k * (k - 1) / 2 > e) --k;
                while (k + 1 < half && (k + 1) * half - (k + 1) * k / 2 <= e) ++k;
                const int k2 = k + (e - (k * half - k * (k - 1) / 2));
                const int p = rp[k], q = rq[k], p2 = rp[k2], q2 = rq[k2];
                const float s = rs[k], s2 = rs[k2];
                if (s == 0.0f && s2 == 0.0f) continue;
                if (k == k2) {
                    // the rotated pair: a_pp - t a_pq, a_qq + t a_pq, a_pq -> 0
                    const float apq = A[p * ld + q], t = rt[k];
                    A[p * ld + p] = A[p * ld + p] - t * apq;
                    A[q * ld + q] = A[q * ld + q] + t * apq;
                    A[p * ld + q] = 0.0f;
                    A[q * ld + p] = 0.0f;
                    continue;
                }
                // Rutishauser's form x' = x - s (y + tau x), y' = y + s (x - tau y)
                // with tau = s / (1 + c): orthogonal to second order even when
                // c rounds to 1
                const float ta = rtau[k], ta2 = rtau[k2];
                const float b00 = A[p * ld + p2], b01 = A[p * ld + q2];
                const float b10 = A[q * ld + p2], b11 = A[q * ld + q2];
                // R_k^T B : rows (p, q)
                const float t00 = b00 - s * (b10 + ta * b00), t01 = b01 - s * (b11 + ta * b01);
                const float t10 = b10 + s * (b00 - ta * b10), t11 = b11 + s * (b01 - ta * b11);
                // (R_k^T B) R_k' : columns (p2, q2)
                const float n00 = t00 - s2 * (t01 + ta2 * t00), n01 = t01 + s2 * (t00 - ta2 * t01);
                const float n10 = t10 - s2 * (t11 + ta2 * t10), n11 = t11 + s2 * (t10 - ta2 * t11);
                A[p * ld + p2] = n00; A[p2 * ld + p] = n00;
                A[p * ld + q2] = n01; A[q2 * ld + p] = n01;
                A[q * ld + p2] = n10; A[p2 * ld + q] = n10;
                A[q * ld + q2] = n11; A[q2 * ld + q] = n11;
            }
            const int vq = mm >> 2;  // float4 per V^T row (mm is a multiple of 4 or 2)
            if ((mm & 3) == 0) {
                for (int e = tid; e < half * vq; e += NT) {
                    const int k = e / vq, j = e - (e / vq) * vq;
                    const float s = rs[k], ta = rtau[k];
                    if (s == 0.0f) continue;
                    float4 *vp = reinterpret_cast<float4 *>(Vt + rp[k] * ldv) + j;
                    float4 *vq4 = reinterpret_cast<float4 *>(Vt + rq[k] * ldv) + j;
                    const float4 x = *vp, y = *vq4;
                    *vp = make_float4(x.x - s * (y.x + ta * x.x), x.y - s * (y.y + ta * x.y),
                                      x.z - s * (y.z + ta * x.z), x.w - s * (y.w + ta * x.w));
                    *vq4 = make_float4(y.x + s * (x.x - ta * y.x), y.y + s * (x.y - ta * y.y),
                                       y.z + s * (x.z - ta * y.z), y.w + s * (x.w - ta * y.w));
                }
            } else {
                for (int e = tid; e < half * mm; e += NT) {
                    const int k = e / mm, j = e - (e / mm) * mm;
                    const float s = rs[k], ta = rtau[k];
                    if (s == 0.0f) continue;
                    const float x = Vt[rp[k] * ldv + j], y = Vt[rq[k] * ldv + j];
                    Vt[rp[k] * ldv + j] = x - s * (y + ta * x);
                    Vt[rq[k] * ldv + j] = y + s * (x - ta * y);
                }
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
    // column col of V is row col of V^T
    for (int e = tid; e < m * m; e += NT) {
        const int row = e % m, col = e / m;
        Vout[(int64_t)s_rank[col] * m + row] = Vt[col * ldv + row];
    }
    for (int i = tid; i < m; i += NT) dout[s_rank[i]] = (double)A[i * ld + i];
}

__global__ void __launch_bounds__(NT, 1)
eig_kernel(const double *__restrict__ C, int m, float *__restrict__ Vout,
           double *__restrict__ dout, float *gA, float *gV, int smem_A, int smem_V,
           int *d_status, const int *only_if)
{
    eig_body(C, m, Vout, dout, gA, gV, smem_A, smem_V, d_status, only_if);
}

// many problems in one launch: block b solves entry b, with both matrices in
// shared memory (m <= 128); fallback: only where the entry's tridiagonal
// solver flagged a failure
__global__ void __launch_bounds__(NT, 1)
eig_grouped_kernel(const psd_g_eig *__restrict__ tab, int *d_status, int fallback)
{
    const psd_g_eig a = tab[blockIdx.x];
    eig_body(a.C, a.m, a.V, a.d, a.scr, a.scr, 1, 1, d_status, fallback ? a.d_fail : nullptr);
}

}  // namespace

cudaError_t launch_eig(cudaStream_t s, const double *C, int m, float *V, double *d,
                       float *scratch, int *d_status, int method, int *d_flag, const float *Cdf)
{
    const int *only_if = nullptr;
    if (method != PSDPROJ_EIG_JACOBI) {
        cudaError_t e = launch_eig_tridiag(s, C, m, V, d, scratch, d_flag,
                                           method == PSDPROJ_EIG_TRIDIAG ? d_status : nullptr, Cdf);
        if (e != cudaSuccess || method == PSDPROJ_EIG_TRIDIAG) return e;
        only_if = d_flag;
    }
    const int mm = m + (m & 1);
    const size_t matA = sizeof(float) * (((size_t)mm * (mm + 1) + 3) & ~(size_t)3);
    const size_t matV = sizeof(float) * (size_t)mm * (mm + 4);
    int smem_A = 1, smem_V = 1;
    size_t smem = matA + matV;
    if (smem > 200 * 1024) { smem_V = 0; smem = matA; }
    if (smem > 200 * 1024) { smem_A = 0; smem = 0; }
    float *gA = scratch;
    float *gV = scratch + matA / sizeof(float);
    // process-wide attribute: the largest size this launcher uses (200 KB)
    cudaError_t e = cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    eig_kernel<<<1, NT, smem, s>>>(C, m, V, d, gA, gV, smem_A, smem_V, d_status, only_if);
    return cudaGetLastError();
}

cudaError_t launch_eig_grouped(cudaStream_t s, const psd_g_eig *tab, int count, const int2 *bmap_ns, int nb_ns,
                               const int2 *bmap_ray, int nb_ray, int m_max, int *d_status, int method)
{
    if (count < 1 || m_max < 1 || m_max > 128) return cudaErrorInvalidValue;
    if (method != PSDPROJ_EIG_JACOBI) {
        cudaError_t e = launch_eig_tridiag_grouped(s, tab, count, bmap_ns, nb_ns, bmap_ray, nb_ray, m_max,
                                                   method == PSDPROJ_EIG_TRIDIAG ? d_status : nullptr);
        if (e != cudaSuccess || method == PSDPROJ_EIG_TRIDIAG) return e;
    }
    const int mm = m_max + (m_max & 1);
    const size_t matA = sizeof(float) * (((size_t)mm * (mm + 1) + 3) & ~(size_t)3);
    const size_t matV = sizeof(float) * (size_t)mm * (mm + 4);
    cudaError_t e = cudaFuncSetAttribute(eig_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    eig_grouped_kernel<<<(unsigned)count, NT, matA + matV, s>>>(tab, d_status, method == PSDPROJ_EIG_AUTO ? 1 : 0);
    return cudaGetLastError();
}
