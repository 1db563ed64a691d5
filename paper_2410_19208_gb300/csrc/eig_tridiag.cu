// Small symmetric eigensolver of Alg. 2 line 2 / Alg. 3 line 3 ("eig(Q^T X Q)")
// by tridiagonalization, in one thread block, FP32:
//
//   1. Householder reduction C = H T H^T (H = H_0 ... H_{m-3}), column by
//      column on the full matrix in shared memory; the reflector vectors are
//      kept below the subdiagonal.
//   2. Eigenvalues of T by bisection on Sturm counts (the number of negative
//      pivots of the LDL^T factorization of T - x I), four lanes per
//      eigenvalue evaluating four points per step (5-way multisection).
//   3. Eigenvectors of T from the twisted factorization of T - lambda I
//      (forward pivots d+, backward pivots d-, twist index r = argmin
//      |d+_r + d-_r - (d_r - lambda)|, then the two recurrences from r).
//      Eigenvalues closer than 1e-4 ||T|| form a cluster; its members take
//      distinct twist indices and are re-orthogonalised (modified
//      Gram-Schmidt) against the earlier members.
//   4. Back-transformation V = H Z.
//   5. One Newton-Schulz step towards the orthogonal polar factor,
//      V <- V (3I - V^T V)/2: the twisted vectors of neighbouring eigenvalues
//      are orthogonal only to ~eps ||T|| / gap (~1e-5 here); the step makes
//      the error quadratic (~1e-10) and mixes each pair symmetrically, which
//      moves V Lambda_+ V^T by O(eps ||T||) only.  It runs on the sorted
//      output (it commutes with reordering the columns, and leaves the unit
//      columns of removed zero rows alone) in two many-block kernels,
//      ns_gram_kernel (S = (3I - V^T V)/2, the orthogonality check) and
//      ns_apply_kernel (V S).
//   6. The eigenvalues refined in FP64 as Rayleigh quotients v^T C v / v^T v
//      of the final vectors against the FP64 input (eig_rayleigh_kernel).
// Output as the Jacobi solver: V (m x m column-major, orthonormal columns)
// and the eigenvalues, sorted by decreasing eigenvalue.  *d_fail is set to
// 1 when a vector is not finite, a twisted residual is large, or V^T V is
// far from I; the caller then runs the Jacobi solver, which reads the flag.
// Cost is O(m^3) work with O(m) block barriers, against O(m^3) work with
// O(m^2) barriers for cyclic Jacobi.
#include "ctx.h"

namespace {

constexpr int NT = 512;
constexpr int SMEM_M = 128;   // largest m kept in shared memory
constexpr int NBIS = 12;      // 5-way multisection steps: width 2.4e-9 of the start interval

// sum of the NT / 32 = 16 warp partials (four 16-byte loads, tree adds)
__device__ __forceinline__ float sum16(const float *red)
{
    const float4 a = reinterpret_cast<const float4 *>(red)[0], b = reinterpret_cast<const float4 *>(red)[1];
    const float4 c = reinterpret_cast<const float4 *>(red)[2], d = reinterpret_cast<const float4 *>(red)[3];
    return (((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w))) +
           (((c.x + c.y) + (c.z + c.w)) + ((d.x + d.y) + (d.z + d.w)));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// number of eigenvalues of tridiag(d, e) below x (ee = e^2); pivots below
// pivmin (>= 1e-30) in magnitude are replaced by -pivmin, so the fast
// division sees |q| in its accurate range
__device__ __forceinline__ int sturm(const float *d, const float *ee, int m, float x, float pivmin)
{
    float q = d[0] - x;
    int c = q < 0.0f;
    for (int i = 1; i < m; ++i) {
        if (fabsf(q) < pivmin) q = -pivmin;
        q = (d[i] - x) - __fdividef(ee[i - 1], q);
        c += q < 0.0f;
    }
    return c;
}

// twisted eigenvector of T for lambda into z (column stride ldz), using t
// (same stride) as scratch; *gamma_out = |gamma_r| at the twist index r,
// which is returned.
__device__ int twisted_vector(const float *d, const float *e, int m, float lambda, float pivmin,
                              float *z, float *t, int ldz, float *gamma_out)
{
    // forward pivots d+ kept in z
    float dp = d[0] - lambda;
    for (int i = 0; i < m; ++i) {
        if (fabsf(dp) < pivmin) dp = -pivmin;
        z[i * ldz] = dp;
        if (i + 1 < m) dp = (d[i + 1] - lambda) - e[i] * e[i] / dp;
    }
    // backward pivots d-, ratios u- kept in t, twist by the smallest |gamma|
    float dm = d[m - 1] - lambda;
    int r = -1;
    float best = 0.0f;
    for (int i = m - 1; i >= 0; --i) {
        if (fabsf(dm) < pivmin) dm = -pivmin;
        const float g = z[i * ldz] + dm - (d[i] - lambda);
        if (r < 0 || fabsf(g) < best) {
            best = fabsf(g);
            r = i;
        }
        if (i > 0) {
            const float u = e[i - 1] / dm;   // u-_{i-1}
            t[(i - 1) * ldz] = u;
            dm = (d[i - 1] - lambda) - u * e[i - 1];
        }
    }
    if (r < 0) r = 0;
    *gamma_out = best;
    // z_r = 1; downward z_i = -(e_i / d+_i) z_{i+1}; upward z_i = -u-_{i-1} z_{i-1}
    float zi = 1.0f;
    for (int i = r - 1; i >= 0; --i) {
        zi = -(e[i] / z[i * ldz]) * zi;
        z[i * ldz] = zi;
    }
    zi = 1.0f;
    for (int i = r + 1; i < m; ++i) {
        zi = -t[(i - 1) * ldz] * zi;
        z[i * ldz] = zi;
    }
    z[r * ldz] = 1.0f;
    return r;
}

// pseudo-random value in [-1, 1) for entry i of start vector k (integer hash)
__device__ __forceinline__ float hash_uniform(int i, int k)
{
    uint32_t x = (uint32_t)i * 0x9E3779B1u + (uint32_t)k * 0x85EBCA77u + 0x165667B1u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    x *= 0x297A2D39u;
    x ^= x >> 15;
    return (float)x * 4.656612873e-10f - 1.0f;
}

// One step of inverse iteration x <- (T - lambda I)^{-1} x through
// T - lambda I = L D L^T (pivots below piv in magnitude are replaced by
// -piv), then x scaled to unit 2-norm.  dp (stride ld) holds the pivots.
// The vector is rescaled by 1e-20 whenever an entry passes 1e20, which
// keeps the solve finite for any shift.
__device__ void inverse_step(const float *d, const float *e, int m, float lambda, float piv,
                             float *x, float *dp, int ld)
{
    constexpr float BIG = 1e20f, SMALL = 1e-20f;
    float q = d[0] - lambda;
    for (int i = 0; i < m; ++i) {
        if (fabsf(q) < piv) q = -piv;
        dp[i * ld] = q;
        if (i + 1 < m) q = (d[i + 1] - lambda) - e[i] * e[i] / q;
    }
    // L y = x
    float yp = x[0];
    for (int i = 1; i < m; ++i) {
        float y = x[i * ld] - (e[i - 1] / dp[(i - 1) * ld]) * yp;
        if (fabsf(y) > BIG) {
            for (int j = 0; j < i; ++j) x[j * ld] *= SMALL;
            y *= SMALL;
        }
        x[i * ld] = y;
        yp = y;
    }
    // D L^T x = y
    float xn = x[(m - 1) * ld] / dp[(m - 1) * ld];
    if (fabsf(xn) > BIG) {
        for (int j = 0; j < m - 1; ++j) x[j * ld] *= SMALL;
        xn *= SMALL;
    }
    x[(m - 1) * ld] = xn;
    for (int i = m - 2; i >= 0; --i) {
        float xi = x[i * ld] / dp[i * ld] - (e[i] / dp[i * ld]) * xn;
        if (fabsf(xi) > BIG) {
            for (int j = 0; j < m; ++j) x[j * ld] *= SMALL;
            xi *= SMALL;
        }
        x[i * ld] = xi;
        xn = xi;
    }
    float mx = 0.0f;
    for (int i = 0; i < m; ++i) mx = fmaxf(mx, fabsf(x[i * ld]));
    const float sc = mx > 0.0f ? 1.0f / mx : 1.0f;
    float nrm = 0.0f;
    for (int i = 0; i < m; ++i) {
        const float v = x[i * ld] * sc;
        nrm = fmaf(v, v, nrm);
    }
    const float inv = sc / sqrtf(nrm);
    for (int i = 0; i < m; ++i) x[i * ld] *= inv;
}

__device__ __forceinline__ void eig_tridiag_body(const double *__restrict__ C, int mfull, float *__restrict__ Vout,
                                                 double *__restrict__ dout, float *gscr, int *__restrict__ d_fail,
                                                 int *d_status_on_fail)
{
    extern __shared__ float sm[];
    const bool in_smem = mfull <= SMEM_M;
    const int ld = mfull + 1;
    float *A = in_smem ? sm : gscr;                 // m x ld, row-major
    float *Z = A + mfull * ld;                      // eigenvectors of T (row i, column k)
    float *T = Z + mfull * ld;                      // scratch of the twisted factorization
    __shared__ float d[PSD_MAX_M], e[PSD_MAX_M], ee[PSD_MAX_M], beta[PSD_MAX_M];
    __shared__ float vv[PSD_MAX_M], pp[PSD_MAX_M], lam[PSD_MAX_M];
    __shared__ __align__(16) float red[NT / 32];
    static_assert(NT / 32 == 16, "sum16");
    __shared__ int cl_start[PSD_MAX_M];
    __shared__ int s_pos[PSD_MAX_M], s_src[PSD_MAX_M];
    __shared__ int s_fail, s_mc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_fail = 0;
    }

    for (int e0 = tid; e0 < mfull * mfull; e0 += NT) {
        const int i = e0 / mfull, j = e0 - (e0 / mfull) * mfull;
        A[i * ld + j] = (float)C[(int64_t)j * mfull + i];
    }
    __syncthreads();

    // Rows that are exactly zero (the zeroed dependent columns of Q) carry
    // the eigenvalue 0 with a unit eigenvector; they are taken out and the
    // solver runs on the remaining m x m block, so that these eigenvalues stay
    // exactly 0 and never count as positive.
    for (int i = tid; i < mfull; i += NT) {
        int nz = 0;
        for (int k = 0; k < mfull; ++k) nz |= (A[i * ld + k] != 0.0f);   // NaN counts as nonzero
        s_pos[i] = nz;
    }
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int i = 0; i < mfull; ++i) s_pos[i] = s_pos[i] ? c++ : -1;
        s_mc = c;
    }
    __syncthreads();
    const int m = s_mc;
    if (m < mfull && m > 0) {
        for (int e0 = tid; e0 < mfull * mfull; e0 += NT) {
            const int i = e0 / mfull, k = e0 - (e0 / mfull) * mfull;
            const int pi = s_pos[i], pk = s_pos[k];
            if (pi >= 0 && pk >= 0) Z[pi * ld + pk] = A[i * ld + k];
        }
        __syncthreads();
        for (int e0 = tid; e0 < m * m; e0 += NT) {
            const int i = e0 / m, k = e0 - (e0 / m) * m;
            A[i * ld + k] = Z[i * ld + k];
        }
        __syncthreads();
    }
    if (m > 0) {
    // ---------------------------------------------------------------- 1
    if (m <= SMEM_M) {
        // The trailing matrix in registers: lane l of warp w holds rows
        // 8 (l % 16) .. + 7, columns 8 w + 4 (l / 16) .. + 3 (zero past m),
        // so a half-warp holds four whole columns.  Step j: the warp owning
        // column j forms the reflector v (zero outside rows >= j + 1) and
        // beta from its own registers; p = beta A v comes from column sums
        // (A is symmetric) reduced over each half-warp; K = beta v^T p / 2 and
        // w = p - K v; the rank-2 update A -= v w^T + w v^T touches only the
        // registers, and the next column's warp can start at once.  v and p
        // are zero outside the trailing block, so finished rows and columns
        // are left alone.  Two barriers per step.
        __shared__ __align__(16) float vq[SMEM_M], pq[SMEM_M];
        __shared__ __align__(16) float rq[NT / 32];
        __shared__ float s_bt;
        const int rb = 8 * (lane & 15), cb = 8 * warp + 4 * (lane >> 4);
        float a[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = rb + r, k = cb + c;
                a[r][c] = (i < m && k < m) ? A[i * ld + k] : 0.0f;
            }
        for (int j = 0; j + 2 < m; ++j) {
            const int r0 = j + 1;
            // (A) the reflector, from column j in its warp's registers (the
            // half-warp holding it; the other half contributes zeros)
            if (warp == (j >> 3)) {
                const bool mine = (lane >> 4) == ((j >> 2) & 1);
                const int cj = j & 3;
                float x[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    x[r] = a[r][0];
#pragma unroll
                    for (int c = 1; c < 4; ++c)
                        if (cj == c) x[r] = a[r][c];
                    if (!mine) x[r] = 0.0f;
                }
                float part = 0.0f;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int i = rb + r;
                    if (i > r0 && i < m) part = fmaf(x[r], x[r], part);
                }
                const float tail = warp_sum(part);
                float x0l = x[0], xjl = x[0];
#pragma unroll
                for (int r = 1; r < 8; ++r) {
                    if ((r0 & 7) == r) x0l = x[r];
                    if ((j & 7) == r) xjl = x[r];
                }
                const int hsrc = 16 * ((j >> 2) & 1);
                const float x0 = __shfl_sync(0xffffffffu, x0l, hsrc + (r0 >> 3));
                const float xj = __shfl_sync(0xffffffffu, xjl, hsrc + (j >> 3));
                const bool skip = !(tail > 0.0f);           // column already tridiagonal
                const float sigma = sqrtf(fmaf(x0, x0, tail));
                const float alpha = -copysignf(sigma, x0);
                const float bt = skip ? 0.0f : 1.0f / (sigma * sigma - alpha * x0);
                if (mine) {
                    float vv8[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const int i = rb + r;
                        const float v = (i < r0 || i >= m || skip) ? 0.0f : (i == r0 ? x0 - alpha : x[r]);
                        vv8[r] = v;
                        if (i >= r0 && i < m) A[i * ld + j] = v;   // kept for the back-transformation
                    }
                    *reinterpret_cast<float4 *>(vq + rb) = make_float4(vv8[0], vv8[1], vv8[2], vv8[3]);
                    *reinterpret_cast<float4 *>(vq + rb + 4) = make_float4(vv8[4], vv8[5], vv8[6], vv8[7]);
                }
                if (lane == 0) {
                    d[j] = xj;
                    e[j] = skip ? x0 : alpha;
                    beta[j] = bt;
                    s_bt = bt;
                }
            }
            __syncthreads();
            // (B) p = beta A v from column sums over each half-warp; the warp's part of v^T p.
            // A warp whose columns are all finished (< r0) has p = w = 0 there
            // and nothing to update: it only writes its zeros.
            const bool live = 8 * warp + 7 >= r0;
            const float bt = s_bt;
            const float4 vr0 = *reinterpret_cast<const float4 *>(vq + rb);
            const float4 vr1 = *reinterpret_cast<const float4 *>(vq + rb + 4);
            const float4 vc4 = *reinterpret_cast<const float4 *>(vq + cb);
            const float vr[8] = {vr0.x, vr0.y, vr0.z, vr0.w, vr1.x, vr1.y, vr1.z, vr1.w};
            const float vc[4] = {vc4.x, vc4.y, vc4.z, vc4.w};
            float pc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (live) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float t0 = fmaf(a[0][c], vr[0], fmaf(a[1][c], vr[1], fmaf(a[2][c], vr[2], a[3][c] * vr[3])));
                    const float t1 = fmaf(a[4][c], vr[4], fmaf(a[5][c], vr[5], fmaf(a[6][c], vr[6], a[7][c] * vr[7])));
                    pc[c] = t0 + t1;
                }
#pragma unroll
                for (int o = 1; o < 16; o <<= 1)
#pragma unroll
                    for (int c = 0; c < 4; ++c) pc[c] += __shfl_xor_sync(0xffffffffu, pc[c], o);
            }
            float vtp = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int k = cb + c;
                pc[c] = (k >= r0 && k < m) ? bt * pc[c] : 0.0f;
                vtp = fmaf(vc[c], pc[c], vtp);
            }
            vtp += __shfl_xor_sync(0xffffffffu, vtp, 16);
            if ((lane & 15) == 0) *reinterpret_cast<float4 *>(pq + cb) = make_float4(pc[0], pc[1], pc[2], pc[3]);
            if (lane == 0) rq[warp] = vtp;
            __syncthreads();
            // (C) K and w, then the rank-2 update of the registers
            if (!live) continue;
            float vt = 0.0f;
#pragma unroll
            for (int q = 0; q < NT / 32; q += 4) {
                const float4 t = *reinterpret_cast<const float4 *>(rq + q);
                vt += (t.x + t.y) + (t.z + t.w);
            }
            const float K = 0.5f * bt * vt;
            const float4 pr0 = *reinterpret_cast<const float4 *>(pq + rb);
            const float4 pr1 = *reinterpret_cast<const float4 *>(pq + rb + 4);
            const float pr[8] = {pr0.x, pr0.y, pr0.z, pr0.w, pr1.x, pr1.y, pr1.z, pr1.w};
            float wc[4], wr[8];
#pragma unroll
            for (int c = 0; c < 4; ++c) wc[c] = fmaf(-K, vc[c], pc[c]);
#pragma unroll
            for (int r = 0; r < 8; ++r) wr[r] = fmaf(-K, vr[r], pr[r]);
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    a[r][c] = fmaf(-vr[r], wc[c], a[r][c]);
                    a[r][c] = fmaf(-wr[r], vc[c], a[r][c]);
                }
        }
        // the last 2 x 2 block of T
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = rb + r, k = cb + c;
                if (m >= 2 && i == m - 2 && k == m - 2) d[m - 2] = a[r][c];
                if (m >= 2 && i == m - 1 && k == m - 2) e[m - 2] = a[r][c];
                if (i == m - 1 && k == m - 1) d[m - 1] = a[r][c];
            }
        if (tid == 0) {
            if (m >= 2) beta[m - 2] = 0.0f;
            e[m - 1] = 0.0f;
            beta[m - 1] = 0.0f;
        }
        __syncthreads();
    } else {
        for (int j = 0; j + 2 < m; ++j) {
            const int r0 = j + 1;                       // first row of the trailing block
            // squared norm of x = A[r0.., j] below its first entry
            float part = 0.0f;
            for (int i = r0 + 1 + tid; i < m; i += NT) part = fmaf(A[i * ld + j], A[i * ld + j], part);
            part = warp_sum(part);
            if (lane == 0) red[warp] = part;
            __syncthreads();
            const float tail = sum16(red);
            const float x0 = A[r0 * ld + j];
            const bool skip = !(tail > 0.0f);           // column already tridiagonal
            const float sigma = sqrtf(fmaf(x0, x0, tail));
            const float alpha = -copysignf(sigma, x0);
            const float bt = skip ? 0.0f : 1.0f / (sigma * sigma - alpha * x0);
            for (int i = r0 + tid; i < m; i += NT) vv[i] = (i == r0) ? (x0 - alpha) : A[i * ld + j];
            if (tid == 0) {
                d[j] = A[j * ld + j];
                e[j] = skip ? x0 : alpha;
                beta[j] = bt;
            }
            __syncthreads();                            // vv ready; red reusable
            if (skip) {
                // keep a zero reflector below the subdiagonal
                for (int i = r0 + tid; i < m; i += NT) A[i * ld + j] = 0.0f;
                __syncthreads();
                continue;
            }
            // p = bt A22 v (four lanes per row, lane q summing the columns
            // k = r0 + q mod 4; the row loop's trip count is the same for every
            // thread, so the shuffles see full warps) and v^T p
            float pv = 0.0f;
            for (int base = r0; base < m; base += NT / 4) {
                const int i = base + (tid >> 2), q = tid & 3;
                float s0 = 0.0f, s1 = 0.0f;
                if (i < m) {
                    const float *row = A + i * ld;
                    int k = r0 + q;
                    for (; k + 4 < m; k += 8) {
                        s0 = fmaf(row[k], vv[k], s0);
                        s1 = fmaf(row[k + 4], vv[k + 4], s1);
                    }
                    if (k < m) s0 = fmaf(row[k], vv[k], s0);
                }
                s0 += s1;
                s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
                s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
                if (i < m && q == 0) {
                    const float p = bt * s0;
                    pp[i] = p;
                    pv = fmaf(p, vv[i], pv);
                }
            }
            pv = warp_sum(pv);
            if (lane == 0) red[warp] = pv;
            __syncthreads();
            const float vtp = sum16(red);
            const float K = 0.5f * bt * vtp;
            // A22 -= v w^T + w v^T with w = p - K v (rows by warp, columns by
            // lane); the reflector goes below the subdiagonal
            for (int i = r0 + warp; i < m; i += NT / 32) {
                const float vi = vv[i], wi = pp[i] - K * vv[i];
                float *row = A + i * ld;
                for (int k = r0 + lane; k < m; k += 32) {
                    const float wk = pp[k] - K * vv[k];
                    row[k] -= vi * wk + wi * vv[k];
                }
            }
            for (int i = r0 + tid; i < m; i += NT) A[i * ld + j] = vv[i];
            __syncthreads();
        }
        if (tid == 0) {
            if (m >= 2) {
                d[m - 2] = A[(m - 2) * ld + (m - 2)];
                e[m - 2] = A[(m - 1) * ld + (m - 2)];
                beta[m - 2] = 0.0f;
            }
            d[m - 1] = A[(m - 1) * ld + (m - 1)];
            e[m - 1] = 0.0f;
            beta[m - 1] = 0.0f;
        }
        __syncthreads();


    }
    // ---------------------------------------------------------------- 2
    __shared__ float s_gl, s_gu, s_pivmin, s_tnorm;
    if (tid == 0) {
        float gl = 3.0e38f, gu = -3.0e38f, emax = 0.0f;
        for (int i = 0; i < m; ++i) {
            const float r = (i > 0 ? fabsf(e[i - 1]) : 0.0f) + (i + 1 < m ? fabsf(e[i]) : 0.0f);
            gl = fminf(gl, d[i] - r);
            gu = fmaxf(gu, d[i] + r);
            if (i + 1 < m) emax = fmaxf(emax, e[i] * e[i]);
        }
        const float tn = fmaxf(fabsf(gl), fabsf(gu));
        const float pad = 2.0f * 1.2e-7f * tn + 1e-30f;
        s_gl = gl - pad;
        s_gu = gu + pad;
        s_tnorm = tn;
        s_pivmin = fmaxf(1e-30f, 1e-30f * emax);
    }
    for (int i = tid; i < m; i += NT) ee[i] = (i + 1 < m) ? e[i] * e[i] : 0.0f;
    __syncthreads();
    const float pivmin = s_pivmin;
    for (int base = 0; base < m; base += NT / 4) {
        const int k = base + (tid >> 2);            // eigenvalue index (ascending)
        const int sub = tid & 3;
        float lo = s_gl, hi = s_gu;
        for (int it = 0; it < NBIS; ++it) {
            const float x = lo + (hi - lo) * (float)(sub + 1) * 0.2f;
            const int c = (k < m) ? sturm(d, ee, m, x, pivmin) : 0;
            // new interval: [largest x with count <= k, smallest x with count > k]
            const unsigned lmask = 0xFu << (lane & ~3);
            const unsigned below = __ballot_sync(0xffffffffu, c <= k) & lmask;
            const int nb = __popc(below);           // points at or below lambda_k
            const float nlo = nb > 0 ? lo + (hi - lo) * (float)nb * 0.2f : lo;
            const float nhi = nb < 4 ? lo + (hi - lo) * (float)(nb + 1) * 0.2f : hi;
            lo = nlo;
            hi = nhi;
        }
        if (k < m && sub == 0) lam[k] = 0.5f * (lo + hi);
    }
    __syncthreads();

    // ---------------------------------------------------------------- 3
    // clusters: runs of eigenvalues closer than 1e-4 ||T||
    const float ctol = 1e-4f * s_tnorm + 1e-30f;
    const float pivsolve = fmaxf(1.2e-7f * s_tnorm, 1e-30f);
    for (int k = tid; k < m; k += NT) {
        int s = k;
        while (s > 0 && lam[s] - lam[s - 1] <= ctol) --s;
        cl_start[k] = s;
    }
    __syncthreads();
    // isolated eigenvalues: twisted factorization, one thread each;
    // cluster members: pseudo-random start vectors
    for (int k = tid; k < m; k += NT) {
        float *z = Z + k, *t = T + k;
        const bool single = cl_start[k] == k && !(k + 1 < m && cl_start[k + 1] == k);
        if (!single) {
            for (int i = 0; i < m; ++i) z[i * ld] = hash_uniform(i, k);
            continue;
        }
        float gam;
        twisted_vector(d, e, m, lam[k], pivmin, z, t, ld, &gam);
        float nrm = 0.0f;
        for (int i = 0; i < m; ++i) nrm = fmaf(z[i * ld], z[i * ld], nrm);
        const float inv = 1.0f / sqrtf(nrm);
        for (int i = 0; i < m; ++i) z[i * ld] *= inv;
        // ||(T - lambda I) z|| = |gamma_r| / ||z|| for the twisted solution
        if (!(nrm >= 1.0f && isfinite(nrm)) || !(gam * inv <= 1e-3f * s_tnorm + 1e-20f)) s_fail = 1;
    }
    __syncthreads();
    // clusters, one warp each: two steps of inverse iteration, each member
    // with its own shift (lanes in parallel), then modified Gram-Schmidt
    // over the members in order (the warp together): subspace iteration
    // onto the cluster's invariant subspace
    {
        int cid = 0;
        for (int s = 0; s < m; ++s) {
            if (cl_start[s] != s) continue;
            int g = 1;
            while (s + g < m && cl_start[s + g] == s) ++g;
            if (g == 1) continue;
            if ((cid++ % (NT / 32)) != warp) continue;
            for (int it = 0; it < 2; ++it) {
                for (int k = s + lane; k < s + g; k += 32)
                    inverse_step(d, e, m, lam[k], pivsolve, Z + k, T + k, ld);
                __syncwarp();
                for (int k = s; k < s + g; ++k) {
                    float *z = Z + k;
                    for (int pass = 0; pass < 2; ++pass) {
                        for (int o = s; o < k; ++o) {
                            float dot = 0.0f;
                            for (int i = lane; i < m; i += 32) dot = fmaf(Z[i * ld + o], z[i * ld], dot);
                            dot = warp_sum(dot);
                            for (int i = lane; i < m; i += 32) z[i * ld] = fmaf(-dot, Z[i * ld + o], z[i * ld]);
                            __syncwarp();
                        }
                    }
                    float nrm = 0.0f;
                    for (int i = lane; i < m; i += 32) nrm = fmaf(z[i * ld], z[i * ld], nrm);
                    nrm = warp_sum(nrm);
                    const float inv = 1.0f / sqrtf(nrm);
                    for (int i = lane; i < m; i += 32) z[i * ld] *= inv;
                    __syncwarp();
                }
            }
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- 4
    // Z <- H_0 H_1 ... H_{m-3} Z in blocks of NB reflectors, last block
    // first, each block in compact WY form H_jb ... H_{jb+nb-1} = I - V T V^T
    // (V: the block's reflector vectors A[i][jb+t], i > jb+t):
    // Z <- Z - V (T (V^T Z)).  T is never formed: T^-1 is the upper
    // triangular matrix with diagonal 1 / beta_t and strictly upper part
    // V^T V, so T W solves T^-1 Y = W by back substitution, a column of W per
    // thread (a zero beta, a skipped reflector, gives a zero row of Y).
    // W = V^T Z and then Y live in the first nb rows of the T buffer.
    {
        constexpr int NB = 16;
        __shared__ float sS[NB][NB + 1];
        const int nref = m - 2;                               // reflectors 0 .. m-3
        for (int jb = nref > 0 ? ((nref - 1) / NB) * NB : -1; jb >= 0; jb -= NB) {
            const int nb = min(NB, nref - jb);
            // (a) W[t][c] = v_t^T Z[:, c] (v_t lives in rows > jb + t of column
            // jb + t), four reflectors per thread so that each Z entry read
            // serves four products; and S[s][t] = v_s^T v_t (s < t)
            for (int q = tid; q < 4 * m; q += NT) {
                const int tg = q / m, c = q - (q / m) * m;
                const int t0 = 4 * tg, col0 = jb + t0;
                if (t0 >= nb) continue;
                float w[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                int i = col0 + 1;
                for (; i < m && i < col0 + 4; ++i) {           // the first rows, where some v_t start
                    const float z = Z[i * ld + c];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (t0 + u < nb && i > col0 + u) w[u] = fmaf(A[i * ld + col0 + u], z, w[u]);
                }
                const int nu = min(4, nb - t0);                  // reflectors of this group
                for (; i < m; ++i) {
                    const float z = Z[i * ld + c];
                    const float *ar = A + i * ld + col0;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (u < nu) w[u] = fmaf(ar[u], z, w[u]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (t0 + u < nb) T[(t0 + u) * ld + c] = w[u];
            }
            for (int q = tid; q < nb * nb; q += NT) {
                const int sI = q / nb, tI = q - (q / nb) * nb;
                if (sI < tI) {
                    float acc = 0.0f;
                    for (int i = jb + tI + 1; i < m; ++i) acc = fmaf(A[i * ld + jb + sI], A[i * ld + jb + tI], acc);
                    sS[sI][tI] = acc;
                }
            }
            __syncthreads();
            // (b) Y = T W: T^-1 Y = W, back substitution down the nb rows,
            // a thread per column
            for (int c = tid; c < m; c += NT) {
                float w[NB];
#pragma unroll
                for (int t = 0; t < NB; ++t) w[t] = t < nb ? T[t * ld + c] : 0.0f;
#pragma unroll
                for (int t = NB - 1; t >= 0; --t) {
                    if (t >= nb) continue;
                    const float bt = beta[jb + t];
                    float acc = w[t];
#pragma unroll
                    for (int u = t + 1; u < NB; ++u)
                        if (u < nb) acc = fmaf(-sS[t][u], w[u], acc);
                    w[t] = bt * acc;        // divided by the diagonal 1 / beta_t
                }
#pragma unroll
                for (int t = 0; t < NB; ++t)
                    if (t < nb) T[t * ld + c] = w[t];
            }
            __syncthreads();
            // (d) Z[i][c] -= sum_t V[i][t] W[t][c], rows i > jb (a warp per row);
            // a lane keeps W of its four columns (c = cb + lane + 32 k) in
            // registers over all of its warp's rows
            for (int cb = 0; cb < m; cb += 128) {
                float wr[4][NB];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = cb + lane + 32 * k;
#pragma unroll
                    for (int t = 0; t < NB; ++t) wr[k][t] = (c < m && t < nb) ? T[t * ld + c] : 0.0f;
                }
                for (int i = jb + 1 + warp; i < m; i += NT / 32) {
                    float v[NB];
#pragma unroll
                    for (int t = 0; t < NB; ++t) v[t] = (t < nb && i > jb + t) ? A[i * ld + jb + t] : 0.0f;
                    float *zr = Z + i * ld;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int c = cb + lane + 32 * k;
                        if (c < m) {
                            float acc = zr[c];
#pragma unroll
                            for (int t = 0; t < NB; ++t) acc = fmaf(-v[t], wr[k][t], acc);
                            zr[c] = acc;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }

    // ---------------------------------------------------------------- 5
    // the Newton-Schulz step runs after the output, in ns_gram_kernel and
    // ns_apply_kernel (many blocks; it commutes with the column ordering)

    }  // m > 0

    // Output in decreasing order: the positive eigenvalues of the block, the
    // exact zeros of the removed rows, then the rest of the block (lam is
    // ascending).  s_src[position] = block index k, or -(i+1) for removed row i.
    if (tid == 0) {
        int bad = s_fail;
        int npos = 0;
        for (int k = 0; k < m; ++k) {
            bad |= !isfinite(lam[k]);
            npos += lam[k] > 0.0f;
        }
        *d_fail = bad;
        if (bad && d_status_on_fail) psd_set_status(d_status_on_fail, PSDPROJ_ENOCONV);
        const int ndead = mfull - m;
        for (int k = 0; k < m; ++k) s_src[lam[k] > 0.0f ? (m - 1 - k) : (m - 1 - k + ndead)] = k;
        int t = 0;
        for (int i = 0; i < mfull; ++i)
            if (s_pos[i] < 0) s_src[npos + t++] = -(i + 1);
    }
    __syncthreads();
    for (int e0 = tid; e0 < mfull * mfull; e0 += NT) {
        const int row = e0 % mfull, col = e0 / mfull;
        const int src = s_src[col];
        float v;
        if (src >= 0) v = s_pos[row] >= 0 ? Z[s_pos[row] * ld + src] : 0.0f;
        else v = (row == -src - 1) ? 1.0f : 0.0f;
        Vout[(int64_t)col * mfull + row] = v;
    }
    for (int col = tid; col < mfull; col += NT) {
        const int src = s_src[col];
        dout[col] = src >= 0 ? (double)lam[src] : 0.0;
    }
}

__global__ void __launch_bounds__(NT, 1)
eig_tridiag_kernel(const double *__restrict__ C, int mfull, float *__restrict__ Vout,
                   double *__restrict__ dout, float *gscr, int *__restrict__ d_fail,
                   int *d_status_on_fail)
{
    eig_tridiag_body(C, mfull, Vout, dout, gscr, d_fail, d_status_on_fail);
}

// many problems in one launch: block b solves entry b (m <= SMEM_M), two
// blocks per SM
__global__ void __launch_bounds__(NT, 2)
eig_tridiag_grouped_kernel(const psd_g_eig *__restrict__ tab, int *d_status_on_fail)
{
    const psd_g_eig a = tab[blockIdx.x];
    eig_tridiag_body(a.C, a.m, a.V, a.d, a.scr, a.d_fail, d_status_on_fail);
}

}  // namespace

namespace {

// V (m x m, column-major): S = (3I - V^T V)/2 and a copy of V (blocks of the
// first block column), both m x m column-major; a block of 16 x 16 entries of
// V^T V per 256 threads, columns staged 32 rows at a time.  V^T V further than
// 1e-2 from I (or not finite) fails the solver: *d_fail = 1 and, when asked,
// ENOCONV.
__device__ __forceinline__ void ns_gram_body(const float *__restrict__ V, int m, float *__restrict__ S,
                                             float *__restrict__ Vc, int *d_fail, int *d_status_on_fail, int bx,
                                             int by)
{
    __shared__ float Va[32][17], Vb[32][17];
    __shared__ float s_dev[8];
    const int a0 = bx * 16, b0 = by * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc = 0.0f;
    for (int r0 = 0; r0 < m; r0 += 32) {
        for (int e = threadIdx.x; e < 512; e += 256) {
            const int c = e >> 5, r = e & 31;
            const bool okr = r0 + r < m;
            const float va = (okr && a0 + c < m) ? V[(int64_t)(a0 + c) * m + r0 + r] : 0.0f;
            Va[r][c] = va;
            Vb[r][c] = (okr && b0 + c < m) ? V[(int64_t)(b0 + c) * m + r0 + r] : 0.0f;
            if (by == 0 && okr && a0 + c < m) Vc[(int64_t)(a0 + c) * m + r0 + r] = va;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) acc = fmaf(Va[r][ty], Vb[r][tx], acc);
        __syncthreads();
    }
    const int a = a0 + ty, b = b0 + tx;
    float dev = 0.0f;
    if (a < m && b < m) {
        const float g = acc - (a == b ? 1.0f : 0.0f);
        dev = isfinite(g) ? fabsf(g) : 3.0e38f;
        S[(int64_t)b * m + a] = (a == b ? 1.0f : 0.0f) - 0.5f * g;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if ((threadIdx.x & 31) == 0) s_dev[threadIdx.x >> 5] = dev;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mx = 0.0f;
        for (int w = 0; w < 8; ++w) mx = fmaxf(mx, s_dev[w]);
        if (!(mx <= 1e-2f)) {
            *d_fail = 1;
            if (d_status_on_fail) psd_set_status(d_status_on_fail, PSDPROJ_ENOCONV);
        }
    }
}

__global__ void __launch_bounds__(256)
ns_gram_kernel(const float *__restrict__ V, int m, float *__restrict__ S, float *__restrict__ Vc, int *d_fail,
               int *d_status_on_fail)
{
    ns_gram_body(V, m, S, Vc, d_fail, d_status_on_fail, blockIdx.x, blockIdx.y);
}

// the scratch of entry a: S, then the copy of V (as launch_eig_tridiag)
__global__ void __launch_bounds__(256)
ns_gram_grouped_kernel(const psd_g_eig *__restrict__ tab, const int2 *__restrict__ bmap, int *d_status_on_fail)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_eig a = tab[b.x];
    const int g = (a.m + 15) / 16;
    ns_gram_body(a.V, a.m, a.scr, a.scr + (size_t)a.m * a.m, a.d_fail, d_status_on_fail, b.y % g, b.y / g);
}

// Vout = V S (m x m, column-major): a block of 16 x 16 entries per 256 threads
__device__ __forceinline__ void ns_apply_body(const float *__restrict__ V, const float *__restrict__ S, int m,
                                              float *__restrict__ Vout, int bx, int by)
{
    __shared__ float Vr[16][33], Sc[32][17];
    const int r0 = bx * 16, c0 = by * 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc = 0.0f;
    for (int k0 = 0; k0 < m; k0 += 32) {
        for (int e = threadIdx.x; e < 512; e += 256) {
            const int k = e >> 4, r = e & 15;                 // V(r0 + r, k0 + k)
            Vr[r][k] = (r0 + r < m && k0 + k < m) ? V[(int64_t)(k0 + k) * m + r0 + r] : 0.0f;
            const int kk = e & 31, c = e >> 5;                // S(k0 + kk, c0 + c)
            Sc[kk][c] = (k0 + kk < m && c0 + c < m) ? S[(int64_t)(c0 + c) * m + k0 + kk] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) acc = fmaf(Vr[tx][k], Sc[k][ty], acc);
        __syncthreads();
    }
    const int r = r0 + tx, c = c0 + ty;
    if (r < m && c < m) Vout[(int64_t)c * m + r] = acc;
}

__global__ void __launch_bounds__(256)
ns_apply_kernel(const float *__restrict__ V, const float *__restrict__ S, int m, float *__restrict__ Vout)
{
    ns_apply_body(V, S, m, Vout, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(256)
ns_apply_grouped_kernel(const psd_g_eig *__restrict__ tab, const int2 *__restrict__ bmap)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_eig a = tab[b.x];
    const int g = (a.m + 15) / 16;
    ns_apply_body(a.scr + (size_t)a.m * a.m, a.scr, a.m, a.V, b.y % g, b.y / g);
}

// d_i <- v_i^T C v_i / v_i^T v_i in FP64: the Rayleigh quotient of the computed
// eigenvector against the FP64 core matrix, whose error is quadratic in the
// vector's (FP32 vectors orthonormal to ~1e-7 give eigenvalues to ~1e-14
// ||C||).  Where the quotient and the FP32 eigenvalue disagree in sign the
// eigenvalue is indistinguishable from zero at FP32 accuracy: 0.  Exact
// zeros (the removed zero rows) stay zero.  One block per eigenpair.
// the quotient's use: the FP64 value where it agrees in sign with the
// solver's eigenvalue l0 (exact zeros kept), else 0
__device__ __forceinline__ double rayleigh_update(double num, double den, double l0)
{
    const double q = den > 0.0 ? num / den : 0.0;
    return (l0 == 0.0 || !isfinite(q)) ? l0 : ((q > 0.0) == (l0 > 0.0) ? q : 0.0);
}

// (C v)_r = sum_c C(r, c) v_c with C as double-float pairs (hi, lo), the form
// the core's Gram reduction sums in: a compensated dot product in FP32
// arithmetic (Dot2 of Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005: each high product split exactly by FMA, the errors summed
// beside the sum), as accurate as FP64 here and without this GPU's slow FP64
// pipe.  Cd(r, c) = cd[c * ldc + r]; v in shared or global memory.
__device__ __forceinline__ double cv_dot2(const float2 *cd, int ldc, const float *v, int m, int r)
{
    float sh = 0.0f, sl = 0.0f;
    for (int c = 0; c < m; ++c) {
        const float2 cc = cd[c * ldc + r];
        const float vc = v[c];
        const float ph = cc.x * vc;
        const float pe = fmaf(cc.x, vc, -ph) + cc.y * vc;
        const float t = sh + ph;                     // two_sum(sh, ph)
        const float bv = t - sh;
        sl += ((sh - (t - bv)) + (ph - bv)) + pe;
        sh = t;
    }
    return (double)sh + (double)sl;
}

// Cd (may be NULL): C also as double-float pairs, from which C v is formed
// (cv_dot2); else from the FP64 C.  The quotient itself is FP64.
__device__ __forceinline__ void eig_rayleigh_body(const double *__restrict__ C, const float2 *__restrict__ Cd,
                                                  const float *__restrict__ V, int m, double *__restrict__ d, int i)
{
    __shared__ double s_red[2][8];
    const float *v = V + (int64_t)i * m;
    double acc = 0.0, nn = 0.0;              // v^T C v and v^T v
    for (int r = threadIdx.x; r < m; r += 256) {
        double y = 0.0;
        if (Cd)
            y = cv_dot2(Cd, m, v, m, r);
        else
            for (int c = 0; c < m; ++c) y = fma(C[(int64_t)c * m + r], (double)v[c], y);
        const double vr = (double)v[r];
        acc = fma(vr, y, acc);
        nn = fma(vr, vr, nn);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = acc;
        s_red[1][threadIdx.x >> 5] = nn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double num = 0.0, den = 0.0;
        for (int w = 0; w < 8; ++w) {
            num += s_red[0][w];
            den += s_red[1][w];
        }
        d[i] = rayleigh_update(num, den, d[i]);
    }
}

// The same quotients for m <= 128, PSD_RQ eigenpairs per block (group g):
// C (pairs, or FP64) and the group's eigenvectors staged in shared memory
// once, then two eigenpairs at a time, thread r of each half of the block
// forming (C v)_r.  Shared memory: psd_rayleigh_smem(m).
__device__ __forceinline__ void eig_rayleigh_smem_body(const double *__restrict__ C, const float2 *__restrict__ Cd,
                                                       const float *__restrict__ V, int m, double *__restrict__ d,
                                                       int g)
{
    extern __shared__ __align__(16) unsigned char rq_sm[];
    float2 *sCd = reinterpret_cast<float2 *>(rq_sm);
    double *sC = reinterpret_cast<double *>(rq_sm);
    float *sV = reinterpret_cast<float *>(rq_sm + sizeof(double) * (size_t)m * m);
    __shared__ double s_red[8][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = g * PSD_RQ, cnt = min(PSD_RQ, m - i0);
    if (Cd)
        for (int e = tid; e < m * m; e += 256) sCd[e] = Cd[e];
    else
        for (int e = tid; e < m * m; e += 256) sC[e] = C[e];
    for (int e = tid; e < cnt * m; e += 256) sV[e] = V[(int64_t)i0 * m + e];
    __syncthreads();
    const int half = tid >> 7, r = tid & 127;
    for (int j0 = 0; j0 < cnt; j0 += 2) {
        const int j = j0 + half;
        double acc = 0.0, nn = 0.0;
        if (j < cnt && r < m) {
            const float *v = sV + j * m;
            double y = 0.0;
            if (Cd)
                y = cv_dot2(sCd, m, v, m, r);
            else
                for (int c = 0; c < m; ++c) y = fma(sC[c * m + r], (double)v[c], y);
            const double vr = (double)v[r];
            acc = vr * y;
            nn = vr * vr;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            nn += __shfl_xor_sync(0xffffffffu, nn, o);
        }
        if (lane == 0) {
            s_red[warp][0] = acc;
            s_red[warp][1] = nn;
        }
        __syncthreads();
        if (r == 0 && j < cnt) {
            double num = 0.0, den = 0.0;
            for (int w = 4 * half; w < 4 * half + 4; ++w) {
                num += s_red[w][0];
                den += s_red[w][1];
            }
            d[i0 + j] = rayleigh_update(num, den, d[i0 + j]);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
eig_rayleigh_kernel(const double *__restrict__ C, const float2 *__restrict__ Cd, const float *__restrict__ V, int m,
                    double *__restrict__ d)
{
    eig_rayleigh_body(C, Cd, V, m, d, blockIdx.x);
}

__global__ void __launch_bounds__(256)
eig_rayleigh_smem_kernel(const double *__restrict__ C, const float2 *__restrict__ Cd, const float *__restrict__ V,
                         int m, double *__restrict__ d)
{
    eig_rayleigh_smem_body(C, Cd, V, m, d, blockIdx.x);
}

// many problems: block b, group bmap[b].y of entry bmap[b].x (m <= 128)
__global__ void __launch_bounds__(256)
eig_rayleigh_grouped_kernel(const psd_g_eig *__restrict__ tab, const int2 *__restrict__ bmap)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_eig a = tab[b.x];
    eig_rayleigh_smem_body(a.C, a.Cd, a.V, a.m, a.d, b.y);
}

}  // namespace

cudaError_t launch_eig_tridiag(cudaStream_t s, const double *C, int m, float *V, double *d,
                               float *scratch, int *d_fail, int *d_status_on_fail, const float *Cdf)
{
    // three m x (m+1) buffers plus 8 slack rows read (never used) by the
    // edge tiles of the Newton-Schulz products
    const size_t smem = m <= SMEM_M ? sizeof(float) * (3 * (size_t)m + 8) * (m + 1) : 0;
    // process-wide attribute: the largest size (m = SMEM_M) for every launch
    constexpr size_t smem_max = sizeof(float) * (3 * (size_t)SMEM_M + 8) * (SMEM_M + 1);
    cudaError_t e = cudaFuncSetAttribute(eig_tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max);
    if (e != cudaSuccess) return e;
    eig_tridiag_kernel<<<1, NT, smem, s>>>(C, m, V, d, scratch, d_fail, d_status_on_fail);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the Newton-Schulz step on the output (scratch: S, then the copy of V;
    // the tridiagonal kernel's use of it is over)
    const dim3 g((unsigned)((m + 15) / 16), (unsigned)((m + 15) / 16));
    float *S = scratch, *Vc = scratch + (size_t)m * m;
    ns_gram_kernel<<<g, 256, 0, s>>>(V, m, S, Vc, d_fail, d_status_on_fail);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ns_apply_kernel<<<g, 256, 0, s>>>(Vc, S, m, V);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float2 *cd = reinterpret_cast<const float2 *>(Cdf);
    if (m <= SMEM_M) {
        e = cudaFuncSetAttribute(eig_rayleigh_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)psd_rayleigh_smem(SMEM_M));
        if (e != cudaSuccess) return e;
        eig_rayleigh_smem_kernel<<<psd_eig_ray_blocks(m), 256, psd_rayleigh_smem(m), s>>>(C, cd, V, m, d);
    } else {
        eig_rayleigh_kernel<<<m, 256, 0, s>>>(C, cd, V, m, d);
    }
    return cudaGetLastError();
}

cudaError_t launch_eig_tridiag_grouped(cudaStream_t s, const psd_g_eig *tab, int count, const int2 *bmap_ns,
                                       int nb_ns, const int2 *bmap_ray, int nb_ray, int m_max,
                                       int *d_status_on_fail)
{
    if (count < 1 || nb_ns < 1 || nb_ray < 1 || m_max < 1 || m_max > SMEM_M) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * (3 * (size_t)m_max + 8) * (m_max + 1);
    constexpr size_t smem_max = sizeof(float) * (3 * (size_t)SMEM_M + 8) * (SMEM_M + 1);
    cudaError_t e = cudaFuncSetAttribute(eig_tridiag_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_max);
    if (e != cudaSuccess) return e;
    eig_tridiag_grouped_kernel<<<(unsigned)count, NT, smem, s>>>(tab, d_status_on_fail);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ns_gram_grouped_kernel<<<(unsigned)nb_ns, 256, 0, s>>>(tab, bmap_ns, d_status_on_fail);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ns_apply_grouped_kernel<<<(unsigned)nb_ns, 256, 0, s>>>(tab, bmap_ns);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(eig_rayleigh_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)psd_rayleigh_smem(SMEM_M));
    if (e != cudaSuccess) return e;
    eig_rayleigh_grouped_kernel<<<(unsigned)nb_ray, 256, psd_rayleigh_smem(m_max), s>>>(tab, bmap_ray);
    return cudaGetLastError();
}
