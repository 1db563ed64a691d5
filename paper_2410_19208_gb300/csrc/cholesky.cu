// CholeskyQR steps of the orthonormalisation (QR 'econ' in Alg. 1):
//   R = chol(G) (double-float for the first pass of CholeskyQR2, whose Gram
//   of the raw product can be ill-conditioned; FP32 for the second, whose
//   Gram is I + O(eps)), with the dependent-column rule; R^-1 in FP32; and
//   Q = Y R^-1 (a tall x small product on the CUDA cores).
// The factorization is right-looking in one thread block with two block
// barriers per column; each thread owns a fixed set of upper-triangle
// entries and every thread computes the pivot itself.  Double-float numbers
// are unevaluated sums hi + lo of two FP32 values (about 48 significant
// bits; Dekker's two-product by FMA and Knuth's two-sum), which keeps the
// O(m^3) update off the FP64 pipe (about 2 FMA/clk/SM on this GPU).  Sizes
// above 128 work in global memory with FP64 for the first pass.
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

// ---- double-float arithmetic ------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df quick_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df df_mul(df x, df y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ df df_sub(df x, df y)
{
    df s = two_sum(x.hi, -y.hi);
    s.lo += x.lo - y.lo;
    return quick_two_sum(s.hi, s.lo);
}

// ---- the three number types behind one interface ------------------------
template <typename T> struct num;

template <> struct num<float> {
    __device__ static float from(double v) { return (float)v; }
    __device__ static float hi(float v) { return v; }
    __device__ static float zero() { return 0.0f; }
    __device__ static float mul(float a, float b) { return a * b; }
    __device__ static float fms(float u, float a, float b) { return fmaf(-a, b, u); }
    // r = sqrt(p), inv = 1 / r
    __device__ static void root(float p, float &r, float &inv)
    {
        r = sqrtf(p);
        inv = 1.0f / r;
    }
    __device__ static float one() { return 1.0f; }
};

template <> struct num<double> {
    __device__ static double from(double v) { return v; }
    __device__ static float hi(double v) { return (float)v; }
    __device__ static double zero() { return 0.0; }
    __device__ static double mul(double a, double b) { return a * b; }
    __device__ static double fms(double u, double a, double b) { return fma(-a, b, u); }
    __device__ static void root(double p, double &r, double &inv)
    {
        r = sqrt(p);
        inv = 1.0 / r;
    }
    __device__ static double one() { return 1.0; }
};

template <> struct num<df> {
    __device__ static df from(double v)
    {
        const float h = (float)v;
        return {h, (float)(v - (double)h)};
    }
    __device__ static float hi(df v) { return v.hi; }
    __device__ static df zero() { return {0.0f, 0.0f}; }
    __device__ static df mul(df a, df b) { return df_mul(a, b); }
    __device__ static df fms(df u, df a, df b) { return df_sub(u, df_mul(a, b)); }
    // one Newton step from the FP32 root: r = x + (p - x^2) / (2x); then
    // inv = q + q (1 - q r) from q = 1 / r.hi
    __device__ static void root(df p, df &r, df &inv)
    {
        const float x = sqrtf(p.hi);
        const float x2 = x * x;
        const df sq = {x2, fmaf(x, x, -x2)};
        const df dlt = df_sub(p, sq);
        r = quick_two_sum(x, dlt.hi / (2.0f * x));
        const float q = 1.0f / r.hi;
        const df qr = df_mul({q, 0.0f}, r);
        const df res = df_sub({1.0f, 0.0f}, qr);
        inv = quick_two_sum(q, res.hi * q);
    }
    __device__ static df one() { return {1.0f, 0.0f}; }
};

// T: df (first pass, m <= 128), double (first pass, m > 128) or float (second
// pass).  CPL: entries of an R^-1 column per lane (m <= 32 CPL).
template <typename T, int CPL>
__global__ void __launch_bounds__(NT)
cholesky_kernel(const double *__restrict__ G, int m, float *Rinv, int *__restrict__ dead,
                int *__restrict__ d_qrank, double tau, T *gU, T *growj, float *gRf,
                int *d_status)
{
    using N = num<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const bool in_smem = m <= SMEM_M;
    const int ldu = in_smem ? (m + 1) : m;
    T *U = in_smem ? reinterpret_cast<T *>(smraw) : gU;             // row-major upper triangle
    T *rowj = in_smem ? (U + m * (m + 1)) : growj;                  // scaled row j
    float *Rf = in_smem ? reinterpret_cast<float *>(rowj + m) : gRf; // FP32 R (row-major, ldu)
    __shared__ double s_gmax;
    __shared__ int s_dead[PSD_MAX_M];
    __shared__ float s_rdinv[PSD_MAX_M];
    __shared__ T s_r[PSD_MAX_M], s_inv[PSD_MAX_M];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    const int nup = m * (m + 1) / 2;

    // U = upper(G)
    for (int e = tid; e < m * m; e += NT) {
        const int i = e / m, k = e - (e / m) * m;
        if (k >= i) U[i * ldu + k] = N::from(G[(int64_t)k * m + i]);
    }
    if (tid < 32) {
        double g = 0.0;
        int bad = 0;
        for (int i = tid; i < m; i += 32) {
            const double v = G[(int64_t)i * m + i];
            if (!isfinite(v)) bad = 1;
            else if (v > g) g = v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (tid == 0) {
            s_gmax = g;
            s_bad = bad;
        }
    }
    // this thread's upper-triangle entries (fixed for the whole factorization),
    // packed as i | k << 16.  They are counted from the END of the row-major
    // order (slot c holds entry nup - 1 - (tid + c NT)), so the entries still
    // to update at column j, rows >= j, are slot prefixes: a thread stops at
    // its first finished slot.
    int eik[EPT];
#pragma unroll
    for (int c = 0; c < EPT; ++c) {
        const int e = nup - 1 - (tid + c * NT);
        eik[c] = -1;
        if (in_smem && e >= 0) {
            // e -> (i <= k), row-major over the upper triangle
            const float hb = 2.0f * m + 1.0f;
            int i = (int)((hb - sqrtf(fmaxf(hb * hb - 8.0f * e, 0.0f))) * 0.5f);
            i = max(0, min(i, m - 1));
            while (i > 0 && i * m - i * (i - 1) / 2 > e) --i;
            while (i + 1 < m && (i + 1) * m - (i + 1) * i / 2 <= e) ++i;
            eik[c] = i | ((i + (e - (i * m - i * (i - 1) / 2))) << 16);
        }
    }
    __syncthreads();
    if (s_bad) psd_set_status(d_status, PSDPROJ_ENOTFINITE);
    const float thr = (float)(tau * s_gmax);
    const bool any = s_gmax > 0.0;
    // pivot j -> R_jj, 1 / R_jj and the dependence flag, by one thread
    auto pivot = [&](int j, T piv) {
        const bool dj = !(N::hi(piv) > thr) || !any;
        T r = N::one(), inv = N::one();
        if (!dj) N::root(piv, r, inv);
        s_r[j] = r;
        s_inv[j] = inv;
        s_dead[j] = dj ? 1 : 0;
        s_rdinv[j] = 1.0f / N::hi(r);
    };
    if (tid == 0) pivot(0, U[0]);
    __syncthreads();

    if (in_smem) {
        // One phase and one barrier per column.  Row j of U is final when
        // column j starts and is only read in its phase: the owners of
        // (j, k) write row j of R, the owners of (i, k), i > j, update
        //   U(i,k) -= U(j,i) U(j,k) / R_jj^2,
        // and the owner of (j+1, j+1) forms the next pivot.  A thread takes
        // its entries in groups of G, loads first, so the loads overlap.
        for (int j = 0; j < m; ++j) {
            const bool dj = s_dead[j] != 0;
            const T inv = s_inv[j];
            const T inv2 = N::mul(inv, inv);
            const T *rowU = U + j * ldu;
            const int nact = nup - (j * m - j * (j - 1) / 2);   // entries (i, k), i >= j
#pragma unroll
            for (int c = 0; c < EPT; ++c) {
                if (tid + c * NT >= nact) break;
                const int i = eik[c] & 0xFFFF, k = eik[c] >> 16;
                const T u0 = U[i * ldu + k];
                if (i == j) {
                    Rf[j * ldu + k] = (k == j) ? N::hi(s_r[j]) : (dj ? 0.0f : N::hi(N::mul(u0, inv)));
                } else {
                    T u = u0;
                    if (!dj) u = N::fms(u, N::mul(rowU[i], inv2), rowU[k]);
                    U[i * ldu + k] = u;
                    if (i == j + 1 && k == j + 1) pivot(j + 1, u);
                }
            }
            __syncthreads();
        }
    } else {
        for (int j = 0; j < m; ++j) {
            // phase A: row j of R into rowj (the update's operand) and Rf
            const bool dj = s_dead[j] != 0;
            const T inv = s_inv[j];
            for (int k = j + tid; k < m; k += NT) {
                const T v = (k == j) ? s_r[j] : (dj ? N::zero() : N::mul(U[j * ldu + k], inv));
                rowj[k] = (k == j) ? N::zero() : v;
                Rf[j * ldu + k] = N::hi(v);
            }
            __syncthreads();
            // phase B: trailing update U(i,k) -= R(j,i) R(j,k), j < i <= k
            const int t = m - j - 1;
            if (!dj) {
                for (int e = tid; e < t * t; e += NT) {
                    const int a = e / t, b = e - (e / t) * t;
                    if (b < a) continue;
                    const int i = j + 1 + a, k = j + 1 + b;
                    U[i * ldu + k] = N::fms(U[i * ldu + k], rowj[i], rowj[k]);
                }
            }
            // e = 0 is entry (j+1, j+1), updated by thread 0 above
            if (tid == 0 && t > 0) pivot(j + 1, U[(j + 1) * ldu + (j + 1)]);
            __syncthreads();
        }
    }

    // R^-1 (upper, FP32), one warp per column j: back substitution in axpy
    // form with the column held in registers (lane l owns rows l + 32 c):
    //   for i = j .. 0:  x_i = b_i / R_ii;  b_r -= x_i R_ri  (r < i),  b = e_j
    // Slots c above the one holding row i hold rows > i and are skipped
    // (a warp-uniform branch).
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < m; j += NT / 32) {
        float b[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) b[c] = (lane + 32 * c == j) ? 1.0f : 0.0f;
        for (int i = j; i >= 0; --i) {
            const int ci = i >> 5;
            float v = b[0];
#pragma unroll
            for (int c = 1; c < CPL; ++c)
                if (c == ci) v = b[c];
            v = __shfl_sync(0xffffffffu, v, i & 31);
            const float xi = v * s_rdinv[i];
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                if (c > ci) break;
                const int r = lane + 32 * c;
                if (r < i) b[c] = fmaf(-xi, Rf[r * ldu + i], b[c]);
                else if (r == i) b[c] = xi;
            }
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int r = lane + 32 * c;
            if (r < m) Rinv[(int64_t)j * m + r] = b[c];
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

// The same product for c <= 128 columns: one block covers 64 rows and all
// c output columns (16 x 16 threads, thread (tx, ty) owns rows 4 tx .. 4 tx + 3
// and columns ty T .. ty T + T-1, T = ceil(c / 16)), so B is staged once per
// K chunk and the rows of Y are read with 16-byte loads.
template <int T>
__global__ void __launch_bounds__(256)
tall_small_wide_kernel(const float *__restrict__ Y, int64_t ldy, int64_t n, int m,
                       const float *__restrict__ B, int c, const int *__restrict__ colmask,
                       const int *__restrict__ d_cols, float *__restrict__ Z, int64_t ldz)
{
    constexpr int S = 16 * T;
    constexpr int KW = 32;                      // K rows staged at a time
    __shared__ __align__(16) float Ys[KW][TR];
    __shared__ float Bs[KW][S + 1];
    const int64_t r0 = (int64_t)blockIdx.x * TR;
    const int ncols = d_cols ? min(*d_cols, c) : c;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][T];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < m; k0 += KW) {
        __syncthreads();
        for (int e = threadIdx.x; e < KW * TR; e += 256) {
            const int k = e / TR, r = e % TR;
            const int64_t gr = r0 + r;
            Ys[k][r] = (gr < n && k0 + k < m) ? Y[(int64_t)(k0 + k) * ldy + gr] : 0.0f;
        }
        for (int e = threadIdx.x; e < KW * S; e += 256) {
            const int cc = e / KW, k = e % KW;
            Bs[k][cc] = (cc < ncols && k0 + k < m) ? B[(int64_t)cc * m + k0 + k] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KW; ++k) {
            const float4 y4 = *reinterpret_cast<const float4 *>(&Ys[k][4 * tx]);
            const float y[4] = {y4.x, y4.y, y4.z, y4.w};
            float b[T];
#pragma unroll
            for (int j = 0; j < T; ++j) b[j] = Bs[k][ty * T + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < T; ++j) acc[i][j] = fmaf(y[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int gc = ty * T + j;
        if (gc >= c) continue;
        const bool zero = gc >= ncols || (colmask && colmask[gc]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t gr = r0 + 4 * tx + i;
            if (gr < n) Z[(int64_t)gc * ldz + gr] = zero ? 0.0f : acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_cholesky(cudaStream_t s, const double *G, int m, float *Rinv, int *dead,
                            int *d_qrank, double tau, int *d_status, int first_pass,
                            double *gscratch)
{
    // large m works in global memory: gscratch holds U (m*m), rowj (m) in
    // the factorization type and the FP32 copy of R (m*m floats)
    const bool sm_path = m <= SMEM_M;
    float *gRf = reinterpret_cast<float *>(gscratch + (size_t)m * m + m);
    cudaError_t e;
    if (first_pass && sm_path) {
        const size_t smem = sizeof(df) * ((size_t)m * (m + 1) + m) + sizeof(float) * m * (m + 1);
        auto kern = cholesky_kernel<df, SMEM_M / 32>;
        // the attribute is process-wide: always the largest size (m = SMEM_M),
        // so that threads launching for different m never undercut each other
        constexpr size_t smem_max = sizeof(df) * ((size_t)SMEM_M * (SMEM_M + 1) + SMEM_M) +
                                    sizeof(float) * SMEM_M * (SMEM_M + 1);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e != cudaSuccess) return e;
        kern<<<1, NT, smem, s>>>(G, m, Rinv, dead, d_qrank, tau, nullptr, nullptr, nullptr, d_status);
    } else if (first_pass) {
        cholesky_kernel<double, PSD_MAX_M / 32><<<1, NT, 0, s>>>(G, m, Rinv, dead, d_qrank, tau, gscratch,
                                                                 gscratch + (size_t)m * m, gRf, d_status);
    } else {
        float *fs = reinterpret_cast<float *>(gscratch);
        if (sm_path) {
            const size_t smem = sizeof(float) * ((size_t)m * (m + 1) + m) + sizeof(float) * m * (m + 1);
            auto kern = cholesky_kernel<float, SMEM_M / 32>;
            constexpr size_t smem_max = sizeof(float) * ((size_t)SMEM_M * (SMEM_M + 1) + SMEM_M) +
                                        sizeof(float) * SMEM_M * (SMEM_M + 1);
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
            if (e != cudaSuccess) return e;
            kern<<<1, NT, smem, s>>>(G, m, Rinv, dead, d_qrank, tau, fs, fs + (size_t)m * m, gRf, d_status);
        } else {
            cholesky_kernel<float, PSD_MAX_M / 32><<<1, NT, 0, s>>>(G, m, Rinv, dead, d_qrank, tau, fs,
                                                                   fs + (size_t)m * m, gRf, d_status);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_tall_small(cudaStream_t s, const float *Y, int64_t ldy, int64_t n, int m,
                              const float *B, int c, const int *colmask, const int *d_cols,
                              float *Z, int64_t ldz)
{
    const unsigned rb = (unsigned)((n + TR - 1) / TR);
    switch ((c + 15) / 16) {
    case 1: tall_small_wide_kernel<1><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    case 2: tall_small_wide_kernel<2><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    case 3: tall_small_wide_kernel<3><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    case 4: tall_small_wide_kernel<4><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    case 5: tall_small_wide_kernel<5><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    case 6: tall_small_wide_kernel<6><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    case 7: tall_small_wide_kernel<7><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    case 8: tall_small_wide_kernel<8><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz); break;
    default: {
        dim3 grid(rb, (unsigned)((c + TC - 1) / TC));
        tall_small_kernel<<<grid, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz);
    }
    }
    return cudaGetLastError();
}
