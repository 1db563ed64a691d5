// CholeskyQR steps of the orthonormalisation (QR 'econ' in Alg. 1):
//   R = chol(G) (double-float for the first pass of CholeskyQR2, whose Gram
//   of the raw product can be ill-conditioned; FP32 for the second, whose
//   Gram is I + O(eps)), with the dependent-column rule; R^-1 in FP32; and
//   Q = Y R^-1 (a tall x small product on the CUDA cores).
// For m <= 128 the factorization is blocked (8- or 16-column blocks, three block
// barriers per block, the diagonal block in one warp's registers) and R^-1
// is formed blockwise (cholesky_blocked_kernel); larger m use a right-looking
// kernel in global memory with one barrier per column, each thread owning a
// fixed set of upper-triangle entries.  Double-float numbers
// are unevaluated sums hi + lo of two FP32 values (about 48 significant
// bits; Dekker's two-product by FMA and Knuth's two-sum), which keeps the
// O(m^3) update off the FP64 pipe (about 2 FMA/clk/SM on this GPU).  Sizes
// above 128 work in global memory with FP64 for the first pass.
//
// Dependent-column rule: column j is dependent when its pivot (the squared
// norm of y_j after removing the earlier columns) is <= tau * max_i G_ii, or
// is not a number.  Its row of R becomes e_j^T, so it feeds no other column,
// and its column of Q is written as zero (it then adds nothing to Q^T A Q).
#include <cuda_bf16.h>

#include "ctx.h"

namespace {

constexpr int NT = 1024;
constexpr int SMEM_M = 128;  // largest m kept in shared memory

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
    __device__ static float from2(float2 v) { return v.x; }
    __device__ static float hi(float v) { return v; }
    __device__ static float zero() { return 0.0f; }
    __device__ static float mul(float a, float b) { return a * b; }
    __device__ static float fms(float u, float a, float b) { return fmaf(-a, b, u); }
    // inv = 1 / sqrt(p) from the hardware estimate and one Newton step,
    // y <- y (3 - p y^2) / 2 (error about 1 ulp), r = p inv: the root is on
    // the factorization's critical path, where correctly rounded sqrt and
    // division cost several times more latency
    __device__ static void root(float p, float &r, float &inv)
    {
        float y = rsqrtf(p);
        y = y * fmaf(-0.5f * p, y * y, 1.5f);
        inv = y;
        r = p * y;
    }
    __device__ static float one() { return 1.0f; }
};

template <> struct num<double> {
    __device__ static double from(double v) { return v; }
    __device__ static double from2(float2 v) { return (double)v.x + (double)v.y; }
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
    __device__ static df from2(float2 v) { return {v.x, v.y}; }
    __device__ static float hi(df v) { return v.hi; }
    __device__ static df zero() { return {0.0f, 0.0f}; }
    __device__ static df mul(df a, df b) { return df_mul(a, b); }
    __device__ static df fms(df u, df a, df b) { return df_sub(u, df_mul(a, b)); }
    // from y ~ 1/sqrt(p.hi) (hardware estimate + one FP32 Newton step,
    // about 1 ulp) and x = p.hi y ~ sqrt(p.hi), one Newton step in
    // double-float for each: r = x + (p - x^2) y / 2, inv = y + y (1 - y r);
    // each doubles the ~23 correct bits (about 46 bits)
    __device__ static void root(df p, df &r, df &inv)
    {
        float y = rsqrtf(p.hi);
        y = y * fmaf(-0.5f * p.hi, y * y, 1.5f);
        const float x = p.hi * y;
        const float x2 = x * x;
        const df sq = {x2, fmaf(x, x, -x2)};
        const df dlt = df_sub(p, sq);
        r = quick_two_sum(x, dlt.hi * (0.5f * y));
        const df qr = df_mul({y, 0.0f}, r);
        const df res = df_sub({1.0f, 0.0f}, qr);
        inv = quick_two_sum(y, res.hi * y);
    }
    __device__ static df one() { return {1.0f, 0.0f}; }
};

// Sizes above SMEM_M: the factorization in global memory (gscratch), one
// barrier per column.  T: double (first pass) or float (second pass).  CPL:
// entries of an R^-1 column per lane (m <= 32 CPL).
template <typename T, int CPL>
__global__ void __launch_bounds__(NT)
cholesky_kernel(const double *__restrict__ G, int m, float *Rinv, int *__restrict__ dead,
                int *__restrict__ d_qrank, double tau, T *gU, T *growj, float *gRf,
                int *d_status)
{
    using N = num<T>;
    const int ldu = m;
    T *U = gU;             // row-major upper triangle
    T *rowj = growj;       // scaled row j
    float *Rf = gRf;       // FP32 R (row-major, ldu)
    __shared__ double s_gmax;
    __shared__ int s_dead[PSD_MAX_M];
    __shared__ float s_rdinv[PSD_MAX_M];
    __shared__ T s_r[PSD_MAX_M], s_inv[PSD_MAX_M];
    __shared__ int s_bad;
    const int tid = threadIdx.x;

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

// ---- blocked factorization for m <= SMEM_M -------------------------------
// The same R and the same dependent-column rule, in blocks of NB columns
// (8 or 16) with three block barriers per block instead of one per column:
//   (1) one warp factors the diagonal block column by column (pivot test,
//       root, the block's part of row j of R, update of the rest of the
//       diagonal block);
//   (2) one thread per later column k finishes the block's 16 rows of R in
//       that column (forward substitution down the rows);
//   (3) the trailing upper triangle loses the block's contribution,
//       U(i,k) -= sum_j R(j,i) R(j,k), in 4 x 4 register tiles.
// R^-1 (FP32, from the FP32 copy of R) then comes blockwise: each diagonal
// block inverted by one warp (a lane per column), the off-diagonal blocks by
// recursive doubling (below), two barriers per level.
constexpr int NTB = 512;
// block width NB: 8 for the double-float pass (shorter dependent chain in the
// diagonal block, measured 185 vs 204 us at m = 110), 16 for FP32 (94 vs 98 us)
template <typename T> struct chol_nb { static constexpr int value = 16; };
template <> struct chol_nb<df> { static constexpr int value = 8; };

// warp shuffle of a number (width: the lane group)
__device__ __forceinline__ float shfl_num(float v, int src, int width = 32)
{
    return __shfl_sync(0xffffffffu, v, src, width);
}

__device__ __forceinline__ df shfl_num(df v, int src, int width = 32)
{
    return {__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width)};
}

template <typename T>
size_t blocked_smem(int m)
{
    const size_t ldu = (size_t)m + 1;
    // Tmp: the NB x m panel of the factorization, then the products of the
    // R^-1 doubling (at most SMEM_M / 2 squared floats over all pairs of a level)
    const size_t tmp = (size_t)chol_nb<T>::value * m > (size_t)(SMEM_M / 2) * (SMEM_M / 2)
                           ? (size_t)chol_nb<T>::value * m : (size_t)(SMEM_M / 2) * (SMEM_M / 2);
    return sizeof(T) * m * ldu + sizeof(float) * m * ldu + sizeof(float) * tmp;
}

template <typename T>
__device__ __forceinline__ void cholesky_blocked_body(const float2 *__restrict__ Gd, int m, float *__restrict__ Rinv,
                                                      int *__restrict__ dead, int *__restrict__ d_qrank, float tau,
                                                      int *d_status)
{
    using N = num<T>;
    constexpr int NB = chol_nb<T>::value;
    static_assert(NB == 8 || NB == 16, "block width: lane groups divide a warp");
    extern __shared__ __align__(16) unsigned char smraw[];
    const int ldu = m + 1;
    T *U = reinterpret_cast<T *>(smraw);                               // m x ldu, row-major, upper part
    float *Rf = reinterpret_cast<float *>(U + (size_t)m * ldu);        // FP32 R, m x ldu
    float *Tmp = Rf + (size_t)m * ldu;      // NB x m (panel), then the R^-1 doubling products
    float *X = reinterpret_cast<float *>(smraw);                       // R^-1, m x ldu (U's bytes, once U is done)
    __shared__ float s_gmax;
    __shared__ int s_bad;
    __shared__ int s_dead[SMEM_M];
    __shared__ float s_rdinv[SMEM_M];
    __shared__ T s_inv[SMEM_M];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // G as double-float pairs, symmetric: row-major reads are coalesced,
    // and no FP64 arithmetic is needed to split it
    for (int e = tid; e < m * m; e += NTB) {
        const int i = e / m, k = e - (e / m) * m;
        if (k >= i) U[i * ldu + k] = N::from2(Gd[e]);
    }
    if (tid < 32) {
        float g = 0.0f;
        int bad = 0;
        for (int i = tid; i < m; i += 32) {
            const float v = Gd[(int64_t)i * m + i].x;
            if (!isfinite(v)) bad = 1;
            else if (v > g) g = v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g = fmaxf(g, __shfl_xor_sync(0xffffffffu, g, o));
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (tid == 0) {
            s_gmax = g;
            s_bad = bad;
        }
    }
    __syncthreads();
    if (s_bad && tid == 0) psd_set_status(d_status, PSDPROJ_ENOTFINITE);
    const float thr = tau * s_gmax;
    const bool any = s_gmax > 0.0f;
    const int nblk = (m + NB - 1) / NB;

    for (int b = 0; b < nblk; ++b) {
        const int j0 = b * NB, j1 = min(j0 + NB, m), w = j1 - j0;
        // (1) the diagonal block, one warp, in registers: lane c (and its
        // mirrors c + NB, ...) holds column c of the block, col[a] = U(j0+a, j0+c)
        if (warp == 0) {
            const int c = lane & (NB - 1);
            T col[NB];
#pragma unroll
            for (int a = 0; a < NB; ++a) col[a] = (a <= c && c < w) ? U[(j0 + a) * ldu + j0 + c] : N::zero();
#pragma unroll
            for (int a = 0; a < NB; ++a) {
                if (a < w) {
                    const int j = j0 + a;
                    const T piv = shfl_num(col[a], a);
                    const bool dj = !(N::hi(piv) > thr) || !any;
                    T r = N::one(), inv = N::one();
                    if (!dj) N::root(piv, r, inv);
                    if (c > a) col[a] = dj ? N::zero() : N::mul(col[a], inv);      // R(j, j0+c)
                    else if (c == a) col[a] = r;
                    if (!dj) {
#pragma unroll
                        for (int i = a + 1; i < NB; ++i) {
                            const T ri = shfl_num(col[a], i);                      // R(j, j0+i)
                            if (i <= c && c < w) col[i] = N::fms(col[i], ri, col[a]);
                        }
                    }
                    if (lane == 0) {
                        s_dead[j] = dj ? 1 : 0;
                        s_inv[j] = inv;
                        s_rdinv[j] = N::hi(inv);                                  // 1 / R(j,j) in FP32
                    }
                }
            }
            if (lane < NB && c < w) {
#pragma unroll
                for (int a = 0; a < NB; ++a)
                    if (a <= c) {
                        U[(j0 + a) * ldu + j0 + c] = col[a];
                        Rf[(j0 + a) * ldu + j0 + c] = N::hi(col[a]);
                    }
            }
        }
        __syncthreads();
        // (2) rows j0 .. j1-1 of R in the later columns: NB lanes per column k,
        // lane a holding U(j0+a, k), forward substitution down the rows
        {
            const int a = lane & (NB - 1);
            T rcol[NB];                               // R(j0+a2, j0+a), a2 < a
#pragma unroll
            for (int a2 = 0; a2 < NB; ++a2) rcol[a2] = (a2 < a && a < w) ? U[(j0 + a2) * ldu + j0 + a] : N::zero();
            const int ncol = m - j1;
            constexpr int GPW = 32 / NB;              // lane groups per warp
            for (int g = tid / NB; g < (ncol + GPW - 1) / GPW * GPW; g += NTB / NB) {
                // g runs over a multiple of GPW so that all groups of a warp stay in the loop together
                const int k = j1 + g;
                const bool act = g < ncol && a < w;
                T x = act ? U[(j0 + a) * ldu + k] : N::zero();
#pragma unroll
                for (int a2 = 0; a2 < NB; ++a2) {
                    if (a2 < w) {
                        const int j = j0 + a2;
                        T v = shfl_num(x, a2, NB);
                        v = s_dead[j] ? N::zero() : N::mul(v, s_inv[j]);
                        if (a == a2) x = v;
                        else if (a > a2) x = N::fms(x, rcol[a2], v);
                    }
                }
                if (act) {
                    U[(j0 + a) * ldu + k] = x;
                    Rf[(j0 + a) * ldu + k] = N::hi(x);
                }
            }
        }
        __syncthreads();
        // (3) trailing update, 2 x 2 tiles of the upper triangle
        const int t = m - j1;
        if (t > 0) {
            const int nt = (t + 1) >> 1;
            for (int q = tid; q < nt * nt; q += NTB) {
                const int ti = q / nt, tk = q - (q / nt) * nt;
                if (tk < ti) continue;
                const int i0 = j1 + 2 * ti, k0 = j1 + 2 * tk;
                T acc[2][2];
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        const int i = i0 + u, k = k0 + v;
                        acc[u][v] = (i <= k && k < m) ? U[i * ldu + k] : N::zero();
                    }
#pragma unroll 4
                for (int a = 0; a < w; ++a) {
                    const int j = j0 + a;
                    T ri[2], rk[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        ri[u] = i0 + u < m ? U[j * ldu + i0 + u] : N::zero();
                        rk[u] = k0 + u < m ? U[j * ldu + k0 + u] : N::zero();
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int v = 0; v < 2; ++v) acc[u][v] = N::fms(acc[u][v], ri[u], rk[v]);
                }
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        const int i = i0 + u, k = k0 + v;
                        if (i <= k && k < m) U[i * ldu + k] = acc[u][v];
                    }
            }
        }
        __syncthreads();
    }

    // R^-1 into X (U is no longer read).  (a) diagonal blocks: warp b, lane c
    // solves R(b,b) x = e_c by back substitution
    if (warp < nblk) {
        const int j0 = warp * NB, w = min(NB, m - j0), c = lane;
        float x[NB];
#pragma unroll
        for (int a = 0; a < NB; ++a) x[a] = 0.0f;
#pragma unroll
        for (int a = NB - 1; a >= 0; --a) {
            if (a <= c && a < w && c < w) {
                float sacc = (a == c) ? 1.0f : 0.0f;
#pragma unroll
                for (int q = a + 1; q < NB; ++q)
                    if (q <= c && q < w) sacc = fmaf(-Rf[(j0 + a) * ldu + j0 + q], x[q], sacc);
                x[a] = sacc * s_rdinv[j0 + a];
            }
        }
        if (c < w) {
#pragma unroll
            for (int a = 0; a < NB; ++a)
                if (a < w) X[(j0 + a) * ldu + j0 + c] = a <= c ? x[a] : 0.0f;
        }
    }
    __syncthreads();
    // (b) off-diagonal blocks by recursive doubling: with the diagonal blocks
    // of size h inverted, each pair of adjacent ones [R11 R12; 0 R22] gets
    //   X12 = -X11 (R12 X22),
    // both products in 4 x 4 register tiles over the triangular ranges only
    // (X11, X22 upper triangular; entries below their diagonals are never
    // read), two barriers per level: log2(m / NB) levels.
    for (int h = NB; h < m; h *= 2) {
        const int s2 = 2 * h, npair = (m + s2 - 1) / s2, nt = (h + 3) / 4;
        // Tmp(pair) = R12 X22, h x h per pair
        for (int e = tid; e < npair * nt * nt; e += NTB) {
            const int pidx = e / (nt * nt), rem = e - pidx * (nt * nt);
            const int ti = rem / nt, tc = rem - ti * nt;
            const int j0 = pidx * s2, j1 = j0 + h, h2 = min(h, m - j1);
            if (h2 <= 0 || 4 * tc >= h2) continue;
            float acc[4][4] = {};
            const int kend = min(4 * tc + 4, h2);              // k <= c
            for (int k = 0; k < kend; ++k) {
                float r[4], x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) r[i] = (4 * ti + i < h) ? Rf[(j0 + 4 * ti + i) * ldu + j1 + k] : 0.0f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int cc = 4 * tc + c;
                    x[c] = (cc < h2 && k <= cc) ? X[(j1 + k) * ldu + j1 + cc] : 0.0f;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(r[i], x[c], acc[i][c]);
            }
            float *tp = Tmp + (size_t)pidx * h * h;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * ti + i < h && 4 * tc + c < h2) tp[(4 * ti + i) * h + 4 * tc + c] = acc[i][c];
        }
        __syncthreads();
        // X12 = -X11 Tmp(pair)
        for (int e = tid; e < npair * nt * nt; e += NTB) {
            const int pidx = e / (nt * nt), rem = e - pidx * (nt * nt);
            const int ti = rem / nt, tc = rem - ti * nt;
            const int j0 = pidx * s2, j1 = j0 + h, h2 = min(h, m - j1);
            if (h2 <= 0 || 4 * tc >= h2) continue;
            const float *tp = Tmp + (size_t)pidx * h * h;
            float acc[4][4] = {};
            for (int k = 4 * ti; k < h; ++k) {                  // k >= i
                float xx[4], t[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int ii = 4 * ti + i;
                    xx[i] = (ii < h && k >= ii) ? X[(j0 + ii) * ldu + j0 + k] : 0.0f;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = (4 * tc + c < h2) ? tp[k * h + 4 * tc + c] : 0.0f;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(xx[i], t[c], acc[i][c]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * ti + i < h && 4 * tc + c < h2) X[(j0 + 4 * ti + i) * ldu + j1 + 4 * tc + c] = -acc[i][c];
        }
        __syncthreads();
    }
    for (int e = tid; e < m * m; e += NTB) {
        const int j = e / m, r = e - (e / m) * m;          // column j, row r
        Rinv[(int64_t)j * m + r] = r <= j ? X[r * ldu + j] : 0.0f;
    }
    for (int j = tid; j < m; j += NTB) dead[j] = s_dead[j];
    if (tid == 0 && d_qrank) {
        int r = 0;
        for (int j = 0; j < m; ++j) r += !s_dead[j];
        *d_qrank = r;
    }
}

template <typename T>
__global__ void __launch_bounds__(NTB, 1)
cholesky_blocked_kernel(const float2 *__restrict__ Gd, int m, float *__restrict__ Rinv,
                        int *__restrict__ dead, int *__restrict__ d_qrank, float tau, int *d_status)
{
    cholesky_blocked_body<T>(Gd, m, Rinv, dead, d_qrank, tau, d_status);
}

// many problems in one launch: block b factors entry b
template <typename T>
// (two blocks per SM: many problems in flight, 64 registers fit both passes)
__global__ void __launch_bounds__(NTB, 2)
cholesky_blocked_grouped_kernel(const psd_g_chol *__restrict__ tab, float tau, int *d_status)
{
    const psd_g_chol a = tab[blockIdx.x];
    cholesky_blocked_body<T>(a.Gd, a.m, a.Rinv, a.dead, a.d_qrank, tau, d_status);
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
                       const int *__restrict__ d_cols, float *__restrict__ Z, int64_t ldz,
                       psd_bf16_side side)
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
    // the next K chunk is read into registers while the current one is
    // multiplied (fixed trip counts, so a thread's loads are in flight together)
    constexpr int NY = KW * TR / 256, NB2 = (KW * S + 255) / 256;
    float ry[NY], rb[NB2];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int i = 0; i < NY; ++i) {
            const int e = i * 256 + threadIdx.x;
            const int k = e / TR, r = e % TR;
            const int64_t gr = r0 + r;
            ry[i] = (gr < n && k0 + k < m) ? Y[(int64_t)(k0 + k) * ldy + gr] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < NB2; ++i) {
            const int e = i * 256 + threadIdx.x;
            const int cc = e / KW, k = e % KW;
            rb[i] = (e < KW * S && cc < ncols && k0 + k < m) ? B[(int64_t)cc * m + k0 + k] : 0.0f;
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < m; k0 += KW) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NY; ++i) {
            const int e = i * 256 + threadIdx.x;
            Ys[e / TR][e % TR] = ry[i];
        }
#pragma unroll
        for (int i = 0; i < NB2; ++i) {
            const int e = i * 256 + threadIdx.x;
            if (e < KW * S) Bs[e % KW][e / KW] = rb[i];
        }
        __syncthreads();
        if (k0 + KW < m) fetch(k0 + KW);
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
    const float shift = side.d_shift ? (float)*side.d_shift : 0.0f;
#pragma unroll
    for (int j = 0; j < T; ++j) {
        const int gc = ty * T + j;
        if (gc >= c) continue;
        const bool zero = gc >= ncols || (colmask && colmask[gc]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t gr = r0 + 4 * tx + i;
            if (gr >= n) continue;
            const float z = zero ? 0.0f : acc[i][j];
            Z[(int64_t)gc * ldz + gr] = z;
            // side outputs for the BF16 pass that reads Z next
            if (side.Xh) side.Xh[(int64_t)gc * side.ldh + gr] = __bfloat16_as_ushort(__float2bfloat16_rn(z));
            if (side.Y) side.Y[(int64_t)gc * side.ldy + gr] = shift * z;
        }
    }
}

// The same product for m <= 128 and c <= 128 with B resident: a persistent
// block (three per SM) copies B (zero past *d_cols) into shared memory once
// and walks 32-row tiles of Y (tiles b, b + grid, ...); thread (tx, ty) =
// (tid % 8, tid / 8) owns rows 4 tx .. 4 tx + 3 of the tile and columns
// 4 ty .. 4 ty + 3 (16 FMAs per two 16-byte shared loads per K step).  The
// tile is staged K-major with batched, coalesced loads; stores are coalesced
// over the rows.
constexpr int RT = PSD_TALL_RT;     // rows per tile
// shared row strides (floats) of B, of the Y tile and of the output tile
constexpr int LDB = 132, LDT = 36, LDO = 36;
// shared memory of the product for m rows of B
constexpr size_t tall_smem(int m) { return sizeof(float) * ((size_t)m * (LDB + LDT) + 128 * (size_t)LDO); }

__device__ __forceinline__ void tall_small_res_body(const float *__restrict__ Y, int64_t ldy, int64_t n, int m,
                                                    const float *__restrict__ B, int c,
                                                    const int *__restrict__ colmask, const int *__restrict__ d_cols,
                                                    float *__restrict__ Z, int64_t ldz, psd_bf16_side side,
                                                    int ntiles, int bid, int nb)
{
    extern __shared__ __align__(16) float smt[];
    float *Bs = smt;                              // Bs[k * LDB + col] = B(k, col)
    float *Ys = smt + (size_t)m * LDB;            // Ys[k * LDT + r] = Y(row0 + r, k)
    float *Os = Ys + (size_t)m * LDT;             // Os[col * LDO + r] = Z(row0 + r, col)
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int ncols = d_cols ? min(*d_cols, c) : c;
    // B, 8 loads in flight per thread before their stores
    for (int base = 0; base < m * 128; base += 256 * 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = base + tid + 256 * u;
            const int col = e / m, k = e - (e / m) * m;
            v[u] = (e < m * 128 && col < ncols) ? B[(int64_t)col * m + k] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = base + tid + 256 * u;
            if (e < m * 128) {
                const int col = e / m, k = e - (e / m) * m;
                Bs[k * LDB + col] = v[u];
            }
        }
    }
    const float shift = side.d_shift ? (float)*side.d_shift : 0.0f;
    bool zero[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gc = 4 * ty + j;
        zero[j] = gc >= ncols || (colmask && gc < c && colmask[gc]);
    }
    for (int tile = bid; tile < ntiles; tile += nb) {
        const int64_t row0 = (int64_t)tile * RT;
        __syncthreads();
        // stage Y(row0 .. row0 + 31, 0 .. m-1), 8 loads in flight per thread
        for (int base = 0; base < m * RT; base += 256 * 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = base + tid + 256 * u;
                const int k = e / RT, r = e % RT;
                v[u] = (e < m * RT && row0 + r < n) ? Y[(int64_t)k * ldy + row0 + r] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = base + tid + 256 * u;
                if (e < m * RT) Ys[(e / RT) * LDT + e % RT] = v[u];
            }
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
        // warp w owns columns 16 w .. 16 w + 15; past the used columns B is
        // zero and so is the product: those warps skip the loop (uniform)
#pragma unroll 4
        for (int k = 0; k < (16 * (tid >> 5) < ncols ? m : 0); ++k) {
            const float4 y4 = *reinterpret_cast<const float4 *>(Ys + k * LDT + 4 * tx);
            const float4 b4 = *reinterpret_cast<const float4 *>(Bs + k * LDB + 4 * ty);
            const float y[4] = {y4.x, y4.y, y4.z, y4.w};
            const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(y[i], bb[j], acc[i][j]);
        }
        // the tile through shared memory (one 16-byte store per column and
        // thread), then stored a column per warp instruction: lane = row
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = 4 * ty + j;
            if (gc < c)
                *reinterpret_cast<float4 *>(Os + gc * LDO + 4 * tx) =
                    zero[j] ? make_float4(0.0f, 0.0f, 0.0f, 0.0f)
                            : make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        }
        __syncthreads();
        for (int e = tid; e < c * RT; e += 256) {
            const int gc = e / RT, r = e % RT;
            const int64_t gr = row0 + r;
            if (gr >= n) continue;
            const float z = Os[gc * LDO + r];
            Z[(int64_t)gc * ldz + gr] = z;
            // side outputs for the BF16 pass that reads Z next (or the
            // split-BF16 SYRK's operands)
            const __nv_bfloat16 zh = __float2bfloat16_rn(z);
            if (side.Xh) side.Xh[(int64_t)gc * side.ldh + gr] = __bfloat16_as_ushort(zh);
            if (side.Xl)
                side.Xl[(int64_t)gc * side.ldh + gr] = __bfloat16_as_ushort(__float2bfloat16_rn(z - __bfloat162float(zh)));
            if (side.Y) side.Y[(int64_t)gc * side.ldy + gr] = shift * z;
        }
    }
}

__global__ void __launch_bounds__(256)
tall_small_res_kernel(const float *__restrict__ Y, int64_t ldy, int64_t n, int m, const float *__restrict__ B,
                      int c, const int *__restrict__ colmask, const int *__restrict__ d_cols, float *__restrict__ Z,
                      int64_t ldz, psd_bf16_side side, int ntiles)
{
    tall_small_res_body(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, side, ntiles, blockIdx.x, gridDim.x);
}

// many problems in one launch: block b runs block bmap[b].y of entry
// bmap[b].x, which strides over that entry's tiles by its nb
__global__ void __launch_bounds__(256, 2)
tall_small_res_grouped_kernel(const psd_g_tall *__restrict__ tab, const int2 *__restrict__ bmap)
{
    const int2 b = bmap[blockIdx.x];
    const psd_g_tall a = tab[b.x];
    tall_small_res_body(a.Y, a.ldy, a.n, a.m, a.B, a.c, a.colmask, a.d_cols, a.Z, a.ldz, a.side, a.ntiles, b.y,
                        a.nb);
}

}  // namespace

cudaError_t launch_cholesky(cudaStream_t s, const double *G, const float *Gdf, int m, float *Rinv,
                            int *dead, int *d_qrank, double tau, int *d_status, int first_pass,
                            double *gscratch)
{
    // large m works in global memory: gscratch holds U (m*m), rowj (m) in
    // the factorization type and the FP32 copy of R (m*m floats)
    const bool sm_path = m <= SMEM_M;
    float *gRf = reinterpret_cast<float *>(gscratch + (size_t)m * m + m);
    cudaError_t e;
    if (sm_path) {
        if (!Gdf) return cudaErrorInvalidValue;
        const float2 *gd = reinterpret_cast<const float2 *>(Gdf);
        // the attribute is process-wide: always the largest size (m = SMEM_M),
        // so that threads launching for different m never undercut each other
        if (first_pass) {
            e = cudaFuncSetAttribute(cholesky_blocked_kernel<df>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)blocked_smem<df>(SMEM_M));
            if (e != cudaSuccess) return e;
            cholesky_blocked_kernel<df><<<1, NTB, blocked_smem<df>(m), s>>>(gd, m, Rinv, dead, d_qrank,
                                                                            (float)tau, d_status);
        } else {
            e = cudaFuncSetAttribute(cholesky_blocked_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)blocked_smem<float>(SMEM_M));
            if (e != cudaSuccess) return e;
            cholesky_blocked_kernel<float><<<1, NTB, blocked_smem<float>(m), s>>>(gd, m, Rinv, dead, d_qrank,
                                                                                  (float)tau, d_status);
        }
    } else if (first_pass) {
        cholesky_kernel<double, PSD_MAX_M / 32><<<1, NT, 0, s>>>(G, m, Rinv, dead, d_qrank, tau, gscratch,
                                                                 gscratch + (size_t)m * m, gRf, d_status);
    } else {
        float *fs = reinterpret_cast<float *>(gscratch);
        cholesky_kernel<float, PSD_MAX_M / 32><<<1, NT, 0, s>>>(G, m, Rinv, dead, d_qrank, tau, fs,
                                                               fs + (size_t)m * m, gRf, d_status);
    }
    return cudaGetLastError();
}

cudaError_t launch_tall_small(cudaStream_t s, const float *Y, int64_t ldy, int64_t n, int m,
                              const float *B, int c, const int *colmask, const int *d_cols,
                              float *Z, int64_t ldz, const psd_bf16_side *side, int sm_count)
{
    const unsigned rb = (unsigned)((n + TR - 1) / TR);
    const psd_bf16_side sd = side ? *side : psd_bf16_side{nullptr, 0, nullptr, 0, nullptr};
    if (side && c > 128) return cudaErrorNotSupported;
    if (m <= 128 && c <= 128 && n > 0) {
        const size_t smem = tall_smem(m);
        // the attribute is process-wide: the largest size (m = 128)
        cudaError_t e = cudaFuncSetAttribute(tall_small_res_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tall_smem(128));
        if (e != cudaSuccess) return e;
        const int ntiles = (int)((n + RT - 1) / RT);
        const int per_sm = smem <= 227 * 1024 / 3 ? 3 : 2;
        int grid = (sm_count > 0 ? sm_count : 148) * per_sm;
        if (grid > ntiles) grid = ntiles;
        tall_small_res_kernel<<<grid, 256, smem, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd, ntiles);
        return cudaGetLastError();
    }
    switch ((c + 15) / 16) {
    case 1: tall_small_wide_kernel<1><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    case 2: tall_small_wide_kernel<2><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    case 3: tall_small_wide_kernel<3><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    case 4: tall_small_wide_kernel<4><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    case 5: tall_small_wide_kernel<5><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    case 6: tall_small_wide_kernel<6><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    case 7: tall_small_wide_kernel<7><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    case 8: tall_small_wide_kernel<8><<<rb, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz, sd); break;
    default: {
        dim3 grid(rb, (unsigned)((c + TC - 1) / TC));
        tall_small_kernel<<<grid, 256, 0, s>>>(Y, ldy, n, m, B, c, colmask, d_cols, Z, ldz);
    }
    }
    return cudaGetLastError();
}

cudaError_t launch_cholesky_grouped(cudaStream_t s, const psd_g_chol *tab, int count, int m_max, int first_pass,
                                    double tau, int *d_status)
{
    if (count < 1 || m_max < 1 || m_max > SMEM_M) return cudaErrorInvalidValue;
    cudaError_t e;
    if (first_pass) {
        e = cudaFuncSetAttribute(cholesky_blocked_grouped_kernel<df>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)blocked_smem<df>(SMEM_M));
        if (e != cudaSuccess) return e;
        cholesky_blocked_grouped_kernel<df><<<(unsigned)count, NTB, blocked_smem<df>(m_max), s>>>(tab, (float)tau,
                                                                                                  d_status);
    } else {
        e = cudaFuncSetAttribute(cholesky_blocked_grouped_kernel<float>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)blocked_smem<float>(SMEM_M));
        if (e != cudaSuccess) return e;
        cholesky_blocked_grouped_kernel<float><<<(unsigned)count, NTB, blocked_smem<float>(m_max), s>>>(
            tab, (float)tau, d_status);
    }
    return cudaGetLastError();
}

cudaError_t launch_tall_small_grouped(cudaStream_t s, const psd_g_tall *tab, const int2 *bmap, int nb, int m_max)
{
    if (nb < 1 || m_max < 1 || m_max > 128) return cudaErrorInvalidValue;
    const size_t smem = tall_smem(m_max);
    cudaError_t e = cudaFuncSetAttribute(tall_small_res_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tall_smem(128));
    if (e != cudaSuccess) return e;
    tall_small_res_grouped_kernel<<<(unsigned)nb, 256, smem, s>>>(tab, bmap);
    return cudaGetLastError();
}
