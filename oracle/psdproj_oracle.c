/*
 * psdproj_oracle.c -- FP64 CPU oracle for the randomized PSD projections of
 * Jones & Anderson, "Approximate Projection onto the Positive Semidefinite Cone
 * Using Randomization" (arXiv 2410.19208).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent, deliberately plain
 * and slow reference that the CUDA library is checked against.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm load it.
 * It shares no source, header, table or helper with the CUDA library
 * (paper_2410_19208_gb300/csrc); both sides implement Philox4x32-10 from its
 * published definition (Salmon, Moraes, Dror, Shaw, SC'11).
 *
 * Conventions
 *   - Everything is double precision.  The input matrix A is dense, row-major,
 *     n x n with leading dimension lda; only its upper triangle (j >= i) is
 *     ever read, as the GPU path does.
 *   - Tall matrices (Omega, Y, Q, W) are row-major n x m (element (i,c) at
 *     [i*m + c]).
 *   - "l" in this file is the sketch width k+p (the paper's k+l; the paper's
 *     oversampling letter l is called p here).
 *
 * Parity status (see the pins in tests/test_oracle_*.py):
 *   philox / gauss      pinned (Triton's Philox4x32-10, moments, KS)
 *   jacobi / exact      pinned (numpy eigh, Householder closed form, Fig. 3
 *                        pair, polar form, Moreau invariants)
 *   range finder        pinned (Q^T Q = I, Y = Q R, one-shot == re-orth range)
 *   alg1 / alg2         pinned (exact recovery, Counterexample 1, Lemma 4,
 *                        invariants, Cor. 1 / Prop. 3 bounds in the mean)
 *   min_eig             pinned (min-eig identity of the appendix lemma,
 *                        convergence in N)
 *   eps1 / eps2         pinned (hand-evaluated closed forms)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOCONV 4

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3 "Philox").                    */
/* One round maps (x0,x1,x2,x3) with key (k0,k1) to                           */
/*   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)),        */
/* and the key is advanced by the Weyl constants between rounds.             */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], uint32_t k0, uint32_t k1,
                       uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Standard normal for element (i, j) of random stream `stream`:
 * counter (i, j, stream, 0), key (seed low word, seed high word);
 * u = (x + 1/2) 2^-32 from words 0 and 1; Box-Muller cosine branch in FP64.
 * The paper only asks for i.i.d. N(0,1) test vectors (Alg. 1 "randn",
 * footnote on the test-vector distribution); this keying is our reading. */
double orc_gauss(uint64_t seed, uint32_t i, uint32_t j, uint32_t stream)
{
    uint32_t c[4] = {i, j, stream, 0u}, o[4];
    orc_philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), o);
    const double two32 = 4294967296.0;
    double u1 = ((double)o[0] + 0.5) / two32;
    double u2 = ((double)o[1] + 0.5) / two32;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Omega: n x m row-major, element (i,c) = gauss(seed, i, c, stream). */
void orc_omega(uint64_t seed, int64_t n, int m, uint32_t stream, double *Om)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < m; ++c)
            Om[i * m + c] = orc_gauss(seed, (uint32_t)i, (uint32_t)c, stream);
}

/* ------------------------------------------------------------------------ */
/* Symmetric product Y = A X + shift * X, reading only the upper triangle.   */
/* X, Y row-major n x m.  Threads own rows of the upper triangle and keep     */
/* private accumulators for the transposed contributions.                    */
/* ------------------------------------------------------------------------ */
static int sym_mul(const double *A, int64_t n, int64_t lda, const double *X,
                   int m, double shift, double *Y)
{
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nt * (size_t)n * (size_t)m, sizeof(double));
    if (!acc) return ORC_ENOMEM;
#pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *Yt = acc + (size_t)t * (size_t)n * (size_t)m;
#pragma omp for schedule(static, 16)
        for (int64_t i = 0; i < n; ++i) {
            const double *Ai = A + i * lda;
            double *yi = Yt + i * m;
            const double *xi = X + i * m;
            for (int64_t j = i; j < n; ++j) {
                double a = Ai[j];
                const double *xj = X + j * m;
                for (int c = 0; c < m; ++c) yi[c] += a * xj[c];
                if (j != i) {
                    double *yj = Yt + j * m;
                    for (int c = 0; c < m; ++c) yj[c] += a * xi[c];
                }
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < m; ++c) {
            double s = shift * X[i * m + c];
            for (int t = 0; t < nt; ++t) s += acc[(size_t)t * n * m + i * m + c];
            Y[i * m + c] = s;
        }
    free(acc);
    return ORC_OK;
}

int orc_sym_mul(const double *A, int64_t n, int64_t lda, const double *X,
                int m, double shift, double *Y)
{
    return sym_mul(A, n, lda, X, m, shift, Y);
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi eigensolver for a dense symmetric m x m matrix (FP64).      */
/* Row-cyclic order; rotation from the classical stable formula               */
/* (Golub & Van Loan, sym.schur2).  C is overwritten (its diagonal holds the  */
/* eigenvalues on exit); V (m x m row-major) receives the eigenvectors as     */
/* columns; d receives the eigenvalues (unsorted, column order of V).          */
/* Returns ORC_OK, or ORC_ENOCONV if max_sweeps did not reach the tolerance.   */
/* ------------------------------------------------------------------------ */
int orc_jacobi_eig(int m, double *C, double *V, double *d, double rel_tol,
                   int max_sweeps, int *sweeps_out)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < m * m; ++i) fro += C[i] * C[i];
    fro = sqrt(fro);
    int sweep = 0, status = ORC_ENOCONV;
    for (; sweep <= max_sweeps; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) off += 2.0 * C[p * m + q] * C[p * m + q];
        if (sqrt(off) <= rel_tol * fro || fro == 0.0) { status = ORC_OK; break; }
        if (sweep == max_sweeps) break;
        for (int p = 0; p < m - 1; ++p) {
            for (int q = p + 1; q < m; ++q) {
                double apq = C[p * m + q];
                if (apq == 0.0) continue;
                double app = C[p * m + p], aqq = C[q * m + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t;
                if (fabs(tau) > 1e150) t = 0.5 / tau;
                else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* columns p, q */
                for (int k = 0; k < m; ++k) {
                    double akp = C[k * m + p], akq = C[k * m + q];
                    C[k * m + p] = c * akp - s * akq;
                    C[k * m + q] = s * akp + c * akq;
                }
                /* rows p, q */
                for (int k = 0; k < m; ++k) {
                    double apk = C[p * m + k], aqk = C[q * m + k];
                    C[p * m + k] = c * apk - s * aqk;
                    C[q * m + k] = s * apk + c * aqk;
                }
                C[p * m + q] = 0.0;
                C[q * m + p] = 0.0;
                for (int k = 0; k < m; ++k) {
                    double vkp = V[k * m + p], vkq = V[k * m + q];
                    V[k * m + p] = c * vkp - s * vkq;
                    V[k * m + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < m; ++i) d[i] = C[i * m + i];
    if (sweeps_out) *sweeps_out = sweep;
    return status;
}

/* Exact projection (Thm 1): X+ = U diag(max(lambda,0)) U^T with the full
 * eigendecomposition from cyclic Jacobi.  P is dense n x n row-major. */
int orc_exact_proj(const double *A, int64_t n, int64_t lda, double *P)
{
    int m = (int)n;
    double *C = (double *)malloc(sizeof(double) * m * m);
    double *V = (double *)malloc(sizeof(double) * m * m);
    double *d = (double *)malloc(sizeof(double) * m);
    if (!C || !V || !d) { free(C); free(V); free(d); return ORC_ENOMEM; }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            C[i * m + j] = (j >= i) ? A[i * lda + j] : A[j * lda + i];
    int st = orc_jacobi_eig(m, C, V, d, 1e-15, 100, NULL);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int k = 0; k < m; ++k)
                if (d[k] > 0.0) s += V[i * m + k] * d[k] * V[j * m + k];
            P[(int64_t)i * n + j] = s;
        }
    free(C); free(V); free(d);
    return st;
}

/* ------------------------------------------------------------------------ */
/* orth(Y): modified Gram-Schmidt with a second full re-orthogonalisation     */
/* pass, the economy QR of Alg. 1.  Column j is declared dependent when its   */
/* squared residual norm is <= tau * max_i ||y_i||^2; a dependent column is   */
/* set to zero (it then adds nothing to Q^T X Q nor to the output).           */
/* Y (n x m row-major) is overwritten by Q.  Returns the numerical rank.      */
/* ------------------------------------------------------------------------ */
int orc_orth(double *Y, int64_t n, int m, double tau)
{
    double gmax = 0.0;
    double *col = (double *)malloc(sizeof(double) * n);
    for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += Y[i * m + j] * Y[i * m + j];
        if (s > gmax) gmax = s;
    }
    int rank = 0;
    for (int j = 0; j < m; ++j) {
        for (int64_t i = 0; i < n; ++i) col[i] = Y[i * m + j];
        for (int pass = 0; pass < 2; ++pass) {
            for (int k = 0; k < j; ++k) {
                double dot = 0.0;
                for (int64_t i = 0; i < n; ++i) dot += Y[i * m + k] * col[i];
                for (int64_t i = 0; i < n; ++i) col[i] -= dot * Y[i * m + k];
            }
        }
        double nrm2 = 0.0;
        for (int64_t i = 0; i < n; ++i) nrm2 += col[i] * col[i];
        if (!(nrm2 > tau * gmax) || gmax == 0.0) {
            for (int64_t i = 0; i < n; ++i) Y[i * m + j] = 0.0;
        } else {
            double inv = 1.0 / sqrt(nrm2);
            for (int64_t i = 0; i < n; ++i) Y[i * m + j] = col[i] * inv;
            ++rank;
        }
    }
    free(col);
    return rank;
}

/* Range finder (Alg. 1) on S = (A + shift I) * scale.
 *   reorth = 1: orthonormalise after every product (subspace iteration):
 *               Q = orth(S Om); repeat 2q times Q = orth(S Q).
 *   reorth = 0: the literal one-shot form Q = orth(S^(2q+1) Om).
 * Om is n x m row-major; Q (n x m) receives the basis.  Returns the rank
 * (>= 0) or a negative status. */
int orc_range_finder(const double *A, int64_t n, int64_t lda, const double *Om,
                     int m, int q, double shift, double scale, int reorth,
                     double tau, double *Q)
{
    double *T = (double *)malloc(sizeof(double) * n * m);
    if (!T) return -ORC_ENOMEM;
    int st = sym_mul(A, n, lda, Om, m, shift, Q);
    if (st) { free(T); return -st; }
    for (int64_t i = 0; i < n * m; ++i) Q[i] *= scale;
    int rank = m;
    if (reorth) rank = orc_orth(Q, n, m, tau);
    for (int t = 0; t < 2 * q; ++t) {
        st = sym_mul(A, n, lda, Q, m, shift, T);
        if (st) { free(T); return -st; }
        for (int64_t i = 0; i < n * m; ++i) Q[i] = T[i] * scale;
        if (reorth) rank = orc_orth(Q, n, m, tau);
    }
    if (!reorth) rank = orc_orth(Q, n, m, tau);
    free(T);
    return rank;
}

/* C = Q^T (A + shift I) Q, symmetrised, m x m row-major. */
static int core(const double *A, int64_t n, int64_t lda, const double *Q, int m,
                double shift, double *C)
{
    double *Z = (double *)malloc(sizeof(double) * n * m);
    if (!Z) return ORC_ENOMEM;
    int st = sym_mul(A, n, lda, Q, m, shift, Z);
    if (st) { free(Z); return st; }
#pragma omp parallel for schedule(static)
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += Q[i * m + a] * Z[i * m + b];
            C[a * m + b] = s;
        }
    for (int a = 0; a < m; ++a)
        for (int b = a + 1; b < m; ++b) {
            double s = 0.5 * (C[a * m + b] + C[b * m + a]);
            C[a * m + b] = s;
            C[b * m + a] = s;
        }
    free(Z);
    return ORC_OK;
}

/* W = Q V diag(sqrt(g(d))) where g(d) = max(d, 0) (mode 0) or
 * alpha * (max(d, 1) - 1) (mode 1, the literal last step of Alg. 3).
 * Returns r+, the number of columns with g(d) > 0. */
static int factor(const double *Q, int64_t n, int m, const double *V,
                  const double *d, int mode, double alpha, double *W)
{
    double *g = (double *)malloc(sizeof(double) * m);
    int rp = 0;
    for (int j = 0; j < m; ++j) {
        double v = (mode == 0) ? (d[j] > 0.0 ? d[j] : 0.0)
                               : alpha * ((d[j] > 1.0 ? d[j] : 1.0) - 1.0);
        g[j] = sqrt(v);
        if (v > 0.0) ++rp;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int a = 0; a < m; ++a) s += Q[i * m + a] * V[a * m + j];
            W[i * m + j] = s * g[j];
        }
    free(g);
    return rp;
}

/* Randomized PSD projection (Alg. 2 with Alg. 1 inside; "Algorithm 1" of the
 * C ABI).  m = k + p columns.  Outputs W (n x m row-major) with P = W W^T,
 * the eigenvalues d (m) of Q^T A Q, the sketch rank and r+.
 * reorth selects the range-finder form (1 = orthonormalise after each
 * product).  Returns a status. */
int orc_alg1(const double *A, int64_t n, int64_t lda, int k, int p, int q,
             uint64_t seed, int reorth, double *W, double *d_out,
             int *rank_out, int *rplus_out)
{
    int m = k + p;
    if (n < 1 || k < 1 || p < 0 || m < 1 || q < 0) return ORC_EINVAL;
    double *Om = (double *)malloc(sizeof(double) * n * m);
    double *Q = (double *)malloc(sizeof(double) * n * m);
    double *C = (double *)malloc(sizeof(double) * m * m);
    double *V = (double *)malloc(sizeof(double) * m * m);
    double *d = (double *)malloc(sizeof(double) * m);
    if (!Om || !Q || !C || !V || !d) {
        free(Om); free(Q); free(C); free(V); free(d);
        return ORC_ENOMEM;
    }
    orc_omega(seed, n, m, 0u, Om);
    int rank = orc_range_finder(A, n, lda, Om, m, q, 0.0, 1.0, reorth, 1e-10, Q);
    int st = rank < 0 ? -rank : ORC_OK;
    if (!st) st = core(A, n, lda, Q, m, 0.0, C);
    if (!st) st = orc_jacobi_eig(m, C, V, d, 1e-15, 100, NULL);
    if (!st) {
        int rp = factor(Q, n, m, V, d, 0, 0.0, W);
        if (rplus_out) *rplus_out = rp;
        if (rank_out) *rank_out = rank;
        if (d_out) memcpy(d_out, d, sizeof(double) * m);
    }
    free(Om); free(Q); free(C); free(V); free(d);
    return st;
}

/* power_iteration (Alg. 4) on S = A + shift I: v = randn (stream), then N
 * times v = S v / ||S v||, then sigma = ||S v||.  N + 1 products. */
double orc_power_iteration(const double *A, int64_t n, int64_t lda, double shift,
                           int N, uint64_t seed, uint32_t stream)
{
    double *v = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    orc_omega(seed, n, 1, stream, v);
    double nrm = 0.0;
    for (int it = 0; it <= N; ++it) {
        sym_mul(A, n, lda, v, 1, shift, w);
        nrm = 0.0;
        for (int64_t i = 0; i < n; ++i) nrm += w[i] * w[i];
        nrm = sqrt(nrm);
        if (it == N || nrm == 0.0) break;
        for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nrm;
    }
    free(v); free(w);
    return nrm;
}

/* min_eig (Alg. 5): sigma1 = PI(A), sigma2 = PI(A - sigma1 I),
 * alpha = |sigma1 - sigma2|.  Power-iteration vectors from streams 3 and 4. */
double orc_min_eig(const double *A, int64_t n, int64_t lda, int N, uint64_t seed,
                   double *sigma1_out, double *sigma2_out)
{
    double s1 = orc_power_iteration(A, n, lda, 0.0, N, seed, 3u);
    double s2 = orc_power_iteration(A, n, lda, -s1, N, seed, 4u);
    if (sigma1_out) *sigma1_out = s1;
    if (sigma2_out) *sigma2_out = s2;
    return fabs(s1 - s2);
}

/* Scaled randomized PSD projection (Alg. 3; "Algorithm 2" of the C ABI).
 * alpha_in > 0 is used as given; otherwise alpha = min_eig(A, N) (Alg. 5).
 * If alpha is not finite or <= 1e-300 the call degrades to Alg. 2 and
 * *degraded = 1.
 * W_lit: the literal last step  alpha Q V (max(D,1) - I) V^T Q^T with
 *        V D V^T = eig(Q^T B Q), B = (A + alpha I)/alpha;
 * W_red: the reduced form Q (Q^T A Q)_+ Q^T of Lemma 4.
 * Either output pointer may be NULL. */
int orc_alg2(const double *A, int64_t n, int64_t lda, int k, int p, int q,
             uint64_t seed, double alpha_in, int N, int reorth, double *W_lit,
             double *W_red, double *alpha_out, int *degraded, int *rank_out,
             int *rplus_out)
{
    int m = k + p;
    if (n < 1 || k < 1 || p < 0 || q < 0 || N < 0) return ORC_EINVAL;
    double alpha = alpha_in;
    if (!(alpha_in > 0.0)) alpha = orc_min_eig(A, n, lda, N, seed, NULL, NULL);
    if (alpha_out) *alpha_out = alpha;
    if (!(alpha > 1e-300) || !isfinite(alpha)) {
        if (degraded) *degraded = 1;
        int st = ORC_OK;
        if (W_red) st = orc_alg1(A, n, lda, k, p, q, seed, reorth, W_red, NULL, rank_out, rplus_out);
        if (!st && W_lit) st = orc_alg1(A, n, lda, k, p, q, seed, reorth, W_lit, NULL, NULL, NULL);
        return st;
    }
    if (degraded) *degraded = 0;
    double *Om = (double *)malloc(sizeof(double) * n * m);
    double *Q = (double *)malloc(sizeof(double) * n * m);
    double *C = (double *)malloc(sizeof(double) * m * m);
    double *V = (double *)malloc(sizeof(double) * m * m);
    double *d = (double *)malloc(sizeof(double) * m);
    if (!Om || !Q || !C || !V || !d) {
        free(Om); free(Q); free(C); free(V); free(d);
        return ORC_ENOMEM;
    }
    orc_omega(seed, n, m, 0u, Om);
    /* Q = range_finder(B) with B = (A + alpha I) / alpha (Alg. 3, lines 1-2) */
    int rank = orc_range_finder(A, n, lda, Om, m, q, alpha, 1.0 / alpha, reorth, 1e-10, Q);
    int st = rank < 0 ? -rank : ORC_OK;
    if (!st && W_lit) {
        /* Q^T B Q = (Q^T A Q + alpha Q^T Q) / alpha, eig, alpha (max(D,1) - I) */
        st = core(A, n, lda, Q, m, alpha, C);
        for (int i = 0; !st && i < m * m; ++i) C[i] /= alpha;
        if (!st) st = orc_jacobi_eig(m, C, V, d, 1e-15, 100, NULL);
        if (!st) factor(Q, n, m, V, d, 1, alpha, W_lit);
    }
    if (!st && W_red) {
        st = core(A, n, lda, Q, m, 0.0, C);
        if (!st) st = orc_jacobi_eig(m, C, V, d, 1e-15, 100, NULL);
        if (!st) {
            int rp = factor(Q, n, m, V, d, 0, 0.0, W_red);
            if (rplus_out) *rplus_out = rp;
        }
    }
    if (rank_out) *rank_out = rank;
    free(Om); free(Q); free(C); free(V); free(d);
    return st;
}

/* Core step of Alg. 2 for a caller-supplied orthonormal Q (used by the
 * Counterexample 1 test): W = Q V diag(sqrt(max(d,0))) with
 * V D V^T = eig(Q^T A Q).  Returns r+ or a negative status. */
int orc_core_project(const double *A, int64_t n, int64_t lda, const double *Q,
                     int m, double *W)
{
    double *C = (double *)malloc(sizeof(double) * m * m);
    double *V = (double *)malloc(sizeof(double) * m * m);
    double *d = (double *)malloc(sizeof(double) * m);
    int st = core(A, n, lda, Q, m, 0.0, C);
    if (!st) st = orc_jacobi_eig(m, C, V, d, 1e-15, 100, NULL);
    int rp = st ? -st : factor(Q, n, m, V, d, 0, 0.0, W);
    free(C); free(V); free(d);
    return rp;
}

/* ------------------------------------------------------------------------ */
/* Error-bound terms, Eqs. (eps1) and (eps2).  sigma: values sorted in        */
/* decreasing order (length n).  k: target rank; p: oversampling (the          */
/* paper's l).                                                                 */
/* ------------------------------------------------------------------------ */
double orc_eps1(const double *sigma, int64_t n, int k, int p)
{
    double tail = 0.0;
    for (int64_t j = k; j < n; ++j) tail += sigma[j] * sigma[j];
    return sqrt((1.0 + (double)k / (double)(p - 1)) * tail);
}

double orc_eps2(double sigma, int64_t n, int k, int p, int q)
{
    double base = 1.0 + sqrt((double)k / (double)(p - 1)) +
                  M_E * sqrt((double)(k + p)) / (double)p * sqrt((double)(n - k));
    return pow(base, 1.0 / (2.0 * q + 1.0)) * sigma;
}

/* ------------------------------------------------------------------------ */
/* Gram-form Frobenius distances (no n x n matrix is formed).                 */
/*   ||W1 W1^T - W2 W2^T||_F^2 = ||W1^T W1||^2 - 2 ||W1^T W2||^2 + ||W2^T W2||^2 */
/* W1: n x m1, W2: n x m2, row-major.                                         */
/* ------------------------------------------------------------------------ */
static double gram_fro2(const double *X, int mx, const double *Y, int my, int64_t n)
{
    double tot = 0.0;
#pragma omp parallel for reduction(+ : tot) schedule(static)
    for (int a = 0; a < mx; ++a)
        for (int b = 0; b < my; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s += X[i * mx + a] * Y[i * my + b];
            tot += s * s;
        }
    return tot;
}

double orc_factor_dist2(const double *W1, int m1, const double *W2, int m2, int64_t n)
{
    return gram_fro2(W1, m1, W1, m1, n) - 2.0 * gram_fro2(W1, m1, W2, m2, n) +
           gram_fro2(W2, m2, W2, m2, n);
}

double orc_factor_norm2(const double *W, int m, int64_t n)
{
    return gram_fro2(W, m, W, m, n);
}

/* Apply U^T = (H_1 H_2 ... H_r)^T = H_r ... H_1 to the columns of X
 * (n x m row-major, in place), with H_t = I - 2 v_t v_t^T / (v_t^T v_t) and the
 * reflector vectors stored as rows of Vr (r x n). */
void orc_apply_Ut(const double *Vr, int r, int64_t n, double *X, int m)
{
    double *w = (double *)malloc(sizeof(double) * m);
    for (int t = 0; t < r; ++t) {
        const double *v = Vr + (int64_t)t * n;
        double vv = 0.0;
        for (int64_t i = 0; i < n; ++i) vv += v[i] * v[i];
        for (int c = 0; c < m; ++c) w[c] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < m; ++c) w[c] += v[i] * X[i * m + c];
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < m; ++c) X[i * m + c] -= 2.0 * v[i] * w[c] / vv;
    }
    free(w);
}

/* ||X+ - W W^T||_F^2 for A = U diag(lam) U^T, U = H_1 ... H_r:
 *   sum lam+^2 - 2 sum_i lam+_i ||(U^T W)_{i,:}||^2 + ||W^T W||_F^2. */
double orc_exact_dist2(const double *Vr, int r, const double *lam, int64_t n,
                       const double *W, int m)
{
    double *X = (double *)malloc(sizeof(double) * n * m);
    memcpy(X, W, sizeof(double) * n * m);
    orc_apply_Ut(Vr, r, n, X, m);
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double lp = lam[i] > 0.0 ? lam[i] : 0.0;
        s0 += lp * lp;
        double rn = 0.0;
        for (int c = 0; c < m; ++c) rn += X[i * m + c] * X[i * m + c];
        s1 += lp * rn;
    }
    free(X);
    return s0 - 2.0 * s1 + gram_fro2(W, m, W, m, n);
}

/* Closed-form exact projection of a generated matrix: P = U diag(lam+) U^T,
 * dense n x n row-major (O(n^2 r) through the reflectors). */
void orc_closed_form_proj(const double *Vr, int r, const double *lam, int64_t n,
                          double *P)
{
    /* start from diag(lam+) and apply P <- H P H for t = r..1 */
    memset(P, 0, sizeof(double) * n * n);
    for (int64_t i = 0; i < n; ++i) P[i * n + i] = lam[i] > 0.0 ? lam[i] : 0.0;
    double *w = (double *)malloc(sizeof(double) * n);
    for (int t = r - 1; t >= 0; --t) {
        const double *v = Vr + (int64_t)t * n;
        double vv = 0.0;
        for (int64_t i = 0; i < n; ++i) vv += v[i] * v[i];
        /* P <- P - (2/vv) v (v^T P) */
        for (int64_t j = 0; j < n; ++j) w[j] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) w[j] += v[i] * P[i * n + j];
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) P[i * n + j] -= 2.0 / vv * v[i] * w[j];
        /* P <- P - (2/vv) (P v) v^T */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += P[i * n + j] * v[j];
            for (int64_t j = 0; j < n; ++j) P[i * n + j] -= 2.0 / vv * s * v[j];
        }
    }
    free(w);
}
