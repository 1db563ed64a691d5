/*
 * psdproj.h -- C ABI of the GB300 (sm_103a) randomized PSD-projection library.
 *
 * Method: Jones & Anderson, "Approximate Projection onto the Positive
 * Semidefinite Cone Using Randomization" (arXiv 2410.19208).
 *   psdproj_alg1  = the paper's Alg. 2 (randomized PSD projection) with the
 *                   randomized range finder of Alg. 1 inside;
 *   psdproj_alg2  = the paper's Alg. 3 (scaled randomized PSD projection) with
 *                   alpha from Alg. 5 (min_eig, built on Alg. 4) unless given.
 * Naming: k is the target rank, p the oversampling (the paper's letter l),
 * l = k + p the sketch width, q the power-iteration exponent of Alg. 1.
 *
 * Memory conventions (all pointers prefixed d are DEVICE pointers on the
 * context's device; h are HOST pointers):
 *   A   n x n symmetric, FP32, row-major with leading dimension lda >= n.
 *       Only the upper triangle A[i*lda + j], j >= i, is ever read (BLAS
 *       uplo='U' in row-major terms); the strict lower triangle may hold
 *       anything, including NaN.
 *   P   n x n FP32 output, row-major, ldp >= n.
 *   tall matrices (Omega, Y, Q, W) are column-major n x c with leading
 *       dimension ld >= n: element (i, c) at X[c*ld + i].
 *   small matrices (Gram, R, core C, V) are column-major m x m, ld = m.
 * Ownership: the caller owns every pointer it passes; the context owns its
 * workspaces (allocated lazily, grown on demand, freed by psdproj_destroy).
 * Asynchrony: every compute call is enqueued on the context's stream and
 * returns without synchronising.  The return code reports argument, resource
 * and launch errors; errors found on the device (non-finite data, eigensolver
 * non-convergence) set a device status word read by psdproj_sync_status.
 * Thread safety: a context may be used by one host thread at a time.
 */
#ifndef PSDPROJ_H
#define PSDPROJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest sketch width l = k + p (and m of the per-step calls). */
#define PSDPROJ_MAX_M 512

/* ---- status codes ------------------------------------------------------- */
#define PSDPROJ_OK          0
#define PSDPROJ_EINVAL      1  /* bad argument (sizes, leading dims, NULL)     */
#define PSDPROJ_ENOMEM      2  /* device allocation failed, or it would exceed the
                                  context's device-memory budget (psdproj_create) */
#define PSDPROJ_ENOTFINITE  3  /* non-finite value met on the device            */
#define PSDPROJ_ENOCONV     4  /* the l x l eigensolver hit its sweep limit     */
#define PSDPROJ_ETIMEOUT    5  /* a bounded device wait gave up                 */
#define PSDPROJ_ECUDA       6  /* a CUDA runtime / launch error                 */
#define PSDPROJ_ENOTSUP     7  /* option not supported for these sizes         */
#define PSDPROJ_ETOOLARGE   8  /* size above a fixed scratch capacity          */

/* ---- precision of the A-passes (sketch, power and core products) -------- */
#define PSDPROJ_PREC_FP32    0 /* FP32 FMA on the CUDA cores (plain FP32)      */
#define PSDPROJ_PREC_TF32    1 /* tcgen05 kind::tf32 on a full TF32 image of A
                                  (both triangles), FP32 accumulation        */
#define PSDPROJ_PREC_BF16    2 /* tcgen05 kind::f16 on a BF16 image of A, FP32
                                  accumulation (see psdproj_alg1)              */
#define PSDPROJ_PREC_BF16X3  3 /* split-BF16: hi*hi + hi*lo + lo*hi, three
                                  tcgen05 passes over BF16 images of A_hi and
                                  A_lo = bf16(A - A_hi), FP32 accumulation    */

/* ---- output modes -------------------------------------------------------- */
#define PSDPROJ_OUT_FULL    0  /* P written in full (upper tiles mirrored)     */
#define PSDPROJ_OUT_UPPER   1  /* only P[i*ldp + j], j >= i, written           */
#define PSDPROJ_OUT_FACTOR  2  /* P not written; W = Q V sqrt(max(D,0)) only   */

/* Small eigensolver used for eig(Q^T X Q) (Alg. 2 line 2, Alg. 3 line 3) */
#define PSDPROJ_EIG_AUTO     0 /* tridiagonal solver, Jacobi when it flags a failure */
#define PSDPROJ_EIG_JACOBI   1 /* parallel cyclic Jacobi only                     */
#define PSDPROJ_EIG_TRIDIAG  2 /* tridiagonal solver only (failure: ENOCONV)      */

/* Test matrix Omega of the randomized range finder (Alg. 1) */
#define PSDPROJ_SKETCH_GAUSS 0 /* i.i.d. N(0,1) (psdproj_gaussian, stream 0)       */
#define PSDPROJ_SKETCH_SRHT  1 /* subsampled randomized Hadamard (psdproj_srht)     */

/* How psdproj_alg2 estimates alpha when alpha_in <= 0 */
#define PSDPROJ_ALPHA_MINEIG 0 /* Alg. 5 (two power iterations, 2(N+1) products)   */
#define PSDPROJ_ALPHA_RITZ   1 /* variant: -(most negative Ritz value) of the sketch
                                  Q0 = orth(A Omega), whose product A Omega is
                                  reused as the first product of Alg. 3: one
                                  extra pass over A instead of 2(N+1)          */

typedef struct psdproj_ctx psdproj_ctx;

typedef struct psdproj_opts {
    int prec;        /* PSDPROJ_PREC_* for the A-passes (default FP32)          */
    int syrk_prec;   /* PSDPROJ_PREC_FP32 or _BF16X3 for P = W W^T (default FP32)*/
    int N;           /* iterations of Alg. 4 inside Alg. 5 (default 10)          */
    int out_mode;    /* PSDPROJ_OUT_* (default FULL)                             */
    int eig;         /* PSDPROJ_EIG_* (default AUTO)                             */
    int sketch;      /* PSDPROJ_SKETCH_* test matrix of Alg. 1 (default GAUSS)   */
    int alpha_mode;  /* PSDPROJ_ALPHA_* estimate of alpha in Alg. 3 (default MINEIG) */
    int deterministic; /* 1: every product with A (passes and power iterations)
                          runs in a fixed summation order, in FP32 on the CUDA
                          cores (prec then applies to nothing but is checked),
                          so that a repeated call with the same inputs and
                          options returns bitwise the same P, W, rank and
                          alpha; such a pass reads each upper-triangle entry
                          twice.  0 (default): the faster forms, whose
                          cross-block sums are added in a timing-dependent
                          order (results agree to rounding). */
    int64_t spin_limit; /* SM clock cycles a device-side wait of the
                          tensor-core and power-iteration kernels may spin
                          for another part of its kernel before it gives up
                          and the call's device status becomes
                          PSDPROJ_ETIMEOUT (the kernel then waits for its own
                          copies and MMAs in flight, frees TMEM and returns);
                          0 (default): 4e9 cycles, about two seconds. */
    int reserved[2];   /* must be zero                                         */
} psdproj_opts;

/* Fill *o with the defaults listed above. */
void psdproj_default_opts(psdproj_opts *o);

/* Create a context bound to CUDA device `device` and CUDA stream `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  hbm_budget_bytes > 0
 * caps the device memory the context may hold for its workspaces, images
 * of A and host-call staging buffers (its batch helpers included, see
 * psdproj_workspace_bytes): a call that would grow them past the budget
 * returns PSDPROJ_ENOMEM before it launches anything; 0 = no cap.  Returns
 * a status. */
int psdproj_create(psdproj_ctx **ctx, int device, void *stream, size_t hbm_budget_bytes);
/* Re-bind the context to another stream of the same device. */
int psdproj_set_stream(psdproj_ctx *ctx, void *stream);
/* Free the context and its workspaces (synchronises its stream first). */
int psdproj_destroy(psdproj_ctx *ctx);
/* Synchronise the context's stream; return the first device-side status
 * recorded since the last call (then clear it), or a CUDA error. */
int psdproj_sync_status(psdproj_ctx *ctx);
/* Human-readable name of a status code (static storage). */
const char *psdproj_status_string(int status);
/* Bytes of device memory the context holds now: workspaces, the tensor-core
 * images of A, host-call staging buffers and those of its batch helpers
 * (the quantity the budget of psdproj_create caps). */
size_t psdproj_workspace_bytes(const psdproj_ctx *ctx);

/* Device bytes a context allocates to run one projection of side n with
 * sketch width k + p under opts (NULL = defaults): its workspace and the
 * image(s) of A of the form (or, with opts->deterministic, the partial-sum
 * scratch instead), as psdproj_workspace_bytes would count them; 0 for bad
 * sizes.  For sizing a budget (psdproj_create) or an admission footprint. */
size_t psdproj_projection_bytes(int64_t n, int k, int p, const psdproj_opts *opts);

/* ---- diagnostics --------------------------------------------------------- */
/* Stage classes timed by the context when timing is on. */
#define PSDPROJ_STAGE_APASS   0  /* symmetric passes Y = (A + s I) X           */
#define PSDPROJ_STAGE_GEMV    1  /* power-iteration products of Alg. 4          */
#define PSDPROJ_STAGE_ORTH    2  /* CholeskyQR2                                 */
#define PSDPROJ_STAGE_CORE    3  /* Q^T Z                                       */
#define PSDPROJ_STAGE_EIG     4  /* l x l eigensolver                           */
#define PSDPROJ_STAGE_FACTOR  5  /* W = Q V sqrt(D+)                            */
#define PSDPROJ_STAGE_SYRK    6  /* P = W W^T                                   */
#define PSDPROJ_STAGE_OTHER   7  /* Omega, alpha, copies                        */
#define PSDPROJ_STAGE_PACK    8  /* BF16 image of A (PSDPROJ_PREC_BF16)          */
#define PSDPROJ_NSTAGES       9

/* Turn per-stage CUDA-event timing on (1) or off (0).  When on, every stage
 * launched on the context's stream is bracketed by two events (at most 4096
 * stages between reads; later ones are not timed). */
int psdproj_timing_enable(psdproj_ctx *ctx, int on);
/* Synchronise the stream, add the elapsed milliseconds of every stage timed
 * since the last read into ms[kind] and their number into count[kind]
 * (arrays of nkinds entries, nkinds <= PSDPROJ_NSTAGES), then forget them. */
int psdproj_timing_read(psdproj_ctx *ctx, double *ms, int *count, int nkinds);
/* Number of kernels this library has launched in this process. */
uint64_t psdproj_kernel_launches(void);

/* ======================================================================== */
/* Whole projections                                                         */
/* ======================================================================== */

/* Randomized PSD projection (Alg. 2 with the range finder of Alg. 1):
 *   Omega = randn(n, k+p) (Philox4x32-10 stream 0 of `seed`),
 *   Q = orth(A^(2q+1) Omega), orthonormalised after every product (by
 *   one CholeskyQR pass where another product follows, which keeps the
 *   span and a well-conditioned basis; by CholeskyQR2 before the core),
 *   Q^T A Q = V D V^T,  W = Q V sqrt(max(D,0)),  P = W W^T.
 * Requires n >= 1, k >= 1, p >= 0, 1 <= k+p <= min(n, 512), 0 <= q <= 16,
 * lda >= n, ldp >= n (when P is written), ldw >= n (when dW != NULL).
 * dP may be NULL only with out_mode FACTOR.  dW (n x (k+p), column-major)
 * may be NULL; its columns beyond r+ are zero.  d_rank (device int, may be
 * NULL) receives r+, the number of positive eigenvalues of Q^T A Q.
 * opts may be NULL (defaults).  With opts->prec = PSDPROJ_PREC_BF16 the
 * call first packs A's block upper triangle into the
 * context's BF16 image (256 x 64 tiles stored contiguously, about n^2 + 128 n
 * bytes; kept for later calls) and every product with A, the power
 * iterations of psdproj_alg2 included, reads that image on the tensor cores
 * or CUDA cores with FP32 accumulation.  opts->prec = PSDPROJ_PREC_BF16X3
 * packs a second image of the residual A - bf16(A) (twice
 * the memory) and computes every product with A as A_hi X_hi + A_hi X_lo +
 * A_lo X_hi on the tensor cores (about 16 significant bits per product);
 * its power iterations run on the CUDA cores in FP32.  opts->prec =
 * PSDPROJ_PREC_TF32 packs a TF32 image of the full
 * symmetric matrix (lower triangle mirrored from the upper one; about
 * 4 n^2 bytes) and computes every product with A from it on the tensor cores
 * (10 fraction bits per operand, products exact in FP32); its power
 * iterations also run in FP32.  In the tensor-core forms a sketch wider than
 * 128 columns (k+p > 128) is multiplied in column slices of 128, one pass
 * over the image each, and with syrk_prec BF16X3 such a P = W W^T is written
 * by the FP32 kernel. */
int psdproj_alg1(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda,
                 int k, int p, int q, uint64_t seed,
                 float *dP, int64_t ldp, float *dW, int64_t ldw, int *d_rank,
                 const psdproj_opts *opts);

/* Scaled randomized PSD projection (Alg. 3):
 *   alpha = alpha_in if alpha_in > 0, else min_eig(A, N) (Alg. 5, start
 *   vectors from Philox streams 3 and 4 of `seed`), or with
 *   opts->alpha_mode = PSDPROJ_ALPHA_RITZ the variant
 *   alpha = -min(eig(Q0^T A Q0)), Q0 = orth(A Omega) (same Omega), whose
 *   product A Omega then serves as (A + alpha I) Omega - alpha Omega;
 *   Q = orth((A + alpha I)^(2q+1) Omega)  -- the range of B = (A+alpha I)/alpha,
 *   output Q (Q^T A Q)_+ Q^T, which equals the literal
 *   alpha Q V (max(D,1) - I) V^T Q^T with V D V^T = Q^T B Q (Lemma 4).
 * If alpha is not finite or alpha <= 1e-300 (A PSD and singular, or A = 0),
 * the call computes psdproj_alg1's output instead and sets bit 0 of
 * *d_info (device int, may be NULL).  d_alpha_out (device double, may be
 * NULL) receives the alpha used.  Other arguments as for psdproj_alg1. */
int psdproj_alg2(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda,
                 int k, int p, int q, uint64_t seed, double alpha_in,
                 double *d_alpha_out, int *d_info,
                 float *dP, int64_t ldp, float *dW, int64_t ldw, int *d_rank,
                 const psdproj_opts *opts);

/* A batch of independent projections (the many-small-matrices workload):
 * one descriptor per problem, each with its own A, sizes, seed, algorithm
 * and outputs (device pointers, meanings as in psdproj_alg1 /
 * psdproj_alg2).  The problems are spread over up to S helper streams of
 * the context (S = psdproj_set_batch_streams, default 8), each with its own
 * workspace: longest-processing-time-first assignment on the cost n^2 x
 * (passes over A), largest problems issued first.  The helper streams start
 * after the work already queued on the context's stream and the context's
 * stream waits for all of them, so the call is asynchronous on that stream
 * like the others; device errors of any problem land in the context's status
 * word.  With S = 1 the problems run in order on the context's stream.  The
 * call returns the first argument error (nothing runs then) or the first
 * launch error.  opts applies to every problem. */
typedef struct psdproj_problem {
    const float *dA;     /* n x n FP32 row-major, upper triangle read       */
    int64_t n, lda;
    int k, p, q;
    int algorithm;       /* 1: psdproj_alg1 (Alg. 2), 2: psdproj_alg2 (Alg. 3) */
    uint64_t seed;
    double alpha_in;     /* Alg. 3 only; <= 0: estimate by min_eig            */
    double *d_alpha_out; /* Alg. 3 only, may be NULL                          */
    int *d_info;         /* Alg. 3 only, may be NULL                          */
    float *dP;           /* may be NULL with out_mode FACTOR                  */
    int64_t ldp;
    float *dW;           /* may be NULL                                       */
    int64_t ldw;
    int *d_rank;         /* may be NULL                                       */
} psdproj_problem;
int psdproj_batched(psdproj_ctx *ctx, int count, const psdproj_problem *probs,
                    const psdproj_opts *opts);

/* psdproj_batched with the batch's launches recorded once in a CUDA graph
 * and replayed: the first call with a given problem table (the descriptors
 * compared byte for byte), options, helper-stream count and reserved SMs
 * allocates every workspace and image the batch needs, records the whole
 * batch (its fork to the helper streams, every projection, the join) into a
 * graph kept by the context and launches it; a later call with the same
 * table and settings launches that graph again, with no per-projection host
 * work.  A call with a different table records a new graph in place of the
 * old one.  The graph reads and writes the buffers the table names, so it
 * replays only while those pointers stay valid.  Stage timing is not
 * recorded into the graph.  Results and errors as for psdproj_batched; the
 * context's stream must not be capturing already. */
int psdproj_batched_graph(psdproj_ctx *ctx, int count, const psdproj_problem *probs,
                          const psdproj_opts *opts);

/* The same batch with its small steps grouped: every problem gets a
 * workspace and image of its own (one allocation held by the context, sized
 * to the sum of the problems' psdproj_projection_bytes), and the batch runs
 * phase by phase, each phase for all problems before the next: the BF16
 * images, alpha (Alg. 3: the power iterations of Alg. 5) and Omega as
 * grouped launches (other forms and options per problem), Y = (A + shift I)
 * Omega per problem on the helper streams; then each of Alg. 1's
 * orthonormalisations (Gram, Cholesky, tall x small product; before the core
 * a second such pass: CholeskyQR2) as grouped launches over the problems
 * whose product it follows; the power and core products per problem on the
 * helper streams; the core Q^T A Q, the l x l eigensolver (Alg. 2) and the
 * factor W = Q V sqrt(max(D, 0)) as grouped launches; P = W W^T per
 * problem.  A grouped launch runs, for each problem, the blocks its own
 * launch would run, so results equal psdproj_batched's up to the order of
 * the passes' floating-point additions.  Recorded once into a CUDA graph and
 * replayed like psdproj_batched_graph (same rules for the table, settings
 * and buffers).  Requires k + p <= 128 in every problem (else
 * PSDPROJ_ENOTSUP) and opts.deterministic = 0 (else PSDPROJ_ENOTSUP).  The
 * first call of a table synchronises the context's stream.  A batch of 32
 * problems or more is recorded as two halves (alternating in decreasing
 * cost), each with half of the helper streams and its own chain of grouped
 * launches on a stream of the context's, so that one half's grouped steps
 * overlap the other half's per-problem products; the environment variable
 * PSDPROJ_GROUPED_SPLIT=1, read when a batch is recorded, keeps it whole. */
int psdproj_batched_grouped(psdproj_ctx *ctx, int count, const psdproj_problem *probs,
                            const psdproj_opts *opts);

/* Number of helper streams psdproj_batched spreads a batch over (1..64,
 * default 8; 1 = the context's own stream only).  Each helper holds its own
 * workspace, sized for the largest problem it has run. */
int psdproj_set_batch_streams(psdproj_ctx *ctx, int streams);

/* Batch autotuning.  psdproj_tune_batch runs `probs` (as psdproj_batched_graph
 * does) on 2, 4, 8, 16, 32 and 64 helper streams, one recording run and `reps` timed
 * replays each on the context's stream, keeps the fastest, sets it on the
 * context (as psdproj_set_batch_streams) and stores it in the tuning table
 * under the batch's bucket: (device name, SM count, floor(log2 of the median
 * side), floor(log2 of count)).  Synchronises the context's stream; the
 * results in P and W are those of the last run.  *best_streams and *best_ms
 * (time per batch; either may be NULL) report the choice.
 *
 * psdproj_batched and psdproj_batched_graph use, in this order: the
 * environment variable PSDPROJ_BATCH_STREAMS (1..64); the context's own lane
 * count if set; the tuning table's entry for the batch's bucket; the default
 * 8.  The table lives in the process and, when PSDPROJ_TUNE_CACHE names a
 * file, in that file (one "key<TAB>streams" line per entry; when the
 * variable names another file the table becomes that file's contents; every
 * store rewrites the file).  psdproj_tune_lookup
 * (EINVAL when there is no entry) and psdproj_tune_store read and write it
 * directly; neither needs a GPU. */
int psdproj_tune_batch(psdproj_ctx *ctx, int count, const psdproj_problem *probs,
                       const psdproj_opts *opts, int reps, int *best_streams, double *best_ms);
int psdproj_tune_lookup(const char *device_name, int sm_count, int64_t median_n, int count,
                        int *streams);
int psdproj_tune_store(const char *device_name, int sm_count, int64_t median_n, int count,
                       int streams);

/* SMs that this context's persistent kernels (the tensor-core passes, the
 * BF16 power iteration, the SYRK) leave free: 0 .. SMs - 1, default 1; also
 * applied to the context's batch helpers.  A persistent grid that finds no
 * free SM for one of its CTAs runs that CTA only when another finishes, so
 * when several contexts run projections on one GPU at once, their
 * single-block steps (Cholesky, eigensolver) need SMs that the others'
 * grids do not take: two per concurrent context measured best for four
 * contexts (4 % more projections/s than the default).  Returns
 * PSDPROJ_EINVAL for a null context or a count outside that range. */
int psdproj_set_reserved_sms(psdproj_ctx *ctx, int sms);

/* ---- dual gradient descent for semidefinite least squares (Alg. 6) ------
 *   min over PSD X of 1/2 ||X - C/rho||_F^2   s.t.  <A_i, X> = b_i, i < mc.
 * Each iteration t forms X_t = C/rho + sum_i y_i A_i (upper triangle; the
 * minimiser of the partial Lagrangian is (X_t)_+), projects it with
 * psdproj_alg1 (algorithm 1, the paper's Alg. 2) or psdproj_alg2 (algorithm
 * 2, Alg. 3; alpha as opts->alpha_mode says) in factor form W (sketch seed
 * = seed + t; with warm_start the test matrix of iteration t > 0 is the
 * previous iteration's orthonormal basis Q, columns that its
 * orthonormalisation dropped replaced by the Gaussian columns of seed + t),
 * takes grad_i = <A_i, W W^T> - b_i (FP32 passes, FP64 sums) and steps
 * y <- y - beta grad.  It stops after the first iteration whose ||grad||_2
 * <= eps, or after max_iter iterations.  Synchronous: the gradient is read
 * back every iteration.  */
typedef struct psdproj_sdls {
    const float *dC;             /* n x n symmetric, row-major (ld), upper read */
    const float *const *dA;      /* HOST array of mc DEVICE pointers, n x n each */
    const double *b;             /* host, mc                                   */
    int64_t n, ld;               /* n <= 65535                                 */
    double rho, beta, eps;       /* rho > 0, step beta > 0, tolerance eps >= 0 */
    uint64_t seed;
    int mc, k, p, q;             /* constraints; sketch of each projection     */
    int algorithm;               /* 1 or 2                                     */
    int max_iter;                /* >= 1                                       */
    int warm_start;              /* 0 or 1                                     */
    int reserved;                /* must be zero                               */
} psdproj_sdls;
/* y (host, mc): the initial multipliers in, the final ones out.  dX (device,
 * may be NULL): the last iterate's projection W W^T, n x n row-major (ldx);
 * its syrk_prec as in opts.  *iters (may be NULL): iterations run;
 * *grad_norm (may be NULL): the last ||grad||; grad_hist (host, max_iter
 * doubles, may be NULL): ||grad|| per iteration.  Returns device errors
 * (non-finite data, ...) as their status. */
int psdproj_sdls_dual_gd(psdproj_ctx *ctx, const psdproj_sdls *problem, double *y, float *dX, int64_t ldx,
                         int *iters, double *grad_norm, double *grad_hist, const psdproj_opts *opts);

/* The cudaError_t behind the last PSDPROJ_ECUDA / ENOMEM / ENOTSUP that a
 * call on this host thread returned (0 if none), and in *line (may be NULL)
 * the line of the library's C-ABI source where it was seen. */
int psdproj_last_cuda_error(int *line);

/* ---- request server (the served workload) --------------------------------
 * Independent projections submitted by any host thread and run by `workers`
 * threads, each with its own context and CUDA stream on `device`.  A request
 * holds device pointers the caller owns until psdproj_server_wait reports it
 * done.  Admission is first come, first served under a device-memory budget:
 * the request at the head of the queue starts when its footprint
 * (footprint_bytes, or when 0 the bytes of its A, P and W plus
 * psdproj_projection_bytes for its size and the server's opts) fits under
 * admit_bytes together with the admitted requests not yet finished; later
 * requests wait behind it.  Each request's status is its own: the worker
 * reads and clears its context's device status word after the request.  Not
 * thread-safe against psdproj_server_destroy. */
typedef struct psdproj_server psdproj_server;
typedef struct psdproj_request {
    const float *dA;     /* n x n FP32 row-major, upper triangle read         */
    int64_t n, lda;
    int k, p, q;
    int algorithm;       /* 1: psdproj_alg1 (Alg. 2), 2: psdproj_alg2 (Alg. 3) */
    uint64_t seed;
    double alpha_in;     /* Alg. 3 only; <= 0: estimate by min_eig              */
    double *d_alpha_out; /* Alg. 3 only, may be NULL                            */
    int *d_info;         /* Alg. 3 only, may be NULL                            */
    float *dP;           /* may be NULL with out_mode FACTOR                    */
    int64_t ldp;
    float *dW;           /* may be NULL                                         */
    int64_t ldw;
    int *d_rank;         /* may be NULL                                         */
    int64_t footprint_bytes; /* device bytes held while admitted; 0: A + P + W and
                                the context memory (psdproj_projection_bytes) */
} psdproj_request;
typedef struct psdproj_server_stats {
    uint64_t submitted, completed, failed;
    int64_t queued;              /* waiting for admission                     */
    int64_t running;             /* admitted, not finished                    */
    int64_t inflight_bytes;      /* footprints of the admitted, unfinished    */
    int64_t inflight_peak_bytes; /* largest inflight_bytes seen               */
    int64_t admit_bytes;
    int last_error_status;       /* status of the last failed request         */
    int last_error_cuda;         /* its psdproj_last_cuda_error (0: none)     */
    int last_error_line;
    int reserved;
} psdproj_server_stats;
/* opts (may be NULL) applies to every request.  EINVAL: workers outside
 * 1..64, admit_bytes 0 or bad opts. */
int psdproj_server_create(psdproj_server **srv, int device, int workers, size_t admit_bytes,
                          const psdproj_opts *opts);
/* Queue a request (never blocks on the device).  *ticket identifies it.
 * EINVAL: bad sizes, algorithm or pointers (as psdproj_alg1/2 would report);
 * ETOOLARGE: its footprint exceeds admit_bytes. */
int psdproj_server_submit(psdproj_server *srv, const psdproj_request *req, uint64_t *ticket);
/* Wait up to timeout_s seconds (0: poll) for a request.  PSDPROJ_OK: done;
 * *status = its result (PSDPROJ_OK or the error of the call or of the
 * device), *latency_ms = submit to completion; the ticket is then released.
 * ETIMEOUT: not done yet; EINVAL: unknown or already collected ticket. */
int psdproj_server_wait(psdproj_server *srv, uint64_t ticket, double timeout_s, int *status,
                        double *latency_ms);
/* Wait up to timeout_s seconds until nothing is queued or running (ETIMEOUT
 * otherwise). */
int psdproj_server_drain(psdproj_server *srv, double timeout_s);
int psdproj_server_get_stats(psdproj_server *srv, psdproj_server_stats *stats);
/* Requests not yet admitted are dropped; admitted ones finish first. */
int psdproj_server_destroy(psdproj_server *srv);

/* Host-buffer forms of the two calls: hA, hP, hW, h_rank are HOST pointers
 * (pinned memory recommended).  From pinned host memory the device reads
 * only A's upper triangle, over the host link: the BF16 form packs its image
 * straight from it, the other forms gather it into a context-owned device
 * buffer; other host memory is copied whole.  The call then runs the
 * projection, copies P (and W, r+) back, and synchronises the stream before
 * returning.  Returns the first error, device-side status
 * included. */
int psdproj_alg1_host(psdproj_ctx *ctx, const float *hA, int64_t n, int64_t lda,
                      int k, int p, int q, uint64_t seed,
                      float *hP, int64_t ldp, float *hW, int64_t ldw, int *h_rank,
                      const psdproj_opts *opts);
int psdproj_alg2_host(psdproj_ctx *ctx, const float *hA, int64_t n, int64_t lda,
                      int k, int p, int q, uint64_t seed, double alpha_in,
                      double *h_alpha_out,
                      float *hP, int64_t ldp, float *hW, int64_t ldw, int *h_rank,
                      const psdproj_opts *opts);

/* ======================================================================== */
/* Steps of the path (each one kernel or a short chain of kernels)           */
/* ======================================================================== */

/* Test matrix of Alg. 1 ("Omega = randn"): dX[c*ldx + i] = N(0,1) sample keyed
 * by Philox4x32-10 counter (i, c, stream, 0) and key (seed lo, seed hi), by
 * Box-Muller (cosine branch) on output words 0 and 1, for i < n, c < m.
 * Requires n >= 1, 1 <= m, ldx >= n. */
int psdproj_gaussian(psdproj_ctx *ctx, uint64_t seed, uint32_t stream,
                     int64_t n, int m, float *dX, int64_t ldx);

/* Structured test matrix, the real counterpart of the subsampled randomized
 * Fourier transform that the footnote to Alg. 1 names: with N the smallest
 * power of two >= n,
 *   dX[c*ldx + i] = d_i * (-1)^popcount(i & s_c),   i < n, c < m,
 * i.e. rows 0..n-1 of D H_N S: d_i = -1 exactly when bit 0 of output word 0
 * of Philox4x32-10 (counter (i, 0, 17, 0), key = seed) is 1; s_c is the
 * first value of word 0 of Philox(counter (c, t, 16, 0)) mod N, t = 0, 1, ...,
 * not taken by a column before c (so the m columns of H_N are distinct).
 * Entries are exactly +-1 (exact in every operand format).  Requires
 * 1 <= m <= min(n, 512), ldx >= n. */
int psdproj_srht(psdproj_ctx *ctx, uint64_t seed, int64_t n, int m, float *dX, int64_t ldx);

/* Symmetric pass over A (Alg. 1 products, and Z = A Q of Alg. 2 line 2):
 *   dY = A dX + shift dX,   shift = (d_shift ? *d_shift : 0),
 * reading only the upper triangle of A.  dX, dY are n x m column-major
 * (ldx, ldy >= n); dY is overwritten.  prec PSDPROJ_PREC_FP32: CUDA cores,
 * A read once.  PSDPROJ_PREC_BF16: A's block upper triangle is first packed
 * into the context's BF16 image (4 bytes read, 2 written per entry), which
 * the tensor-core pass then reads.  PSDPROJ_PREC_BF16X3: a second image
 * holds bf16(A - A_hi) and three tensor-core passes add A_hi X_hi +
 * A_hi X_lo + A_lo X_hi into dY.  PSDPROJ_PREC_TF32: A's upper triangle is
 * mirrored into a full TF32 image (4 bytes written per entry of the n x n
 * matrix) and one tensor-core pass reads it.  The tensor-core passes take
 * 128 columns at a time: wider X runs as column slices. */
int psdproj_sym_pass(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda,
                     const float *dX, int64_t ldx, int m, const double *d_shift,
                     float *dY, int64_t ldy, int prec);

/* Orthonormalisation of Alg. 1 (QR 'econ') by CholeskyQR2: G = Y^T Y with
 * FP32 products accumulated in FP64, R = chol(G) in FP64, Q = Y R^-1, done
 * twice.  A column whose pivot R_jj^2 <= 1e-10 * max_i G_ii is dependent: its
 * Q column is set to zero.  dY (input) and dQ (output) are n x m column-major;
 * they may alias.  d_qrank (device int, may be NULL) receives the number of
 * independent columns.  Requires 1 <= m <= 512. */
int psdproj_cholqr2(psdproj_ctx *ctx, const float *dY, int64_t n, int64_t ldy,
                    int m, float *dQ, int64_t ldq, int *d_qrank);

/* Projected core of Alg. 2 line 2: dC = (X^T Z + Z^T X) / 2 (m x m FP64,
 * column-major), with FP32 products accumulated in FP64. */
int psdproj_core(psdproj_ctx *ctx, const float *dX, int64_t ldx, const float *dZ,
                 int64_t ldz, int64_t n, int m, double *dC);

/* Small symmetric eigensolver of Alg. 2 line 2 ("eig(Q^T X Q)") on dC (m x m
 * FP64 in, read only), in FP32 in one thread block.  dV (m x m column-major
 * FP32) receives orthonormal eigenvectors, dd (m doubles) the eigenvalues;
 * eigenpairs are sorted by decreasing eigenvalue.  Requires 1 <= m <= 512.
 * psdproj_eig uses PSDPROJ_EIG_AUTO: Householder tridiagonalization,
 * bisection, twisted-factorization eigenvectors and one Newton-Schulz
 * orthogonalization step; when that solver flags a failure (a non-finite or
 * inaccurate vector, V^T V far from I) the Jacobi solver recomputes the
 * result on the device.  Jacobi non-convergence, or a failure of the
 * tridiagonal solver under PSDPROJ_EIG_TRIDIAG, sets PSDPROJ_ENOCONV in the
 * device status. */
int psdproj_eig(psdproj_ctx *ctx, const double *dC, int m, float *dV, double *dd);
/* As psdproj_eig with the solver chosen by `method` (PSDPROJ_EIG_*). */
int psdproj_eig_method(psdproj_ctx *ctx, const double *dC, int m, float *dV, double *dd,
                       int method);

/* Factor of Alg. 2 line 3: dW = Q V diag(sqrt(max(d, 0))) (n x m, column-
 * major; the r+ columns with d > 0 first, zero columns after), and *d_rank =
 * r+.  dV, dd as produced by psdproj_eig (sorted decreasingly). */
int psdproj_factor(psdproj_ctx *ctx, const float *dQ, int64_t ldq, int64_t n,
                   int m, const float *dV, const double *dd, float *dW,
                   int64_t ldw, int *d_rank);

/* Reconstruction P = W W^T (Alg. 2 line 3) over the first *d_rank columns of
 * dW (device int; NULL = all m).  out_mode FULL writes all of P, UPPER only
 * j >= i.  prec: PSDPROJ_PREC_FP32 or PSDPROJ_PREC_BF16X3. */
int psdproj_syrk(psdproj_ctx *ctx, const float *dW, int64_t ldw, int64_t n,
                 int m, const int *d_rank, float *dP, int64_t ldp,
                 int out_mode, int prec);

/* min_eig of Alg. 5 on the device: sigma1 = power_iteration(A, N) (Alg. 4,
 * start vector stream 3), sigma2 = power_iteration(A - sigma1 I, N) (stream
 * 4), alpha = |sigma1 - sigma2|.  Each power iteration makes N + 1 symmetric
 * matrix-vector passes over the upper triangle with FP64 norms.  Outputs are
 * device doubles; d_sigma1 and d_sigma2 may be NULL. */
int psdproj_min_eig(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda,
                    int N, uint64_t seed, double *d_alpha, double *d_sigma1,
                    double *d_sigma2);

/* Allocation-free min_eig (no counterpart in the paper; same result as
 * psdproj_min_eig).  For callers that cannot call cudaMalloc: code running
 * under another library's memory manager or a caching allocator that forbids
 * allocations in its hot path, plug-ins whose host cannot grant device
 * allocations, or processes whose device memory is reserved up front.  It
 * needs no context and allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine): its scratch is a fixed device array of
 * 2 * PSDPROJ_NOALLOC_MAX_N floats plus a few scalars, held by every GPU that
 * loads this library until the process exits.
 *   dA: device, n x n FP32 row-major (upper triangle read), lda >= n;
 *   n <= PSDPROJ_NOALLOC_MAX_N, otherwise PSDPROJ_ETOOLARGE and nothing runs;
 *   d_alpha (required), d_sigma1, d_sigma2 (may be NULL): device doubles;
 *   stream: the cudaStream_t to enqueue on (NULL = legacy default stream).
 * The first call on a device (with that device current) looks up the device
 * address of the scratch array and keeps it for later calls; make that first
 * call before any stream capture.  The kept address does not survive a reset
 * of the device's primary context (cudaDeviceReset): do not call this entry
 * point again in a process after such a reset.  dA must be device memory of
 * the current device (otherwise PSDPROJ_EINVAL) and stream a stream of it.  Every call shares the one array per device and leaves its
 * contents behind: calls that overlap on the GPU (other streams, or
 * concurrent host threads) race and must be serialised by the caller.
 * Errors found on the host are returned; nothing is synchronised. */
#define PSDPROJ_NOALLOC_MAX_N 131072
int psdproj_min_eig_noalloc(const float *dA, int64_t n, int64_t lda, int N, uint64_t seed,
                            double *d_alpha, double *d_sigma1, double *d_sigma2, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PSDPROJ_H */
