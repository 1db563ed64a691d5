// Internal declarations of the psdproj CUDA library (sm_103a).
// The context, its workspace layout and the kernel launchers used by capi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/psdproj.h"

// Device status word: the first error code recorded wins.
__device__ __forceinline__ void psd_set_status(int *st, int code)
{
    if (st) atomicCAS(st, 0, code);
}

static inline int64_t psd_round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Tall-matrix leading dimension used for context-owned buffers: rows padded
// to a multiple of 128 (TMA strides stay 16-byte aligned, tiles never read
// past the allocation).
static inline int64_t psd_ld(int64_t n) { return psd_round_up(n, 128); }
// Sketch width padded to a multiple of 16 (UMMA N granularity at M = 128).
static inline int psd_lpad(int m) { return (int)psd_round_up(m, 16); }

constexpr int PSD_GRAM_CHUNK = 64;    // rows per Gram partial

// Tiles of the BF16 image of A (tensor-core pass and BF16 power iteration):
// the block upper triangle of A in tiles of 256 rows x 64 columns, stored
// tile after tile in row-major tile order (block row I holds the tiles
// J = 4 I .. nbc - 1), each tile 32 KB in the 128-byte-swizzled layout of a
// UMMA operand: row r at r * 128 bytes, its 16-byte chunk k (columns
// 8k..8k+7) at position k ^ (r & 7) within the row.
constexpr int PSD_TILE_M = 256, PSD_TILE_N = 64;
constexpr int PSD_TILE_R = PSD_TILE_M / PSD_TILE_N;
constexpr int64_t PSD_TILE_ELEMS = (int64_t)PSD_TILE_M * PSD_TILE_N;
constexpr int64_t PSD_TILE_BYTES = 32768;
// first tile of block row I (nbc = 64-column tiles of the padded matrix)
__host__ __device__ inline int64_t psd_tile_row_start(int I, int nbc)
{
    return (int64_t)I * nbc - (int64_t)PSD_TILE_R * I * (I - 1) / 2;
}
__host__ __device__ inline int64_t psd_tile_count(int64_t n)
{
    const int nbr = (int)((n + PSD_TILE_M - 1) / PSD_TILE_M);
    return psd_tile_row_start(nbr, nbr * PSD_TILE_R);
}
// The TF32 image holds the FULL symmetric matrix (both triangles, the lower
// one mirrored from the upper) in tiles of 256 x 32 FP32 entries rounded to
// TF32, again 128-byte swizzled rows (chunk k = columns 4k..4k+3), tile
// (I, J) at index I * nbc + J with nbc = 8 * nbr.
constexpr int PSD_TILE32_N = 32;
__host__ __device__ inline int64_t psd_tile32_count(int64_t n)
{
    const int64_t nbr = (n + PSD_TILE_M - 1) / PSD_TILE_M;
    return nbr * nbr * (PSD_TILE_M / PSD_TILE32_N);
}
constexpr int PSD_MAX_M = PSDPROJ_MAX_M;  // largest sketch width

struct psd_workspace {
    int64_t n = 0;      // rows the tall buffers hold
    int lpad = 0;       // columns they hold
    int64_t ld = 0;     // their leading dimension
    void *base = nullptr;
    size_t bytes = 0;
    // tall FP32 buffers, ld x lpad each
    float *Om = nullptr, *Y = nullptr, *Q = nullptr, *T = nullptr, *W = nullptr;
    // bf16 hi / lo images of a tall buffer (tensor-core passes)
    uint16_t *Xhi = nullptr, *Xlo = nullptr;
    float *Xf = nullptr;  // X rounded to TF32 (TF32 pass operand)
    // Gram partials: nchunk x lpad x lpad floats
    float *gpart = nullptr;
    // small matrices
    double *G = nullptr, *R = nullptr, *C = nullptr, *d = nullptr, *cholscr = nullptr;
    float *Rinv = nullptr, *V = nullptr, *M = nullptr, *eigscr = nullptr;
    int *dead = nullptr;
    // power iteration: two n-vectors (ld floats) and scalars
    float *pv0 = nullptr, *pv1 = nullptr, *pv2 = nullptr;   // power-iteration vectors (a rotation of three)
    double *scal = nullptr;     // 16 doubles
    int *ints = nullptr;         // 16 ints (ranks, info)
    int *picks = nullptr;        // PSD_MAX_M ints (SRHT column picks)
};

constexpr int PSD_MAX_TIMED = 4096;

struct psd_timing {
    int on = 0;
    int n = 0;                       // stages recorded since the last read
    bool created = false;
    cudaEvent_t ev[2 * PSD_MAX_TIMED];
    int kind[PSD_MAX_TIMED];
};

constexpr int PSD_MAX_LANES = 64;     // most streams a batch is spread over

struct psdproj_ctx {
    int device = 0;
    psd_timing timing;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int persist_sms = 0;         // grid of the persistent kernels
    int *d_status = nullptr;     // device status word
    psd_workspace ws;
    // host-API staging buffers
    float *dA_stage = nullptr;  size_t dA_stage_bytes = 0;
    float *dP_stage = nullptr;  size_t dP_stage_bytes = 0;
    float *dW_stage = nullptr;  size_t dW_stage_bytes = 0;
    int *d_misc = nullptr;       // rank / info for host calls
    double *d_misc_f = nullptr;  // alpha for host calls
    // BF16 image of the block upper triangle of A (tensor-core passes)
    uint16_t *Ab = nullptr;
    size_t Ab_bytes = 0;
    uint16_t *Ab_lo = nullptr;   // low parts (split-BF16 form)
    size_t Ab_lo_bytes = 0;
    // psdproj_batched: helper contexts ("lanes"), each with its own stream,
    // workspace and images, sharing this context's status word; the batch
    // forks from `stream` to the lanes and joins back by events
    int batch_streams = 8;
    bool lanes_explicit = false; // set by psdproj_set_batch_streams or psdproj_tune_batch
    int tune_force = 0;          // psdproj_tune_batch: lane count under trial (0: none)
    psdproj_ctx *lane[PSD_MAX_LANES] = {};
    cudaEvent_t lane_ev[PSD_MAX_LANES + 1] = {};
    bool owns_status = true;     // false for a lane (the status word is its parent's)
    bool owns_stream = false;    // true for a lane (stream created by the library)
    // device-memory budget (psdproj_create): held by this context and its
    // lanes together; a lane's root is its parent, a context's is itself
    size_t budget = 0;           // 0: no cap
    psdproj_ctx *root = nullptr;
    long long wait_limit = 0;    // opts.spin_limit of the call in progress
    bool det = false;            // opts.deterministic of the call in progress
    // partial sums of the deterministic products (psd_det_part_floats)
    float *det_part = nullptr;  size_t det_part_bytes = 0;
    // psdproj_batched_graph: the recorded batch and what it was recorded for
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<psdproj_problem> graph_probs;
    psdproj_opts graph_opts = {};
    int graph_streams = 0, graph_persist = 0;
    uint64_t graph_launches = 0;     // kernels in the graph (counted per replay)
    cudaStream_t capture_stream = nullptr;   // the stream a graph is recorded on
    // psdproj_batched_grouped: a workspace and image(s) per problem (g_slots)
    // and the grouped launches' tables (g_tabs); the recorded batch and what
    // it was recorded for
    // (the batch in up to two halves, each with its own slots and tables;
    // the second half's grouped launches on g_stream2, forked from and
    // joined back to the context's stream by g_ev)
    void *g_slots[2] = {};    size_t g_slots_bytes[2] = {};
    void *g_tabs[2] = {};     size_t g_tabs_bytes[2] = {};
    cudaStream_t g_stream2 = nullptr;
    cudaEvent_t g_ev[2] = {};
    cudaGraphExec_t g_exec = nullptr;
    std::vector<psdproj_problem> g_probs;
    psdproj_opts g_opts = {};
    int g_streams = 0, g_persist = 0;
    uint64_t g_launches = 0;
};

// PSDPROJ_OK when the budget of ctx's root allows replacing `old_bytes` of
// device memory by `new_bytes`, else PSDPROJ_ENOMEM.
int psd_budget_check(const psdproj_ctx *ctx, size_t old_bytes, size_t new_bytes);

// Make sure the workspace holds n rows x m columns; may synchronise the
// stream and reallocate.  Returns a PSDPROJ_* status.
int psd_ensure_workspace(psdproj_ctx *ctx, int64_t n, int m);
// Device bytes a context allocates for one projection of side n and sketch
// width m in form prec: its workspace and image(s) of A (or, deterministic,
// the partial sums instead of the images).
size_t psd_projection_device_bytes(int64_t n, int m, int prec, int deterministic);

// ---- launchers (all asynchronous on `s`; return cudaGetLastError) -------
// Side outputs of a kernel that writes a tall matrix Z (n x m) which the
// BF16 tensor-core pass reads next: Xh = bf16(Z) (column-major, ldh >= n)
// and Y = shift Z with shift = *d_shift (Y = 0 when d_shift is NULL; ldy >=
// n), both over rows < n and columns < m, so that the pass needs no
// conversion sweep of its own.  Xh / Y may be NULL.
struct psd_bf16_side {
    uint16_t *Xh;
    int64_t ldh;
    float *Y;
    int64_t ldy;
    const double *d_shift;
    // the tall x small product only (may be NULL): also the low parts
    // bf16(Z - bf16(Z)) at leading dimension ldh, the split-BF16 SYRK's
    // second operand
    uint16_t *Xl;
};

cudaError_t launch_gaussian(cudaStream_t s, uint64_t seed, uint32_t stream_id,
                            int64_t n, int m, int mpad, int64_t rows_pad,
                            float *X, int64_t ldx, const psd_bf16_side *side = nullptr);

// D[i*ldd + j] = S[i*lds + j] for j >= i (the upper triangle; S may be
// pinned host memory read over the host link)
cudaError_t launch_copy_upper(cudaStream_t s, const float *S, int64_t n, int64_t lds, float *D, int64_t ldd);

// alpha = -min(d) (Ritz values of an unshifted sketch's core), shift and
// info as launch_alpha_finish; Y += shift X (n x m, leading dimension ld)
cudaError_t launch_ritz_alpha(cudaStream_t s, const double *d, int m, double *d_alpha, double *d_shift,
                              int *d_info);
cudaError_t launch_add_shift(cudaStream_t s, float *Y, const float *X, int64_t n, int m, int64_t ld,
                             const double *d_shift);

// Alg. 6 (dual gradient descent for semidefinite least squares):
// X = C / rho + sum_i y_i A_i on the upper triangle (dA: device array of mc
// device pointers, y: device doubles; n <= 65535); g += <W, Z> (FP64);
// Om[:, c] = Q[:, c] where dead[c] == 0.
cudaError_t launch_sdls_combine(cudaStream_t s, const float *C, const float *const *dA, int mc, const double *y,
                                double rho, int64_t n, int64_t ld, float *X, int64_t ldx);
cudaError_t launch_sdls_dot(cudaStream_t s, const float *W, const float *Z, int64_t n, int m, int64_t ld,
                            double *g);
cudaError_t launch_sdls_warm_omega(cudaStream_t s, float *Om, const float *Q, const int *dead, int64_t n,
                                   int m, int64_t ld);

// Philox streams of the SRHT test matrix: column picks and row signs
constexpr uint32_t PSD_SRHT_PICKS = 16u, PSD_SRHT_SIGNS = 17u;
// SRHT test matrix (see gauss.cu); picks: m ints of device scratch; n >= m.
cudaError_t launch_srht(cudaStream_t s, uint64_t seed, int64_t n, int m, int mpad, int64_t rows_pad,
                        int *picks, int *d_status, float *X, int64_t ldx);

cudaError_t launch_sym_pass_simt(cudaStream_t s, const float *A, int64_t n, int64_t lda,
                                 const float *X, int64_t ldx, int m, const double *d_shift,
                                 float *Y, int64_t ldy);

// BF16 image A' of the block upper triangle of A (256 x 256 diagonal blocks
// strictly upper, diagonal halved, zero below; A = A' + A'^T), in the tile
// layout described with PSD_TILE_M (psd_tile_count(n) tiles of 32 KB), zero
// padded past row / column n.  Ab 16-byte aligned.
// part 1: the low parts bf16(a - bf16(a)) instead (split-BF16 form).
cudaError_t launch_pack_bf16(cudaStream_t s, const float *A, int64_t n, int64_t lda, uint16_t *Ab,
                             int part);

// TF32 image of the full symmetric matrix (psd_tile32_count(n) tiles; the
// lower triangle is mirrored from the upper one, which alone is read).
cudaError_t launch_pack_tf32(cudaStream_t s, const float *A, int64_t n, int64_t lda, float *At);

// Tensor-core symmetric pass in TF32 (tcgen05 kind::tf32, K-major operands
// only) on the full TF32 image: Y = A X + shift X; Xf (ldf >= n, multiple of
// 4, 16-byte aligned) receives X rounded to TF32.  Requires m <= 128.
cudaError_t launch_sym_pass_tf32(cudaStream_t s, int sm_count, const float *At, int64_t n,
                                 const float *X, int64_t ldx, int m, const double *d_shift,
                                 float *Y, int64_t ldy, float *Xf, int64_t ldf, int *d_status,
                                 long long wait_limit = 0);

// Tensor-core symmetric pass Y = (A' + A'^T) X + shift X on the BF16 image;
// Xh (ldh >= n, multiple of 8) receives the BF16 image of X.  Returns
// cudaErrorNotSupported when the configuration is outside what the kernel
// handles (m > 128, misaligned buffers).
// x_part 0 / 1: multiply by the high / low BF16 part of X; accumulate != 0:
// add to Y instead of overwriting it (pass d_shift = NULL then).
// prepared != 0: the producer of X already wrote Xh = bf16(X) and Y = shift X
// (psd_bf16_side; x_part 0, accumulate 0 only): no conversion sweep.
cudaError_t launch_sym_pass_tc(cudaStream_t s, int sm_count, const uint16_t *Ab,
                               int64_t n, const float *X, int64_t ldx, int m,
                               const double *d_shift, float *Y, int64_t ldy, uint16_t *Xh,
                               int64_t ldh, int *d_status, int x_part, int accumulate,
                               int prepared = 0, long long wait_limit = 0);

// Gram partials + FP64 reduction: G = X^T Z (sym = 1: X == Z, symmetric;
// 2: (X^T Z + Z^T X)/2).  Gdf (may be NULL; symmetric forms): the same sums
// as double-float pairs (hi, lo), m x m.  sm_count: SMs the partial
// products may spread over (0: a default).
cudaError_t launch_gram(cudaStream_t s, const float *X, int64_t ldx, const float *Z,
                        int64_t ldz, int64_t n, int m, float *gpart, double *G,
                        int symmetrize, float *Gdf = nullptr, int sm_count = 0);

// Rows per block of launch_gram's product kernel for the symmetric forms
// with m <= 128 (about two blocks per SM, at least PSD_GRAM_CHUNK rows, so
// that the partials fit a workspace sized for ceil(n / PSD_GRAM_CHUNK)
// chunks), its block count, and the blocks of its reduction.
inline int64_t psd_gram_rows(int64_t n, int sm_count)
{
    if (sm_count <= 0) sm_count = 148;
    const int64_t rows = (n + 2 * sm_count - 1) / (2 * sm_count);
    return psd_round_up(rows < PSD_GRAM_CHUNK ? PSD_GRAM_CHUNK : rows, 8);
}
inline int psd_gram_blocks(int64_t n, int sm_count)
{
    const int64_t rows = psd_gram_rows(n, sm_count);
    return (int)((n + rows - 1) / rows);
}
inline int psd_gram_reduce_blocks(int m)
{
    const int nt8 = (int)psd_round_up(m, 8) / 8;
    return (nt8 * (nt8 + 1) / 2 * 64 + 31) / 32;
}
// In a grouped reduction an entry with at most PSD_GRAM_RED_SEQ partials
// takes a thread per position (256 per block), others the form above
constexpr int PSD_GRAM_RED_SEQ = 32;
inline int psd_gram_reduce_grouped_blocks(int m, int nblk)
{
    const int nt8 = (int)psd_round_up(m, 8) / 8;
    return nblk <= PSD_GRAM_RED_SEQ ? (nt8 * (nt8 + 1) / 2 * 64 + 255) / 256 : psd_gram_reduce_blocks(m);
}

// ---- grouped launches (psdproj_batched_grouped) --------------------------
// One launch runs one small step for many problems.  Entry e of a table
// holds the arguments problem e's own launch would take (all with m <= 128);
// for the kernels with several blocks per problem, bmap[b] = (entry, block
// of that entry) says what block b of the launch does; the one-block
// kernels run entry b in block b.  Tables and maps live in device memory.
struct psd_g_gram {          // launch_gram, symmetric forms, m <= 128
    const float *X, *Z;      // Z: the two-sided form only
    int64_t ldx, ldz, n;
    int m, mp, rows, nblk;   // mp = round_up(m, 8); rows, nblk: psd_gram_rows / psd_gram_blocks
    float *gpart;
    double *G;
    float2 *Gdf;             // may be NULL
};
// two: the two-sided form (S = (X^T Z + Z^T X)/2); nb / nb_red: the blocks
// of the product and of the reduction (bmap: block < nblk of its entry;
// bmap_red: block < psd_gram_reduce_grouped_blocks(m, nblk))
cudaError_t launch_gram_grouped(cudaStream_t s, const psd_g_gram *tab, int two, const int2 *bmap, int nb,
                                const int2 *bmap_red, int nb_red, int mp_max);

struct psd_g_chol {          // launch_cholesky, m <= 128 (reads the double-float Gram)
    const float2 *Gd;
    int m;
    float *Rinv;
    int *dead;
    int *d_qrank;            // may be NULL
};
cudaError_t launch_cholesky_grouped(cudaStream_t s, const psd_g_chol *tab, int count, int m_max, int first_pass,
                                    double tau, int *d_status);

constexpr int PSD_TALL_RT = 32;   // rows per tile of the tall x small product (m, c <= 128)
struct psd_g_tall {          // launch_tall_small, m, c <= 128
    const float *Y;
    int64_t ldy, n;
    int m;
    const float *B;
    int c;
    const int *colmask, *d_cols;
    float *Z;
    int64_t ldz;
    psd_bf16_side side;      // no side outputs: Xh = Y = NULL
    int ntiles, nb;          // ntiles = ceil(n / PSD_TALL_RT); nb blocks stride over them
};
cudaError_t launch_tall_small_grouped(cudaStream_t s, const psd_g_tall *tab, const int2 *bmap, int nb, int m_max);

struct psd_g_eig {           // launch_eig, m <= 128
    const double *C;
    const float2 *Cd;        // C as double-float pairs, may be NULL
    int m;
    float *V;
    double *d;
    float *scr;              // 3 (m+2)^2 floats
    int *d_fail;             // the tridiagonal solver's failure flag
};
// blocks per problem of the Newton-Schulz kernels and of the Rayleigh
// quotients (m <= 128: PSD_RQ eigenpairs per block, C and the eigenvectors
// in psd_rayleigh_smem(m) bytes of shared memory)
constexpr int PSD_RQ = 8;
inline int psd_eig_ns_blocks(int m) { return ((m + 15) / 16) * ((m + 15) / 16); }
inline int psd_eig_ray_blocks(int m) { return (m + PSD_RQ - 1) / PSD_RQ; }
inline size_t psd_rayleigh_smem(int m) { return sizeof(double) * (size_t)m * m + sizeof(float) * PSD_RQ * (size_t)m; }
// bmap_ns: block < psd_eig_ns_blocks(m) of its entry; bmap_ray: block < psd_eig_ray_blocks(m)
cudaError_t launch_eig_grouped(cudaStream_t s, const psd_g_eig *tab, int count, const int2 *bmap_ns, int nb_ns,
                               const int2 *bmap_ray, int nb_ray, int m_max, int *d_status, int method);
cudaError_t launch_eig_tridiag_grouped(cudaStream_t s, const psd_g_eig *tab, int count, const int2 *bmap_ns,
                                       int nb_ns, const int2 *bmap_ray, int nb_ray, int m_max,
                                       int *d_status_on_fail);

struct psd_g_pi {            // one power iteration on the BF16 image (launch_power_iteration_bf16)
    const uint16_t *Ab;
    int64_t n;
    float *v0, *v1, *v2;     // 16-byte aligned, n floats each
    double *scal;            // the iteration's scales (scal[0], scal[1])
    const double *shift_neg; // may be NULL: as launch_power_iteration_bf16's d_shift_neg
    double *sigma;           // ||y|| of the last product
    uint64_t seed;
    int nb;                  // CTAs per product, 1 <= nb <= psd_tile_count(n); also the start's blocks
};
// the start vector (Philox stream stream_id of seed) and scales; bmap: block
// < nb of its entry
cudaError_t launch_pi_start_grouped(cudaStream_t s, const psd_g_pi *tab, const int2 *bmap, int nb,
                                   uint32_t stream_id);
// N + 1 products, each normalising its input, then the norms
cudaError_t launch_power_iteration_grouped(cudaStream_t s, const psd_g_pi *tab, int count, const int2 *bmap,
                                          int nb, int N, int *d_status, long long wait_limit = 0);

struct psd_g_alpha {         // launch_alpha_finish
    const double *s1, *s2;
    double alpha_in;
    double *d_alpha;         // may be NULL
    double *d_shift;
    int *d_info;             // may be NULL
};
cudaError_t launch_alpha_finish_grouped(cudaStream_t s, const psd_g_alpha *tab, int count);

struct psd_g_pack {          // launch_pack_bf16 (device A)
    const float *A;
    int64_t n, lda;
    uint16_t *Ab;
    int nbc, vec;            // tile columns; A rows 16-byte aligned
};
// part as launch_pack_bf16; bmap: (entry, block) over the blocks of the
// upper block triangle (tile column J >= PSD_TILE_R * block row)
cudaError_t launch_pack_grouped(cudaStream_t s, const psd_g_pack *tab, const int2 *bmap, int nb, int part);

struct psd_g_gauss {         // launch_gaussian
    uint64_t seed;
    int64_t n;
    int m, mpad;
    int64_t rows_pad;
    float *X;
    int64_t ldx;
    psd_bf16_side side;
    int nb;                  // blocks striding over the entry's rows_pad x mpad values
};
cudaError_t launch_gaussian_grouped(cudaStream_t s, const psd_g_gauss *tab, const int2 *bmap, int nb,
                                    uint32_t stream_id);

struct psd_g_factor {        // launch_factor_prep
    const float *V;
    const double *d;
    int m;
    float *M;
    int *d_rank;
    int *d_rank_out;         // may be NULL: a second copy of the rank (the caller's)
};
cudaError_t launch_factor_prep_grouped(cudaStream_t s, const psd_g_factor *tab, int count);

// first_pass = 1: double-float factorization (FP64 when m > 128); 0: FP32.
// Writes R^-1 (m x m column-major FP32), the dependent-column flags and
// (d_qrank, may be NULL) the number of independent columns.  m <= 128
// reads Gdf (the Gram as double-float pairs, symmetric, both halves), larger
// m read G; gscratch: (m*m + m) doubles + m*m floats of device memory, used
// when m > 128.
cudaError_t launch_cholesky(cudaStream_t s, const double *G, const float *Gdf, int m, float *Rinv,
                            int *dead, int *d_qrank, double tau, int *d_status, int first_pass,
                            double *gscratch);

// Y (n x m) times a small m x c matrix B (column-major, ld = m) -> Z (n x c).
// colmask (may be NULL): columns j with colmask[j] != 0 are written as zero.
// d_cols (may be NULL): device int; only the first *d_cols columns of B are
// used and the rest of Z is written as zero.
// side (may be NULL, c <= 128 only): the BF16 pass's side outputs of Z.
cudaError_t launch_tall_small(cudaStream_t s, const float *Y, int64_t ldy, int64_t n, int m,
                              const float *B, int c, const int *colmask, const int *d_cols,
                              float *Z, int64_t ldz, const psd_bf16_side *side = nullptr, int sm_count = 0);

// scratch: 3 (m+2)^2 floats of device memory (used when m is too large for
// shared memory); d_flag: one device int (the tridiagonal solver's failure
// flag); method: PSDPROJ_EIG_*.
// kernels launch_eig starts: the tridiagonal solver, its Newton-Schulz step
// and the FP64 Rayleigh quotients (four), the Jacobi solver (one, also after
// the others in AUTO)
inline int psd_eig_launches(int method)
{
    return method == PSDPROJ_EIG_JACOBI ? 1 : (method == PSDPROJ_EIG_AUTO ? 5 : 4);
}
// Cdf (may be NULL): C also as double-float pairs (hi, lo), m x m, from
// which the eigenvalues' FP64 Rayleigh quotients take C v (else from C).
cudaError_t launch_eig(cudaStream_t s, const double *C, int m, float *V, double *d,
                       float *scratch, int *d_status, int method, int *d_flag, const float *Cdf = nullptr);
cudaError_t launch_eig_tridiag(cudaStream_t s, const double *C, int m, float *V, double *d,
                               float *scratch, int *d_fail, int *d_status_on_fail, const float *Cdf = nullptr);

cudaError_t launch_factor_prep(cudaStream_t s, const float *V, const double *d, int m,
                               float *M, int *d_rank);

cudaError_t launch_syrk_simt(cudaStream_t s, const float *W, int64_t ldw, int64_t n, int m,
                             const int *d_rank, float *P, int64_t ldp, int upper_only);

// prepared != 0: Whi / Wlo already hold W's BF16 high and low parts (the
// producer of W wrote them), so the split is not launched
cudaError_t launch_syrk_tc(cudaStream_t s, int sm_count, const float *W, int64_t ldw,
                           int64_t n, int m, const int *d_rank, float *P, int64_t ldp,
                           int upper_only, uint16_t *Whi, uint16_t *Wlo, int64_t ldh,
                           int *d_status, long long wait_limit = 0, int prepared = 0);

// Power iteration (Alg. 4) with optional shift taken from *d_shift_in
// (negated sigma); writes sigma to *d_sigma.
cudaError_t launch_power_iteration(cudaStream_t s, const float *A, int64_t n, int64_t lda,
                                   int N, uint64_t seed, uint32_t stream_id,
                                   const double *d_shift_neg, float *v0, float *v1,
                                   double *scal, double *d_sigma);

// The same on the BF16 image (launch_pack_bf16), N + 4 launches: each
// product normalises its own input and clears the next product's output,
// the three vectors v0, v1, v2 (16-byte aligned) taking turns; the products
// are chained by programmatic dependent launch.
cudaError_t launch_power_iteration_bf16(cudaStream_t s, int sm_count, const uint16_t *Ab, int64_t n,
                                        int N, uint64_t seed, uint32_t stream_id,
                                        const double *d_shift_neg, float *v0, float *v1, float *v2,
                                        double *scal, double *d_sigma, int *d_status,
                                        long long wait_limit = 0);

// The power iteration's start (scal[0] = 1, v1 = 0) and its norm step
// (scal[0] = 1/||y||, scal[1] = ||y||, *d_sigma = ||y|| when asked; other = 0).
cudaError_t launch_pi_init(cudaStream_t s, double *scal, float *v1, int64_t n);
cudaError_t launch_pi_norm(cudaStream_t s, const float *y, float *other, int64_t n, double *scal,
                           double *d_sigma);

// Deterministic (fixed summation order, no atomics) forms of the FP32 pass
// and of the power iteration (csrc/detpass.cu).  part: psd_det_part_floats(n,
// m) floats of device scratch.
int64_t psd_det_part_floats(int64_t n, int m);
cudaError_t launch_sym_pass_det(cudaStream_t s, const float *A, int64_t n, int64_t lda, const float *X,
                                int64_t ldx, int m, const double *d_shift, float *Y, int64_t ldy, float *part);
cudaError_t launch_power_iteration_det(cudaStream_t s, const float *A, int64_t n, int64_t lda, int N,
                                       uint64_t seed, uint32_t stream_id, const double *d_shift_neg,
                                       float *v0, float *v1, double *scal, double *d_sigma, float *part);

cudaError_t launch_alpha_finish(cudaStream_t s, const double *d_s1, const double *d_s2,
                                double alpha_in, double *d_alpha, double *d_shift,
                                int *d_info);

cudaError_t launch_copy_tall(cudaStream_t s, const float *X, int64_t ldx, int64_t n, int m,
                             float *Y, int64_t ldy);
