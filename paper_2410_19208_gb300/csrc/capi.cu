// C ABI of the psdproj library: context, workspace and the two pipelines.
//
//   psdproj_alg1: Alg. 2 (randomized PSD projection) with the range finder of
//                 Alg. 1, orthonormalising after every product.
//   psdproj_alg2: Alg. 3 (scaled randomized PSD projection) with alpha from
//                 Alg. 5 unless given; the core and last step use the reduced
//                 form Q (Q^T A Q)_+ Q^T of Lemma 4.
// Every step is a kernel of this library; nothing runs on the host but
// argument checks, workspace management and launches.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <cstring>
#include <vector>
#include <algorithm>
#include <new>
#include <map>
#include <mutex>
#include <string>

#include "ctx.h"

namespace {

// the last CUDA error this host thread turned into a status, and where
thread_local int t_last_cuda = 0, t_last_line = 0;

int cuda_status(cudaError_t e, int line = 0)
{
    if (e == cudaSuccess) return PSDPROJ_OK;
    t_last_cuda = (int)e;
    t_last_line = line;
    if (e == cudaErrorMemoryAllocation) return PSDPROJ_ENOMEM;
    if (e == cudaErrorNotSupported) return PSDPROJ_ENOTSUP;
    return PSDPROJ_ECUDA;
}

#define PSD_CK(expr)                              \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) return cuda_status(_e, __LINE__); \
    } while (0)

#define PSD_TRY(expr)                 \
    do {                              \
        int _s = (expr);              \
        if (_s != PSDPROJ_OK) return _s; \
    } while (0)

struct device_guard {
    int prev = -1;
    explicit device_guard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~device_guard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

std::atomic<uint64_t> g_launches{0};

// counts the kernels a launcher started, then checks its status
#define PSD_KL(expr, nk)                                   \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_status(_e, __LINE__); \
        g_launches.fetch_add((uint64_t)(nk));              \
    } while (0)

// brackets one stage with two events when timing is on
struct stage_scope {
    psdproj_ctx *c;
    bool rec = false;
    stage_scope(psdproj_ctx *ctx, int kind) : c(ctx)
    {
        psd_timing &t = c->timing;
        if (t.on && t.created && t.n < PSD_MAX_TIMED) {
            cudaEventRecord(t.ev[2 * t.n], c->stream);
            t.kind[t.n] = kind;
            rec = true;
        }
    }
    ~stage_scope()
    {
        if (rec) {
            psd_timing &t = c->timing;
            cudaEventRecord(t.ev[2 * t.n + 1], c->stream);
            ++t.n;
        }
    }
};

void free_workspace(psd_workspace &ws)
{
    if (ws.base) cudaFree(ws.base);
    ws = psd_workspace();
}

}  // namespace

int psd_budget_check(const psdproj_ctx *ctx, size_t old_bytes, size_t new_bytes)
{
    const psdproj_ctx *root = ctx->root ? ctx->root : ctx;
    if (root->budget == 0 || new_bytes <= old_bytes) return PSDPROJ_OK;
    const size_t held = psdproj_workspace_bytes(root);
    if (held - old_bytes + new_bytes > root->budget) return PSDPROJ_ENOMEM;
    return PSDPROJ_OK;
}

namespace {

// The workspace's carve-up for nn rows and lp columns: one function serves
// both the size (base == nullptr: offsets only) and the pointers, so the two
// cannot disagree.  Returns the total bytes.
size_t carve_workspace(psd_workspace &lay, char *base, int64_t nn, int lp)
{
    const int64_t ld = psd_ld(nn);
    const int64_t nchunk = (nn + PSD_GRAM_CHUNK - 1) / PSD_GRAM_CHUNK;
    const size_t tall = align256(sizeof(float) * (size_t)ld * lp);
    const size_t half_tall = align256(sizeof(uint16_t) * (size_t)ld * lp);
    const size_t small_d = align256(sizeof(double) * (size_t)lp * lp);
    const size_t small_f = align256(sizeof(float) * (size_t)lp * lp);
    const size_t chol_scr = align256(sizeof(double) * ((size_t)lp * lp + lp) + sizeof(float) * (size_t)lp * lp);
    size_t off = 0;
    auto take = [&](size_t b) { char *q = base ? base + off : nullptr; off += align256(b); return q; };
    lay.Om = reinterpret_cast<float *>(take(tall));
    lay.Y = reinterpret_cast<float *>(take(tall));
    lay.Q = reinterpret_cast<float *>(take(tall));
    lay.T = reinterpret_cast<float *>(take(tall));
    lay.W = reinterpret_cast<float *>(take(tall));
    lay.Xf = reinterpret_cast<float *>(take(tall));
    lay.Xhi = reinterpret_cast<uint16_t *>(take(half_tall));
    lay.Xlo = reinterpret_cast<uint16_t *>(take(half_tall));
    lay.gpart = reinterpret_cast<float *>(take(sizeof(float) * nchunk * lp * lp));
    lay.G = reinterpret_cast<double *>(take(small_d));
    lay.R = reinterpret_cast<double *>(take(small_d));
    lay.C = reinterpret_cast<double *>(take(small_d));
    lay.cholscr = reinterpret_cast<double *>(take(chol_scr));
    lay.d = reinterpret_cast<double *>(take(sizeof(double) * lp));
    lay.Rinv = reinterpret_cast<float *>(take(small_f));
    lay.V = reinterpret_cast<float *>(take(small_f));
    lay.M = reinterpret_cast<float *>(take(small_f));
    lay.eigscr = reinterpret_cast<float *>(take(sizeof(float) * 3 * (size_t)(lp + 2) * (lp + 2)));
    lay.dead = reinterpret_cast<int *>(take(sizeof(int) * lp));
    lay.pv0 = reinterpret_cast<float *>(take(sizeof(float) * ld));
    lay.pv1 = reinterpret_cast<float *>(take(sizeof(float) * ld));
    lay.pv2 = reinterpret_cast<float *>(take(sizeof(float) * ld));
    lay.scal = reinterpret_cast<double *>(take(sizeof(double) * 16));
    lay.ints = reinterpret_cast<int *>(take(sizeof(int) * 16));
    lay.picks = reinterpret_cast<int *>(take(sizeof(int) * PSD_MAX_M));
    return off;
}

}  // namespace

size_t psd_projection_device_bytes(int64_t n, int m, int prec, int deterministic)
{
    psd_workspace lay;
    size_t b = carve_workspace(lay, nullptr, n, psd_lpad(m));
    if (deterministic) return b + sizeof(float) * (size_t)psd_det_part_floats(n, m);
    if (prec == PSDPROJ_PREC_TF32) b += (size_t)psd_tile32_count(n) * (size_t)PSD_TILE_BYTES;
    else if (prec == PSDPROJ_PREC_BF16) b += (size_t)psd_tile_count(n) * (size_t)PSD_TILE_BYTES;
    else if (prec == PSDPROJ_PREC_BF16X3) b += 2 * (size_t)psd_tile_count(n) * (size_t)PSD_TILE_BYTES;
    return b;
}

int psd_ensure_workspace(psdproj_ctx *ctx, int64_t n, int m)
{
    psd_workspace &ws = ctx->ws;
    const int lpad = psd_lpad(m);
    if (ws.base && ws.n >= n && ws.lpad >= lpad) return PSDPROJ_OK;
    const int64_t nn = ws.base ? (n > ws.n ? n : ws.n) : n;
    const int lp = ws.base ? (lpad > ws.lpad ? lpad : ws.lpad) : lpad;
    const int64_t ld = psd_ld(nn);
    psd_workspace lay;
    auto carve = [&](char *base) -> size_t { return carve_workspace(lay, base, nn, lp); };
    const size_t total = carve(nullptr);
    PSD_TRY(psd_budget_check(ctx, ws.bytes, total));
    if (ws.base) {
        cudaStreamSynchronize(ctx->stream);
        free_workspace(ws);
    }
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, total);
    if (e != cudaSuccess) return cuda_status(e, __LINE__);
    carve(static_cast<char *>(base));
    ws = lay;
    ws.base = base;
    ws.bytes = total;
    ws.n = nn;
    ws.lpad = lp;
    ws.ld = ld;
    // zero everything once: padded rows / columns of the tall buffers stay 0
    e = cudaMemsetAsync(base, 0, total, ctx->stream);
    if (e != cudaSuccess) return cuda_status(e, __LINE__);
    return PSDPROJ_OK;
}

namespace {

int ensure_stage(psdproj_ctx *ctx, float **buf, size_t *cap, size_t bytes, cudaStream_t s);

// scalar slots in ws.scal
enum { SC_SHIFT = 4, SC_SIGMA1 = 5, SC_SIGMA2 = 6, SC_ALPHA = 7 };
// int slots in ws.ints
enum { IN_RANK = 0, IN_INFO = 1, IN_QRANK = 2, IN_EIGFAIL = 3 };

int check_opts(const psdproj_opts *o)
{
    if (o->prec < PSDPROJ_PREC_FP32 || o->prec > PSDPROJ_PREC_BF16X3) return PSDPROJ_EINVAL;
    if (o->syrk_prec != PSDPROJ_PREC_FP32 && o->syrk_prec != PSDPROJ_PREC_BF16X3) return PSDPROJ_EINVAL;
    if (o->out_mode < PSDPROJ_OUT_FULL || o->out_mode > PSDPROJ_OUT_FACTOR) return PSDPROJ_EINVAL;
    if (o->N < 0 || o->N > 10000) return PSDPROJ_EINVAL;
    if (o->eig < PSDPROJ_EIG_AUTO || o->eig > PSDPROJ_EIG_TRIDIAG) return PSDPROJ_EINVAL;
    if (o->sketch != PSDPROJ_SKETCH_GAUSS && o->sketch != PSDPROJ_SKETCH_SRHT) return PSDPROJ_EINVAL;
    if (o->alpha_mode != PSDPROJ_ALPHA_MINEIG && o->alpha_mode != PSDPROJ_ALPHA_RITZ) return PSDPROJ_EINVAL;
    if (o->deterministic != 0 && o->deterministic != 1) return PSDPROJ_EINVAL;
    if (o->spin_limit < 0) return PSDPROJ_EINVAL;
    if (o->reserved[0] != 0 || o->reserved[1] != 0) return PSDPROJ_EINVAL;
    return PSDPROJ_OK;
}

// The image of A read by the tensor-core passes: allocated on first use
// (32 KB tiles, kept for later calls) and written from A.  BF16: the block
// upper triangle, psd_tile_count(n) tiles; the split form also writes the
// image of the low parts.  TF32: the full symmetric matrix,
// psd_tile32_count(n) tiles, in the same buffer.
int alloc_image(psdproj_ctx *ctx, uint16_t **buf, size_t *cap, size_t bytes, cudaStream_t s)
{
    if (*cap >= bytes) return PSDPROJ_OK;
    PSD_TRY(psd_budget_check(ctx, *cap, bytes));
    if (*buf) {
        cudaStreamSynchronize(s);
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) return cuda_status(e, __LINE__);
    *cap = bytes;
    return PSDPROJ_OK;
}

int pack_image(psdproj_ctx *ctx, const float *A, int64_t n, int64_t lda, int prec)
{
    if (prec == PSDPROJ_PREC_TF32) {
        const size_t bytes = (size_t)psd_tile32_count(n) * (size_t)PSD_TILE_BYTES;
        PSD_TRY(alloc_image(ctx, &ctx->Ab, &ctx->Ab_bytes, bytes, ctx->stream));
        stage_scope st(ctx, PSDPROJ_STAGE_PACK);
        PSD_KL(launch_pack_tf32(ctx->stream, A, n, lda, reinterpret_cast<float *>(ctx->Ab)), 1);
        return PSDPROJ_OK;
    }
    const bool with_lo = prec == PSDPROJ_PREC_BF16X3;
    const size_t bytes = (size_t)psd_tile_count(n) * (size_t)PSD_TILE_BYTES;
    PSD_TRY(alloc_image(ctx, &ctx->Ab, &ctx->Ab_bytes, bytes, ctx->stream));
    if (with_lo) PSD_TRY(alloc_image(ctx, &ctx->Ab_lo, &ctx->Ab_lo_bytes, bytes, ctx->stream));
    stage_scope st(ctx, PSDPROJ_STAGE_PACK);
    PSD_KL(launch_pack_bf16(ctx->stream, A, n, lda, ctx->Ab, 0), 1);
    if (with_lo) PSD_KL(launch_pack_bf16(ctx->stream, A, n, lda, ctx->Ab_lo, 1), 1);
    return PSDPROJ_OK;
}

// Y = A X + shift X in the requested precision (tensor-core forms: from the
// image(s) that pack_image wrote last).  Split BF16: A X ~ A_hi X_hi + A_hi X_lo
// + A_lo X_hi, three tensor-core passes adding into Y.
// prepared: the producer of X already wrote the BF16 form's side outputs
// (ws.Xhi = bf16(X), Y = shift X; see psd_bf16_side), so the pass skips its
// conversion sweep (BF16 form, m <= 128 only).
int sym_pass(psdproj_ctx *ctx, const float *A, int64_t n, int64_t lda, const float *X,
             int64_t ldx, int m, const double *d_shift, float *Y, int64_t ldy, int prec,
             bool prepared = false)
{
    if (ctx->det) {
        // fixed summation order, FP32 on the CUDA cores (opts.deterministic)
        const size_t bytes = sizeof(float) * (size_t)psd_det_part_floats(n, m);
        PSD_TRY(ensure_stage(ctx, &ctx->det_part, &ctx->det_part_bytes, bytes, ctx->stream));
        stage_scope st(ctx, PSDPROJ_STAGE_APASS);
        PSD_KL(launch_sym_pass_det(ctx->stream, A, n, lda, X, ldx, m, d_shift, Y, ldy, ctx->det_part), 2);
        return PSDPROJ_OK;
    }
    stage_scope st(ctx, PSDPROJ_STAGE_APASS);
    if (prec == PSDPROJ_PREC_FP32) {
        PSD_KL(launch_sym_pass_simt(ctx->stream, A, n, lda, X, ldx, m, d_shift, Y, ldy), 1);
        return PSDPROJ_OK;
    }
    psd_workspace &ws = ctx->ws;
    if (prec != PSDPROJ_PREC_TF32 && prec != PSDPROJ_PREC_BF16 && prec != PSDPROJ_PREC_BF16X3)
        return PSDPROJ_ENOTSUP;
    // the tensor-core passes take up to 128 columns (M = 128 rows of X^T):
    // wider sketches run as column slices, one pass over the image each
    for (int c0 = 0; c0 < m; c0 += 128) {
        const int mc = m - c0 < 128 ? m - c0 : 128;
        const float *Xc = X + (int64_t)c0 * ldx;
        float *Yc = Y + (int64_t)c0 * ldy;
        if (prec == PSDPROJ_PREC_TF32) {
            PSD_KL(launch_sym_pass_tf32(ctx->stream, ctx->persist_sms, reinterpret_cast<const float *>(ctx->Ab), n,
                                        Xc, ldx, mc, d_shift, Yc, ldy, ws.Xf + (int64_t)c0 * ws.ld, ws.ld,
                                        ctx->d_status, ctx->wait_limit), 2);
            continue;
        }
        uint16_t *Xhi = ws.Xhi + (int64_t)c0 * ws.ld, *Xlo = ws.Xlo + (int64_t)c0 * ws.ld;
        const bool prep = prepared && prec == PSDPROJ_PREC_BF16 && m <= 128;
        PSD_KL(launch_sym_pass_tc(ctx->stream, ctx->persist_sms, ctx->Ab, n, Xc, ldx, mc, d_shift, Yc, ldy,
                                  Xhi, ws.ld, ctx->d_status, 0, 0, prep ? 1 : 0, ctx->wait_limit), prep ? 1 : 2);
        if (prec == PSDPROJ_PREC_BF16X3) {
            PSD_KL(launch_sym_pass_tc(ctx->stream, ctx->persist_sms, ctx->Ab, n, Xc, ldx, mc, nullptr, Yc, ldy,
                                      Xlo, ws.ld, ctx->d_status, 1, 1, 0, ctx->wait_limit), 2);
            PSD_KL(launch_sym_pass_tc(ctx->stream, ctx->persist_sms, ctx->Ab_lo, n, Xc, ldx, mc, nullptr, Yc, ldy,
                                      Xhi, ws.ld, ctx->d_status, 0, 1, 0, ctx->wait_limit), 2);
        }
    }
    return PSDPROJ_OK;
}

// CholeskyQR2: Q = orth(Y); Y is read only in the first half.  side (may be
// NULL): the final product also writes the BF16 pass's side outputs of Q.
// passes = 1 (an orthonormalisation between two power products): the first
// half only, Q = Y R^-1 with R from the double-float Cholesky, the same span
// as Y and orthonormal to about eps32 kappa(Y)^2, i.e. well conditioned
// wherever the second half could run at all; the products that follow only
// need a well-conditioned basis of that span.
int cholqr2(psdproj_ctx *ctx, const float *Y, int64_t ldy, int64_t n, int m, float *Q,
            int64_t ldq, int *d_qrank, const psd_bf16_side *side = nullptr, int passes = 2)
{
    psd_workspace &ws = ctx->ws;
    cudaStream_t s = ctx->stream;
    const double tau = 1e-10;
    stage_scope st(ctx, PSDPROJ_STAGE_ORTH);
    // m <= 128: the Gram also as double-float pairs, in the (then unused) large-m scratch
    float *gdf = m <= 128 ? reinterpret_cast<float *>(ws.cholscr) : nullptr;
    PSD_KL(launch_gram(s, Y, ldy, Y, ldy, n, m, ws.gpart, ws.G, 1, gdf, ctx->persist_sms), 2);
    PSD_KL(launch_cholesky(s, ws.G, gdf, m, ws.Rinv, ws.dead, passes == 1 ? d_qrank : nullptr, tau, ctx->d_status,
                           1, ws.cholscr), 1);
    if (passes == 1) {
        PSD_KL(launch_tall_small(s, Y, ldy, n, m, ws.Rinv, m, ws.dead, nullptr, Q, ldq, side, ctx->persist_sms), 1);
        return PSDPROJ_OK;
    }
    PSD_KL(launch_tall_small(s, Y, ldy, n, m, ws.Rinv, m, ws.dead, nullptr, ws.T, ws.ld, nullptr, ctx->persist_sms), 1);
    PSD_KL(launch_gram(s, ws.T, ws.ld, ws.T, ws.ld, n, m, ws.gpart, ws.G, 1, gdf, ctx->persist_sms), 2);
    PSD_KL(launch_cholesky(s, ws.G, gdf, m, ws.Rinv, ws.dead, d_qrank, tau, ctx->d_status, 0,
                           ws.cholscr), 1);
    PSD_KL(launch_tall_small(s, ws.T, ws.ld, n, m, ws.Rinv, m, ws.dead, nullptr, Q, ldq, side, ctx->persist_sms), 1);
    return PSDPROJ_OK;
}

int validate(int64_t n, int64_t lda, int k, int p, int q, const void *A)
{
    if (!A || n < 1 || k < 1 || p < 0 || q < 0 || q > 16 || lda < n) return PSDPROJ_EINVAL;
    const int64_t m = (int64_t)k + p;
    if (m < 1 || m > n || m > PSD_MAX_M) return PSDPROJ_EINVAL;
    return PSDPROJ_OK;
}

// One projection's arguments and the state its phases share.  A projection
// runs as: proj_begin (image, alpha, Omega, the first product), the
// orthonormalisation after each product with A, proj_power_pass for each
// power product, proj_core_pass, proj_core_small (core, eigensolver, factor)
// and proj_finish (P = W W^T).  run_projection issues them in that order on
// one context; psdproj_batched_grouped issues each phase for all problems of
// a batch before the next, the small steps as grouped launches.
struct proj_call {
    const float *dA = nullptr;
    int64_t n = 0, lda = 0;
    int k = 0, p = 0, q = 0, m = 0;
    uint64_t seed = 0;
    bool scaled = false;                 // Alg. 3 (the shifted form)
    double alpha_in = 0.0;
    double *d_alpha_out = nullptr;
    int *d_info = nullptr;
    float *dP = nullptr;
    int64_t ldp = 0;
    float *dW = nullptr;
    int64_t ldw = 0;
    int *d_rank = nullptr;
    psdproj_opts opts = {};
    bool omega_ready = false;            // Omega already in the workspace (warm start of Alg. 6)
    // set by the grouped batch for the phases it runs as grouped launches
    bool omega_prepared = false;         // Omega and its BF16 side outputs already written
    bool w_split = false;                // W's BF16 high and low parts written with W
    bool rank_written = false;           // the factor step wrote *d_rank
    // set by proj_begin
    const double *shift = nullptr;       // device shift of the power products (NULL: none)
    bool fuse = false;                   // BF16 side outputs written by X's producers
};

// Alg. 3 with alpha from the Ritz values of the unshifted sketch
bool proj_ritz(const proj_call &pc)
{
    return pc.scaled && !(pc.alpha_in > 0.0) && pc.opts.alpha_mode == PSDPROJ_ALPHA_RITZ;
}
// BF16 form: the producers of each pass's X write its side outputs
bool proj_fuse(const proj_call &pc)
{
    return pc.opts.prec == PSDPROJ_PREC_BF16 && pc.m <= 128 && !proj_ritz(pc);
}
// where the shift of the power products lives (Alg. 3), else NULL
const double *proj_shift(const proj_call &pc, const psd_workspace &ws)
{
    return pc.scaled ? ws.scal + SC_SHIFT : nullptr;
}

// The core C also as double-float pairs (m <= 128: the Gram reduction's own
// sums, in the orthonormalisation's then unused scratch), for the
// eigenvalues' Rayleigh quotients; NULL for wider sketches
float *core_gdf(const psd_workspace &ws, int m)
{
    return m <= 128 ? reinterpret_cast<float *>(ws.cholscr) : nullptr;
}

// The BF16 pass's side outputs for the next pass over ctx's workspace
psd_bf16_side proj_side(psdproj_ctx *ctx, const double *next_shift)
{
    psd_workspace &ws = ctx->ws;
    return psd_bf16_side{ws.Xhi, ws.ld, ws.Y, ws.ld, next_shift};
}

// the tensor-core forms read A once here and their image(s) in every later pass
int proj_pack(psdproj_ctx *ctx, const proj_call &pc)
{
    if (pc.opts.prec == PSDPROJ_PREC_FP32) return PSDPROJ_OK;
    return pack_image(ctx, pc.dA, pc.n, pc.lda, pc.opts.prec);
}

// Alg. 3's alpha by Alg. 5 (two power iterations, Alg. 4) unless given or
// taken from the Ritz values (proj_sketch), and the shift it sets
int proj_alpha(psdproj_ctx *ctx, const proj_call &pc)
{
    if (!pc.scaled || proj_ritz(pc)) return PSDPROJ_OK;
    const psdproj_opts &opts = pc.opts;
    psd_workspace &ws = ctx->ws;
    cudaStream_t s = ctx->stream;
    const float *dA = pc.dA;
    const int64_t n = pc.n, lda = pc.lda;
    const uint64_t seed = pc.seed;
    const double alpha_in = pc.alpha_in;
    const bool bf16 = opts.prec == PSDPROJ_PREC_BF16;
    {
        double *sc = ws.scal;
        if (!(alpha_in > 0.0)) {
            stage_scope st(ctx, PSDPROJ_STAGE_GEMV);
            if (ctx->det) {
                PSD_KL(launch_power_iteration_det(s, dA, n, lda, opts.N, seed, 3u, nullptr, ws.pv0, ws.pv1, sc,
                                                  sc + SC_SIGMA1, ctx->det_part), 3 * opts.N + 5);
                PSD_KL(launch_power_iteration_det(s, dA, n, lda, opts.N, seed, 4u, sc + SC_SIGMA1, ws.pv0, ws.pv1,
                                                  sc, sc + SC_SIGMA2, ctx->det_part), 3 * opts.N + 5);
            } else if (bf16) {
                PSD_KL(launch_power_iteration_bf16(s, ctx->persist_sms, ctx->Ab, n, opts.N, seed, 3u, nullptr,
                                                   ws.pv0, ws.pv1, ws.pv2, sc, sc + SC_SIGMA1,
                                                   ctx->d_status, ctx->wait_limit),
                       opts.N + 4);
                PSD_KL(launch_power_iteration_bf16(s, ctx->persist_sms, ctx->Ab, n, opts.N, seed, 4u,
                                                   sc + SC_SIGMA1, ws.pv0, ws.pv1, ws.pv2, sc,
                                                   sc + SC_SIGMA2, ctx->d_status, ctx->wait_limit),
                       opts.N + 4);
            } else {
                PSD_KL(launch_power_iteration(s, dA, n, lda, opts.N, seed, 3u, nullptr, ws.pv0, ws.pv1,
                                              sc, sc + SC_SIGMA1), 2 * opts.N + 4);
                PSD_KL(launch_power_iteration(s, dA, n, lda, opts.N, seed, 4u, sc + SC_SIGMA1, ws.pv0,
                                              ws.pv1, sc, sc + SC_SIGMA2), 2 * opts.N + 4);
            }
        }
        stage_scope st(ctx, PSDPROJ_STAGE_OTHER);
        PSD_KL(launch_alpha_finish(s, sc + SC_SIGMA1, sc + SC_SIGMA2, alpha_in,
                                   pc.d_alpha_out ? pc.d_alpha_out : sc + SC_ALPHA, sc + SC_SHIFT,
                                   pc.d_info ? pc.d_info : ws.ints + IN_INFO), 1);
    }
    return PSDPROJ_OK;
}

// Omega (Alg. 1) and Y = (A + shift I) Omega, after proj_pack and proj_alpha
// (the Ritz variant of alpha: its unshifted sketch first)
int proj_sketch(psdproj_ctx *ctx, proj_call &pc)
{
    psdproj_opts &opts = pc.opts;
    psd_workspace &ws = ctx->ws;
    cudaStream_t s = ctx->stream;
    const float *dA = pc.dA;
    const int64_t n = pc.n, lda = pc.lda;
    const int m = pc.m;
    const uint64_t seed = pc.seed;
    const bool ritz = proj_ritz(pc);
    const double *shift = pc.scaled && !ritz ? ws.scal + SC_SHIFT : nullptr;
    const int lpad = psd_lpad(m);
    // BF16 form: every kernel that writes the next pass's X (Omega, the last
    // product of each CholeskyQR2) also writes that pass's BF16 image of X
    // and starts its Y, so the passes need no conversion sweep
    const bool fuse = proj_fuse(pc);
    bool prepared = pc.omega_prepared && fuse;
    // Omega (Alg. 1), then Y = (A + shift I) Omega
    if (!pc.omega_ready && !pc.omega_prepared) {
        stage_scope st(ctx, PSDPROJ_STAGE_OTHER);
        if (opts.sketch == PSDPROJ_SKETCH_SRHT) {
            PSD_KL(launch_srht(s, seed, n, m, lpad, ws.ld, ws.picks, ctx->d_status, ws.Om, ws.ld), 2);
        } else {
            const psd_bf16_side sd = proj_side(ctx, shift);
            PSD_KL(launch_gaussian(s, seed, 0u, n, m, lpad, ws.ld, ws.Om, ws.ld, fuse ? &sd : nullptr), 1);
            prepared = fuse;
        }
    }
    if (ritz) {
        // Alg. 3's first product without the shift, A Omega, does not depend
        // on alpha: its sketch Q0 = orth(A Omega) gives Ritz values
        // eig(Q0^T A Q0) whose most negative one sets alpha; then
        // (A + alpha I) Omega = A Omega + alpha Omega needs no further pass.
        double *sc = ws.scal;
        PSD_TRY(sym_pass(ctx, dA, n, lda, ws.Om, ws.ld, m, nullptr, ws.Y, ws.ld, opts.prec));
        PSD_TRY(cholqr2(ctx, ws.Y, ws.ld, n, m, ws.Q, ws.ld, ws.ints + IN_QRANK));
        PSD_TRY(sym_pass(ctx, dA, n, lda, ws.Q, ws.ld, m, nullptr, ws.W, ws.ld, opts.prec));
        float *cdf = core_gdf(ws, m);
        {
            stage_scope st(ctx, PSDPROJ_STAGE_CORE);
            PSD_KL(launch_gram(s, ws.Q, ws.ld, ws.W, ws.ld, n, m, ws.gpart, ws.C, 2, cdf, ctx->persist_sms), 2);
        }
        {
            stage_scope st(ctx, PSDPROJ_STAGE_EIG);
            PSD_KL(launch_eig(s, ws.C, m, ws.V, ws.d, ws.eigscr, ctx->d_status, opts.eig,
                              ws.ints + IN_EIGFAIL, cdf), psd_eig_launches(opts.eig));
        }
        stage_scope st(ctx, PSDPROJ_STAGE_OTHER);
        PSD_KL(launch_ritz_alpha(s, ws.d, m, pc.d_alpha_out ? pc.d_alpha_out : sc + SC_ALPHA, sc + SC_SHIFT,
                                 pc.d_info ? pc.d_info : ws.ints + IN_INFO), 1);
        PSD_KL(launch_add_shift(s, ws.Y, ws.Om, n, m, ws.ld, sc + SC_SHIFT), 1);
        shift = sc + SC_SHIFT;
    } else {
        PSD_TRY(sym_pass(ctx, dA, n, lda, ws.Om, ws.ld, m, shift, ws.Y, ws.ld, opts.prec, prepared));
    }
    pc.shift = shift;
    pc.fuse = fuse;
    return PSDPROJ_OK;
}

// The image of A, alpha (Alg. 3), Omega (Alg. 1) and Y = (A + shift I) Omega
int proj_begin(psdproj_ctx *ctx, proj_call &pc)
{
    PSD_TRY(proj_pack(ctx, pc));
    PSD_TRY(proj_alpha(ctx, pc));
    return proj_sketch(ctx, pc);
}

// power product: Y = (A + shift I) Q
int proj_power_pass(psdproj_ctx *ctx, const proj_call &pc)
{
    psd_workspace &ws = ctx->ws;
    return sym_pass(ctx, pc.dA, pc.n, pc.lda, ws.Q, ws.ld, pc.m, pc.shift, ws.Y, ws.ld, pc.opts.prec, pc.fuse);
}

// core product Y = A Q (Lemma 4: the unshifted A in both algorithms)
int proj_core_pass(psdproj_ctx *ctx, const proj_call &pc)
{
    psd_workspace &ws = ctx->ws;
    return sym_pass(ctx, pc.dA, pc.n, pc.lda, ws.Q, ws.ld, pc.m, nullptr, ws.Y, ws.ld, pc.opts.prec, pc.fuse);
}

float *proj_w(psdproj_ctx *ctx, const proj_call &pc) { return pc.dW ? pc.dW : ctx->ws.W; }
int64_t proj_ldw(psdproj_ctx *ctx, const proj_call &pc) { return pc.dW ? pc.ldw : ctx->ws.ld; }

// C = Q^T A Q, its eigenpairs, M = V sqrt(max(D, 0)) and W = Q M
int proj_core_small(psdproj_ctx *ctx, const proj_call &pc)
{
    psd_workspace &ws = ctx->ws;
    cudaStream_t s = ctx->stream;
    const int64_t n = pc.n;
    const int m = pc.m;
    float *cdf = core_gdf(ws, m);
    {
        stage_scope st(ctx, PSDPROJ_STAGE_CORE);
        PSD_KL(launch_gram(s, ws.Q, ws.ld, ws.Y, ws.ld, n, m, ws.gpart, ws.C, 2, cdf, ctx->persist_sms), 2);
    }
    {
        stage_scope st(ctx, PSDPROJ_STAGE_EIG);
        PSD_KL(launch_eig(s, ws.C, m, ws.V, ws.d, ws.eigscr, ctx->d_status, pc.opts.eig,
                          ws.ints + IN_EIGFAIL, cdf), psd_eig_launches(pc.opts.eig));
    }
    int *rk = ws.ints + IN_RANK;
    stage_scope st(ctx, PSDPROJ_STAGE_FACTOR);
    PSD_KL(launch_factor_prep(s, ws.V, ws.d, m, ws.M, rk), 1);
    PSD_KL(launch_tall_small(s, ws.Q, ws.ld, n, m, ws.M, m, nullptr, rk, proj_w(ctx, pc), proj_ldw(ctx, pc), nullptr,
                             ctx->persist_sms), 1);
    return PSDPROJ_OK;
}

// P = W W^T (unless only the factor is asked for) and the rank
int proj_finish(psdproj_ctx *ctx, const proj_call &pc)
{
    psd_workspace &ws = ctx->ws;
    cudaStream_t s = ctx->stream;
    const int m = pc.m;
    int *rk = ws.ints + IN_RANK;
    float *Wd = proj_w(ctx, pc);
    const int64_t ldwd = proj_ldw(ctx, pc);
    if (pc.opts.out_mode != PSDPROJ_OUT_FACTOR) {
        stage_scope st(ctx, PSDPROJ_STAGE_SYRK);
        const int upper = pc.opts.out_mode == PSDPROJ_OUT_UPPER;
        // the tensor-core SYRK takes up to 128 columns of W; wider factors
        // are written by the FP32 kernel (at least as accurate)
        if (pc.opts.syrk_prec == PSDPROJ_PREC_FP32 || m > 128)
            PSD_KL(launch_syrk_simt(s, Wd, ldwd, pc.n, m, rk, pc.dP, pc.ldp, upper), 1);
        else
            PSD_KL(launch_syrk_tc(s, ctx->persist_sms, Wd, ldwd, pc.n, m, rk, pc.dP, pc.ldp, upper, ws.Xhi,
                                  ws.Xlo, ws.ld, ctx->d_status, ctx->wait_limit, pc.w_split ? 1 : 0),
                   pc.w_split ? 1 : 2);
    }
    if (pc.d_rank && !pc.rank_written)
        PSD_CK(cudaMemcpyAsync(pc.d_rank, rk, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return PSDPROJ_OK;
}

// omega_ready: the workspace's Omega already holds the test matrix (warm
// start of Alg. 6); it is not drawn again
int run_projection(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda, int k, int p,
                   int q, uint64_t seed, bool scaled, double alpha_in, double *d_alpha_out,
                   int *d_info, float *dP, int64_t ldp, float *dW, int64_t ldw, int *d_rank,
                   const psdproj_opts *opts_in, bool omega_ready = false)
{
    if (!ctx) return PSDPROJ_EINVAL;
    psdproj_opts opts;
    if (opts_in) opts = *opts_in; else psdproj_default_opts(&opts);
    PSD_TRY(check_opts(&opts));
    PSD_TRY(validate(n, lda, k, p, q, dA));
    if (opts.out_mode != PSDPROJ_OUT_FACTOR && (!dP || ldp < n)) return PSDPROJ_EINVAL;
    if (dW && ldw < n) return PSDPROJ_EINVAL;
    const int m = k + p;
    device_guard g(ctx->device);
    // per-call settings read by the launches below, cleared again on return
    // (the step-level entry points take neither)
    struct call_settings {
        psdproj_ctx *c;
        ~call_settings() { c->wait_limit = 0; c->det = false; }
    } settings_scope{ctx};
    ctx->wait_limit = (long long)opts.spin_limit;
    ctx->det = opts.deterministic != 0;
    if (ctx->det) opts.prec = PSDPROJ_PREC_FP32;     // every product with A: the fixed-order FP32 kernels
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    if (ctx->det)
        PSD_TRY(ensure_stage(ctx, &ctx->det_part, &ctx->det_part_bytes,
                             sizeof(float) * (size_t)psd_det_part_floats(n, m), ctx->stream));
    psd_workspace &ws = ctx->ws;
    proj_call pc;
    pc.dA = dA;
    pc.n = n;
    pc.lda = lda;
    pc.k = k;
    pc.p = p;
    pc.q = q;
    pc.m = m;
    pc.seed = seed;
    pc.scaled = scaled;
    pc.alpha_in = alpha_in;
    pc.d_alpha_out = d_alpha_out;
    pc.d_info = d_info;
    pc.dP = dP;
    pc.ldp = ldp;
    pc.dW = dW;
    pc.ldw = ldw;
    pc.d_rank = d_rank;
    pc.opts = opts;
    pc.omega_ready = omega_ready;
    PSD_TRY(proj_begin(ctx, pc));
    // the orthonormalisation after product t writes the side outputs of the
    // next pass: a power product (shifted) while t < 2q, else the core (Y = 0)
    // (one CholeskyQR pass where a power product follows, both before the core)
    {
        const psd_bf16_side sd = proj_side(ctx, q > 0 ? pc.shift : nullptr);
        PSD_TRY(cholqr2(ctx, ws.Y, ws.ld, n, m, ws.Q, ws.ld, ws.ints + IN_QRANK, pc.fuse ? &sd : nullptr,
                        q > 0 ? 1 : 2));
    }
    for (int t = 0; t < 2 * q; ++t) {
        PSD_TRY(proj_power_pass(ctx, pc));
        const psd_bf16_side sd = proj_side(ctx, t + 1 < 2 * q ? pc.shift : nullptr);
        PSD_TRY(cholqr2(ctx, ws.Y, ws.ld, n, m, ws.Q, ws.ld, ws.ints + IN_QRANK, pc.fuse ? &sd : nullptr,
                        t + 1 < 2 * q ? 1 : 2));
    }
    PSD_TRY(proj_core_pass(ctx, pc));
    PSD_TRY(proj_core_small(ctx, pc));
    return proj_finish(ctx, pc);
}

int ensure_stage(psdproj_ctx *ctx, float **buf, size_t *cap, size_t bytes, cudaStream_t s)
{
    if (*cap >= bytes) return PSDPROJ_OK;
    PSD_TRY(psd_budget_check(ctx, *cap, bytes));
    if (*buf) {
        cudaStreamSynchronize(s);
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) return cuda_status(e, __LINE__);
    *cap = bytes;
    return PSDPROJ_OK;
}

int run_host(psdproj_ctx *ctx, const float *hA, int64_t n, int64_t lda, int k, int p, int q,
             uint64_t seed, bool scaled, double alpha_in, double *h_alpha, float *hP,
             int64_t ldp, float *hW, int64_t ldw, int *h_rank, const psdproj_opts *opts_in)
{
    if (!ctx) return PSDPROJ_EINVAL;
    psdproj_opts opts;
    if (opts_in) opts = *opts_in; else psdproj_default_opts(&opts);
    PSD_TRY(check_opts(&opts));
    PSD_TRY(validate(n, lda, k, p, q, hA));
    const bool wantP = opts.out_mode != PSDPROJ_OUT_FACTOR;
    if (wantP && (!hP || ldp < n)) return PSDPROJ_EINVAL;
    if (hW && ldw < n) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    cudaStream_t s = ctx->stream;
    const int m = k + p;
    PSD_TRY(ensure_stage(ctx, &ctx->dA_stage, &ctx->dA_stage_bytes, sizeof(float) * n * n, s));
    if (wantP) PSD_TRY(ensure_stage(ctx, &ctx->dP_stage, &ctx->dP_stage_bytes, sizeof(float) * n * n, s));
    if (hW) PSD_TRY(ensure_stage(ctx, &ctx->dW_stage, &ctx->dW_stage_bytes, sizeof(float) * n * m, s));
    // Only A's upper triangle is ever read.  Pinned host memory is reachable
    // from the GPU (NVLink-C2C), so the device reads that half of A over the
    // link: the BF16 form packs its image straight from the host buffer (it
    // reads A nowhere else), the others gather it into the staging buffer
    // with a kernel.  Other host memory is copied whole (one contiguous copy
    // when lda == n).
    cudaPointerAttributes pa;
    const bool mapped = cudaPointerGetAttributes(&pa, hA) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                        pa.devicePointer != nullptr;
    if (!mapped) cudaGetLastError();            // clear the query's error for unregistered memory
    const float *dA = ctx->dA_stage;
    int64_t ldA = n;
    if (mapped && opts.prec == PSDPROJ_PREC_BF16) {
        dA = static_cast<const float *>(pa.devicePointer);
        ldA = lda;
    } else if (mapped) {
        PSD_KL(launch_copy_upper(s, static_cast<const float *>(pa.devicePointer), n, lda, ctx->dA_stage, n), 1);
    } else {
        PSD_CK(cudaMemcpy2DAsync(ctx->dA_stage, sizeof(float) * n, hA, sizeof(float) * lda,
                                 sizeof(float) * n, n, cudaMemcpyHostToDevice, s));
    }
    PSD_TRY(run_projection(ctx, dA, n, ldA, k, p, q, seed, scaled, alpha_in,
                           ctx->d_misc_f, ctx->d_misc + 1, wantP ? ctx->dP_stage : nullptr, n,
                           hW ? ctx->dW_stage : nullptr, n, ctx->d_misc, &opts));
    if (wantP)
        PSD_CK(cudaMemcpy2DAsync(hP, sizeof(float) * ldp, ctx->dP_stage, sizeof(float) * n,
                                 sizeof(float) * n, n, cudaMemcpyDeviceToHost, s));
    if (hW)
        PSD_CK(cudaMemcpy2DAsync(hW, sizeof(float) * ldw, ctx->dW_stage, sizeof(float) * n,
                                 sizeof(float) * n, m, cudaMemcpyDeviceToHost, s));
    if (h_rank) PSD_CK(cudaMemcpyAsync(h_rank, ctx->d_misc, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (h_alpha && scaled)
        PSD_CK(cudaMemcpyAsync(h_alpha, ctx->d_misc_f, sizeof(double), cudaMemcpyDeviceToHost, s));
    return psdproj_sync_status(ctx);
}

}  // namespace

extern "C" {

void psdproj_default_opts(psdproj_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->prec = PSDPROJ_PREC_FP32;
    o->syrk_prec = PSDPROJ_PREC_FP32;
    o->N = 10;
    o->out_mode = PSDPROJ_OUT_FULL;
}

int psdproj_create(psdproj_ctx **out, int device, void *stream, size_t hbm_budget_bytes)
{
    if (!out) return PSDPROJ_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return PSDPROJ_EINVAL;
    device_guard g(device);
    psdproj_ctx *c = new (std::nothrow) psdproj_ctx();
    if (!c) return PSDPROJ_ENOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    c->budget = hbm_budget_bytes;
    c->root = c;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    // persistent kernels (one CTA per SM for the whole pass) leave one SM to
    // single-block kernels that another stream may run at the same time: a
    // CTA that found no free SM would otherwise start only when another
    // finished, doubling the pass
    c->persist_sms = c->sm_count > 8 ? c->sm_count - 1 : c->sm_count;
    cudaError_t e = cudaMalloc(&c->d_status, 64);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_misc, 64);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_misc_f, 64);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, 64);
    if (e == cudaSuccess) e = cudaMemset(c->d_misc, 0, 64);
    if (e != cudaSuccess) {
        psdproj_destroy(c);
        return cuda_status(e, __LINE__);
    }
    *out = c;
    return PSDPROJ_OK;
}

int psdproj_set_stream(psdproj_ctx *ctx, void *stream)
{
    if (!ctx) return PSDPROJ_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return PSDPROJ_OK;
}

int psdproj_destroy(psdproj_ctx *ctx)
{
    if (!ctx) return PSDPROJ_OK;
    device_guard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_workspace(ctx->ws);
    if (ctx->timing.created)
        for (int i = 0; i < 2 * PSD_MAX_TIMED; ++i) cudaEventDestroy(ctx->timing.ev[i]);
    if (ctx->d_status && ctx->owns_status) cudaFree(ctx->d_status);
    if (ctx->d_misc) cudaFree(ctx->d_misc);
    if (ctx->d_misc_f) cudaFree(ctx->d_misc_f);
    if (ctx->dA_stage) cudaFree(ctx->dA_stage);
    if (ctx->dP_stage) cudaFree(ctx->dP_stage);
    if (ctx->dW_stage) cudaFree(ctx->dW_stage);
    if (ctx->det_part) cudaFree(ctx->det_part);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->g_exec) cudaGraphExecDestroy(ctx->g_exec);
    for (int w = 0; w < 2; ++w) {
        if (ctx->g_slots[w]) cudaFree(ctx->g_slots[w]);
        if (ctx->g_tabs[w]) cudaFree(ctx->g_tabs[w]);
        if (ctx->g_ev[w]) cudaEventDestroy(ctx->g_ev[w]);
    }
    if (ctx->g_stream2) cudaStreamDestroy(ctx->g_stream2);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->Ab) cudaFree(ctx->Ab);
    if (ctx->Ab_lo) cudaFree(ctx->Ab_lo);
    for (int i = 0; i < PSD_MAX_LANES; ++i) {
        if (ctx->lane[i]) psdproj_destroy(ctx->lane[i]);
        if (ctx->lane_ev[i]) cudaEventDestroy(ctx->lane_ev[i]);
    }
    if (ctx->lane_ev[PSD_MAX_LANES]) cudaEventDestroy(ctx->lane_ev[PSD_MAX_LANES]);
    if (ctx->owns_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return PSDPROJ_OK;
}

int psdproj_set_batch_streams(psdproj_ctx *ctx, int streams)
{
    if (!ctx || streams < 1 || streams > PSD_MAX_LANES) return PSDPROJ_EINVAL;
    ctx->batch_streams = streams;
    ctx->lanes_explicit = true;
    return PSDPROJ_OK;
}

// ---- batch tuning table ----------------------------------------------------
// (device name, SM count, floor(log2 median side), floor(log2 count)) ->
// lane count; kept in memory and, when PSDPROJ_TUNE_CACHE names a file, in
// that file (one "key<TAB>streams" line per entry); when the variable names
// another file than the one last read, the table becomes that file's contents.
namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
std::string g_tune_file;          // the file g_tune was last read from

int ilog2(int64_t x)
{
    int r = 0;
    while (x > 1) {
        x >>= 1;
        ++r;
    }
    return r;
}

std::string tune_key(const char *device, int sm_count, int64_t median_n, int count)
{
    std::string name = device ? device : "";
    for (char &c : name)
        if (c == ' ' || c == '\t' || c == '\n') c = '_';
    return name + ":" + std::to_string(sm_count) + ":" + std::to_string(ilog2(median_n)) + ":" +
           std::to_string(ilog2(count));
}

// with g_tune_mu held
void tune_sync_file()
{
    const char *f = getenv("PSDPROJ_TUNE_CACHE");
    const std::string path = f ? f : "";
    if (path == g_tune_file) return;
    // another file: the table becomes its contents
    g_tune_file = path;
    g_tune.clear();
    if (path.empty()) return;
    FILE *fp = fopen(path.c_str(), "r");
    if (!fp) return;
    char line[512];
    while (fgets(line, sizeof line, fp)) {
        char *tab = strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        const int v = atoi(tab + 1);
        if (v >= 1 && v <= PSD_MAX_LANES) g_tune[line] = v;
    }
    fclose(fp);
}

int env_batch_streams()
{
    const char *e = getenv("PSDPROJ_BATCH_STREAMS");
    if (!e) return 0;
    const int v = atoi(e);
    return (v >= 1 && v <= PSD_MAX_LANES) ? v : 0;
}

struct dev_ident {
    char name[256];
    int sms;
};

dev_ident device_ident(int device)
{
    dev_ident d{};
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
        snprintf(d.name, sizeof d.name, "%s", prop.name);
        d.sms = prop.multiProcessorCount;
    } else {
        snprintf(d.name, sizeof d.name, "device%d", device);
    }
    return d;
}

int64_t median_side(int count, const psdproj_problem *probs)
{
    std::vector<int64_t> v((size_t)count);
    for (int i = 0; i < count; ++i) v[(size_t)i] = probs[i].n;
    std::nth_element(v.begin(), v.begin() + count / 2, v.end());
    return v[(size_t)count / 2];
}

}  // namespace

int psdproj_tune_lookup(const char *device_name, int sm_count, int64_t median_n, int count, int *streams)
{
    if (!device_name || !streams || median_n < 1 || count < 1) return PSDPROJ_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_sync_file();
    const auto it = g_tune.find(tune_key(device_name, sm_count, median_n, count));
    if (it == g_tune.end()) return PSDPROJ_EINVAL;
    *streams = it->second;
    return PSDPROJ_OK;
}

int psdproj_tune_store(const char *device_name, int sm_count, int64_t median_n, int count, int streams)
{
    if (!device_name || median_n < 1 || count < 1 || streams < 1 || streams > PSD_MAX_LANES) return PSDPROJ_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_sync_file();
    g_tune[tune_key(device_name, sm_count, median_n, count)] = streams;
    if (!g_tune_file.empty()) {
        FILE *fp = fopen(g_tune_file.c_str(), "w");
        if (!fp) return PSDPROJ_EINVAL;
        for (const auto &kv : g_tune) fprintf(fp, "%s\t%d\n", kv.first.c_str(), kv.second);
        fclose(fp);
    }
    return PSDPROJ_OK;
}

int psdproj_set_reserved_sms(psdproj_ctx *ctx, int sms)
{
    if (!ctx || sms < 0 || sms >= ctx->sm_count) return PSDPROJ_EINVAL;
    ctx->persist_sms = ctx->sm_count - sms;
    for (int i = 0; i < PSD_MAX_LANES; ++i)
        if (ctx->lane[i]) ctx->lane[i]->persist_sms = ctx->persist_sms;
    return PSDPROJ_OK;
}

int psdproj_sync_status(psdproj_ctx *ctx)
{
    if (!ctx) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_status(e, __LINE__);
    int st = 0;
    e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e, __LINE__);
    if (st) cudaMemset(ctx->d_status, 0, sizeof(int));
    return st;
}

int psdproj_last_cuda_error(int *line)
{
    if (line) *line = t_last_line;
    return t_last_cuda;
}

const char *psdproj_status_string(int s)
{
    switch (s) {
    case PSDPROJ_OK: return "PSDPROJ_OK";
    case PSDPROJ_EINVAL: return "PSDPROJ_EINVAL: invalid argument";
    case PSDPROJ_ENOMEM: return "PSDPROJ_ENOMEM: device allocation failed";
    case PSDPROJ_ENOTFINITE: return "PSDPROJ_ENOTFINITE: non-finite value";
    case PSDPROJ_ENOCONV: return "PSDPROJ_ENOCONV: eigensolver did not converge";
    case PSDPROJ_ETIMEOUT: return "PSDPROJ_ETIMEOUT: device wait gave up";
    case PSDPROJ_ECUDA: return "PSDPROJ_ECUDA: CUDA error";
    case PSDPROJ_ENOTSUP: return "PSDPROJ_ENOTSUP: unsupported option";
    case PSDPROJ_ETOOLARGE: return "PSDPROJ_ETOOLARGE: size above the fixed scratch capacity";
    default: return "PSDPROJ: unknown status";
    }
}

size_t psdproj_workspace_bytes(const psdproj_ctx *ctx)
{
    if (!ctx) return 0;
    size_t b = ctx->ws.bytes + ctx->Ab_bytes + ctx->Ab_lo_bytes + ctx->dA_stage_bytes + ctx->dP_stage_bytes +
               ctx->dW_stage_bytes + ctx->det_part_bytes + ctx->g_slots_bytes[0] + ctx->g_slots_bytes[1] +
               ctx->g_tabs_bytes[0] + ctx->g_tabs_bytes[1];
    for (int i = 0; i < PSD_MAX_LANES; ++i)
        if (ctx->lane[i]) b += psdproj_workspace_bytes(ctx->lane[i]);
    return b;
}

int psdproj_timing_enable(psdproj_ctx *ctx, int on)
{
    if (!ctx) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    psd_timing &t = ctx->timing;
    if (on && !t.created) {
        for (int i = 0; i < 2 * PSD_MAX_TIMED; ++i) PSD_CK(cudaEventCreate(&t.ev[i]));
        t.created = true;
    }
    t.on = on ? 1 : 0;
    return PSDPROJ_OK;
}

int psdproj_timing_read(psdproj_ctx *ctx, double *ms, int *count, int nkinds)
{
    if (!ctx || nkinds < 0 || nkinds > PSDPROJ_NSTAGES) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_CK(cudaStreamSynchronize(ctx->stream));
    psd_timing &t = ctx->timing;
    for (int i = 0; i < t.n; ++i) {
        float e = 0.0f;
        PSD_CK(cudaEventElapsedTime(&e, t.ev[2 * i], t.ev[2 * i + 1]));
        const int k = t.kind[i];
        if (k < nkinds) {
            if (ms) ms[k] += e;
            if (count) count[k] += 1;
        }
    }
    t.n = 0;
    return PSDPROJ_OK;
}

uint64_t psdproj_kernel_launches(void) { return g_launches.load(); }

size_t psdproj_projection_bytes(int64_t n, int k, int p, const psdproj_opts *opts_in)
{
    psdproj_opts o;
    if (opts_in) o = *opts_in; else psdproj_default_opts(&o);
    if (n < 1 || k < 1 || p < 0 || (int64_t)k + p > n || k + p > PSD_MAX_M || check_opts(&o) != PSDPROJ_OK)
        return 0;
    return psd_projection_device_bytes(n, k + p, o.prec, o.deterministic);
}

int psdproj_alg1(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda, int k, int p, int q,
                 uint64_t seed, float *dP, int64_t ldp, float *dW, int64_t ldw, int *d_rank,
                 const psdproj_opts *opts)
{
    return run_projection(ctx, dA, n, lda, k, p, q, seed, false, 0.0, nullptr, nullptr, dP, ldp, dW,
                          ldw, d_rank, opts);
}

int psdproj_alg2(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda, int k, int p, int q,
                 uint64_t seed, double alpha_in, double *d_alpha_out, int *d_info, float *dP,
                 int64_t ldp, float *dW, int64_t ldw, int *d_rank, const psdproj_opts *opts)
{
    return run_projection(ctx, dA, n, lda, k, p, q, seed, true, alpha_in, d_alpha_out, d_info, dP,
                          ldp, dW, ldw, d_rank, opts);
}

// Lane j of a batch: a helper context on its own non-blocking stream that
// shares ctx's device status word; created on first use with its events.
int ensure_lane(psdproj_ctx *ctx, int j)
{
    if (ctx->lane[j]) return PSDPROJ_OK;
    if (!ctx->lane_ev[PSD_MAX_LANES])
        PSD_CK(cudaEventCreateWithFlags(&ctx->lane_ev[PSD_MAX_LANES], cudaEventDisableTiming));
    if (!ctx->lane_ev[j]) PSD_CK(cudaEventCreateWithFlags(&ctx->lane_ev[j], cudaEventDisableTiming));
    psdproj_ctx *c = new (std::nothrow) psdproj_ctx();
    if (!c) return PSDPROJ_ENOMEM;
    c->device = ctx->device;
    c->sm_count = ctx->sm_count;
    c->persist_sms = ctx->persist_sms;
    c->root = ctx->root ? ctx->root : ctx;
    c->batch_streams = 1;
    c->owns_status = false;
    c->d_status = ctx->d_status;
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) c->owns_stream = true;
    if (e == cudaSuccess) e = cudaMalloc(&c->d_misc, 64);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_misc_f, 64);
    if (e == cudaSuccess) e = cudaMemset(c->d_misc, 0, 64);
    if (e != cudaSuccess) {
        psdproj_destroy(c);
        return cuda_status(e, __LINE__);
    }
    ctx->lane[j] = c;
    return PSDPROJ_OK;
}

}  // extern "C"

namespace {

// A batch's plan: the problems spread over S lanes (own stream and
// workspace) by longest-processing-time-first on the cost n^2 (2q + 2 +
// [alg 2] 2(N + 1)), issued largest first so that the long ones start early.
struct batch_plan {
    int S = 1;
    std::vector<int> order, lane_of;
};

int batch_validate(const psdproj_opts &opts, int count, const psdproj_problem *probs, int64_t &nmax, int &mmax)
{
    nmax = 0;
    mmax = 0;
    for (int i = 0; i < count; ++i) {
        const psdproj_problem &pb = probs[i];
        PSD_TRY(validate(pb.n, pb.lda, pb.k, pb.p, pb.q, pb.dA));
        if (pb.algorithm != 1 && pb.algorithm != 2) return PSDPROJ_EINVAL;
        if (opts.out_mode != PSDPROJ_OUT_FACTOR && (!pb.dP || pb.ldp < pb.n)) return PSDPROJ_EINVAL;
        if (pb.dW && pb.ldw < pb.n) return PSDPROJ_EINVAL;
        if (pb.n > nmax) nmax = pb.n;
        if (pb.k + pb.p > mmax) mmax = pb.k + pb.p;
    }
    return PSDPROJ_OK;
}

// The lane count of a batch: PSDPROJ_BATCH_STREAMS if set; a trial of
// psdproj_tune_batch; the context's own setting if it was made
// (psdproj_set_batch_streams, or a finished tuning); the tuning table's entry
// for the batch's bucket; else the default (8).
int batch_lanes(const psdproj_ctx *ctx, int count, const psdproj_problem *probs)
{
    if (const int e = env_batch_streams()) return e;
    if (ctx->tune_force > 0) return ctx->tune_force;
    if (ctx->lanes_explicit || count < 1) return ctx->batch_streams;
    const dev_ident d = device_ident(ctx->device);
    int v = 0;
    if (psdproj_tune_lookup(d.name, d.sms, median_side(count, probs), count, &v) == PSDPROJ_OK) return v;
    return ctx->batch_streams;
}

batch_plan batch_make_plan(const psdproj_ctx *ctx, const psdproj_opts &opts, int count, const psdproj_problem *probs,
                           int lanes)
{
    batch_plan pl;
    pl.S = count < lanes ? count : lanes;
    pl.order.resize(count);
    pl.lane_of.assign(count, 0);
    std::vector<double> cost(count), load(pl.S > 0 ? pl.S : 1, 0.0);
    for (int i = 0; i < count; ++i) {
        const psdproj_problem &pb = probs[i];
        pl.order[i] = i;
        cost[i] = (double)pb.n * (double)pb.n * (2.0 * pb.q + 2.0 + (pb.algorithm == 2 ? 2.0 * (opts.N + 1) : 0.0));
    }
    std::stable_sort(pl.order.begin(), pl.order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    if (pl.S > 1)
        for (int i : pl.order) {
            int best = 0;
            for (int j = 1; j < pl.S; ++j)
                if (load[j] < load[best]) best = j;
            pl.lane_of[i] = best;
            load[best] += cost[i];
        }
    return pl;
}

// Every workspace and image a plan's problems will use, allocated now (so
// that issuing the batch allocates nothing: required inside a graph capture).
int batch_presize(psdproj_ctx *ctx, const batch_plan &pl, const psdproj_opts &opts, int count,
                  const psdproj_problem *probs)
{
    const int nl = pl.S > 1 ? pl.S : 1;
    for (int j = 0; j < nl; ++j) {
        psdproj_ctx *c = pl.S > 1 ? ctx->lane[j] : ctx;
        int64_t nmax = 0;
        int mmax = 0;
        for (int i = 0; i < count; ++i) {
            if (pl.S > 1 && pl.lane_of[i] != j) continue;
            if (probs[i].n > nmax) nmax = probs[i].n;
            if (probs[i].k + probs[i].p > mmax) mmax = probs[i].k + probs[i].p;
        }
        if (nmax == 0) continue;
        PSD_TRY(psd_ensure_workspace(c, nmax, mmax));
        if (opts.deterministic) {
            PSD_TRY(ensure_stage(c, &c->det_part, &c->det_part_bytes,
                                 sizeof(float) * (size_t)psd_det_part_floats(nmax, mmax), c->stream));
        } else if (opts.prec == PSDPROJ_PREC_TF32) {
            PSD_TRY(alloc_image(c, &c->Ab, &c->Ab_bytes, (size_t)psd_tile32_count(nmax) * PSD_TILE_BYTES, c->stream));
        } else if (opts.prec != PSDPROJ_PREC_FP32) {
            const size_t b = (size_t)psd_tile_count(nmax) * PSD_TILE_BYTES;
            PSD_TRY(alloc_image(c, &c->Ab, &c->Ab_bytes, b, c->stream));
            if (opts.prec == PSDPROJ_PREC_BF16X3) PSD_TRY(alloc_image(c, &c->Ab_lo, &c->Ab_lo_bytes, b, c->stream));
        }
    }
    return PSDPROJ_OK;
}

// Issue a planned batch on the context's stream (fork to the lanes, join back).
int batch_issue(psdproj_ctx *ctx, const batch_plan &pl, const psdproj_opts &opts, int count,
                const psdproj_problem *probs)
{
    auto run_one = [&](psdproj_ctx *c, const psdproj_problem &pb) {
        return run_projection(c, pb.dA, pb.n, pb.lda, pb.k, pb.p, pb.q, pb.seed, pb.algorithm == 2, pb.alpha_in,
                              pb.d_alpha_out, pb.d_info, pb.dP, pb.ldp, pb.dW, pb.ldw, pb.d_rank, &opts);
    };
    if (pl.S <= 1) {
        for (int i = 0; i < count; ++i) PSD_TRY(run_one(ctx, probs[i]));
        return PSDPROJ_OK;
    }
    cudaEvent_t fork = ctx->lane_ev[PSD_MAX_LANES];
    PSD_CK(cudaEventRecord(fork, ctx->stream));
    for (int j = 0; j < pl.S; ++j) PSD_CK(cudaStreamWaitEvent(ctx->lane[j]->stream, fork, 0));
    int rc = PSDPROJ_OK;
    for (int i : pl.order) {
        rc = run_one(ctx->lane[pl.lane_of[i]], probs[i]);
        if (rc != PSDPROJ_OK) break;
    }
    // join every lane back, also after an error, so that the context's stream
    // orders after all the work the batch issued
    for (int j = 0; j < pl.S; ++j) {
        cudaEventRecord(ctx->lane_ev[j], ctx->lane[j]->stream);
        cudaStreamWaitEvent(ctx->stream, ctx->lane_ev[j], 0);
    }
    return rc;
}

void batch_graph_free(psdproj_ctx *ctx)
{
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    ctx->graph_probs.clear();
    ctx->graph_launches = 0;
}

// ---- grouped batch (psdproj_batched_grouped) -------------------------------
// Every problem gets a workspace and image(s) of its own (one allocation), so
// that all of them are in flight together, and the batch runs phase by phase:
// the streaming phases (image, alpha, the products with A, the SYRK) per
// problem on the lanes, and each small step of the orthonormalisations and of
// the core (Gram, Cholesky, tall x small product, eigensolver, factor) as one
// grouped launch over all problems on the context's stream, where the
// single-problem path runs one block (or a few) per launch.

struct grouped_slot {
    psd_workspace ws;
    uint16_t *Ab = nullptr, *Ab_lo = nullptr;
    size_t Ab_bytes = 0, Ab_lo_bytes = 0;
};

// a grouped launch in device memory: its table and block maps
struct gl_gram {
    const psd_g_gram *tab = nullptr;
    const int2 *bm = nullptr, *bm_red = nullptr;
    int nb = 0, nb_red = 0;
};
struct gl_tall {
    const psd_g_tall *tab = nullptr;
    const int2 *bm = nullptr;
    int nb = 0;
};
struct gl_qr {                 // one CholeskyQR2 over the problems of a stage
    int count = 0, count2 = 0;    // problems; those that take the second half
    gl_gram g1, g2;
    const psd_g_chol *c1 = nullptr, *c2 = nullptr;
    gl_tall t1, t2;
};
struct gl_core {               // core, eigensolver, factor
    int count = 0;
    gl_gram g;
    const psd_g_eig *eig = nullptr;
    const int2 *bm_ns = nullptr, *bm_ray = nullptr;
    int nb_ns = 0, nb_ray = 0;
    const psd_g_factor *fac = nullptr;
    gl_tall t;
};

struct grouped_plan {
    batch_plan lanes;          // lane_of: relative to lane0
    int lane0 = 0;             // the plan's first lane (ctx->lane[lane0 + j])
    std::vector<grouped_slot> slot;
    std::vector<proj_call> pc;
    int qmax = 0, m_max = 0, mp_max = 0;
    std::vector<gl_qr> qr;     // stage s: the orthonormalisation after product s - 1 (s = 0: after Y = A Omega)
    gl_core core;
    // Alg. 3's alpha by grouped power iterations (BF16 form, alpha not given,
    // not the Ritz variant): which problems, and the launches' tables
    std::vector<char> galpha;
    int n_galpha = 0, N = 0;
    const psd_g_pi *pi1 = nullptr, *pi2 = nullptr;
    const int2 *bm_pi = nullptr;
    int nb_pi = 0;
    const psd_g_alpha *al = nullptr;
    // grouped images (BF16 forms) and test matrices (Gaussian sketch)
    bool gpack = false, gpack_lo = false;
    const psd_g_pack *pk = nullptr, *pk_lo = nullptr;
    const int2 *bm_pk = nullptr;
    int nb_pk = 0;
    const psd_g_gauss *gs = nullptr;
    const int2 *bm_gs = nullptr;
    int nb_gs = 0;
};

// alpha of this problem comes from the grouped power iterations
bool grouped_alpha(const proj_call &pc)
{
    return pc.scaled && !proj_ritz(pc) && !(pc.alpha_in > 0.0) && pc.opts.prec == PSDPROJ_PREC_BF16;
}

// image bytes of one problem in form prec: (high or only part, low part)
void slot_image_bytes(int64_t n, int prec, size_t &hi, size_t &lo)
{
    hi = lo = 0;
    if (prec == PSDPROJ_PREC_TF32) hi = (size_t)psd_tile32_count(n) * (size_t)PSD_TILE_BYTES;
    else if (prec == PSDPROJ_PREC_BF16) hi = (size_t)psd_tile_count(n) * (size_t)PSD_TILE_BYTES;
    else if (prec == PSDPROJ_PREC_BF16X3) hi = lo = (size_t)psd_tile_count(n) * (size_t)PSD_TILE_BYTES;
}

size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// Per-problem workspaces and images, carved from ctx->g_slots[w] (grown when
// too small; zeroed whenever the plan is made, as a workspace is when
// allocated)
int grouped_slots(psdproj_ctx *ctx, int w, const psdproj_opts &opts, int count, const psdproj_problem *probs,
                  std::vector<grouped_slot> &slot)
{
    slot.assign(count, grouped_slot());
    std::vector<size_t> off(count);
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        psd_workspace lay;
        const int lp = psd_lpad(probs[i].k + probs[i].p);
        size_t hi, lo;
        slot_image_bytes(probs[i].n, opts.prec, hi, lo);
        off[i] = total;
        total += align_up(carve_workspace(lay, nullptr, probs[i].n, lp), 1024) + align_up(hi, 1024) +
                 align_up(lo, 1024);
    }
    if (ctx->g_slots_bytes[w] < total) {
        PSD_TRY(psd_budget_check(ctx, ctx->g_slots_bytes[w], total));
        if (ctx->g_slots[w]) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->g_slots[w]);
            ctx->g_slots[w] = nullptr;
            ctx->g_slots_bytes[w] = 0;
        }
        PSD_CK(cudaMalloc(&ctx->g_slots[w], total));
        ctx->g_slots_bytes[w] = total;
    }
    char *base = static_cast<char *>(ctx->g_slots[w]);
    for (int i = 0; i < count; ++i) {
        grouped_slot &sl = slot[i];
        const int64_t n = probs[i].n;
        const int lp = psd_lpad(probs[i].k + probs[i].p);
        char *b = base + off[i];
        const size_t wb = carve_workspace(sl.ws, b, n, lp);
        sl.ws.base = nullptr;              // part of g_slots: never freed on its own
        sl.ws.bytes = 0;
        sl.ws.n = n;
        sl.ws.lpad = lp;
        sl.ws.ld = psd_ld(n);
        size_t hi, lo;
        slot_image_bytes(n, opts.prec, hi, lo);
        char *img = b + align_up(wb, 1024);
        if (hi) {
            sl.Ab = reinterpret_cast<uint16_t *>(img);
            sl.Ab_bytes = hi;
        }
        if (lo) {
            sl.Ab_lo = reinterpret_cast<uint16_t *>(img + align_up(hi, 1024));
            sl.Ab_lo_bytes = lo;
        }
    }
    PSD_CK(cudaMemsetAsync(ctx->g_slots[w], 0, total, ctx->stream));
    return PSDPROJ_OK;
}

// Host copies of the grouped tables, laid out for one upload
struct table_blob {
    std::vector<char> h;
    template <class T>
    size_t put(const std::vector<T> &v)
    {
        const size_t off = align_up(h.size(), 64);
        h.resize(off + sizeof(T) * v.size());
        if (!v.empty()) memcpy(h.data() + off, v.data(), sizeof(T) * v.size());
        return off;
    }
};

// table offsets of a grouped launch before the upload
struct gram_off { size_t tab, bm, bm_red; int nb, nb_red; };
struct tall_off { size_t tab, bm; int nb; };

gram_off put_gram(table_blob &tb, const std::vector<psd_g_gram> &t)
{
    std::vector<int2> bm, bmr;
    for (int e = 0; e < (int)t.size(); ++e) {
        for (int b = 0; b < t[e].nblk; ++b) bm.push_back(make_int2(e, b));
        const int nr = psd_gram_reduce_grouped_blocks(t[e].m, t[e].nblk);
        for (int b = 0; b < nr; ++b) bmr.push_back(make_int2(e, b));
    }
    gram_off o;
    o.tab = tb.put(t);
    o.bm = tb.put(bm);
    o.bm_red = tb.put(bmr);
    o.nb = (int)bm.size();
    o.nb_red = (int)bmr.size();
    return o;
}

tall_off put_tall(table_blob &tb, const std::vector<psd_g_tall> &t)
{
    std::vector<int2> bm;
    for (int e = 0; e < (int)t.size(); ++e)
        for (int b = 0; b < t[e].nb; ++b) bm.push_back(make_int2(e, b));
    tall_off o;
    o.tab = tb.put(t);
    o.bm = tb.put(bm);
    o.nb = (int)bm.size();
    return o;
}

psd_g_gram gram_entry(const psd_workspace &ws, const float *X, const float *Z, int64_t n, int m, double *G,
                      float2 *Gdf, int sms)
{
    psd_g_gram g;
    g.X = X;
    g.Z = Z;
    g.ldx = g.ldz = ws.ld;
    g.n = n;
    g.m = m;
    g.mp = (int)psd_round_up(m, 8);
    g.rows = (int)psd_gram_rows(n, sms);
    g.nblk = psd_gram_blocks(n, sms);
    g.gpart = ws.gpart;
    g.G = G;
    g.Gdf = Gdf;
    return g;
}

psd_g_tall tall_entry(const float *Y, int64_t ldy, int64_t n, int m, const float *B, const int *colmask,
                      const int *d_cols, float *Z, int64_t ldz, const psd_bf16_side *side)
{
    psd_g_tall t;
    t.Y = Y;
    t.ldy = ldy;
    t.n = n;
    t.m = m;
    t.B = B;
    t.c = m;
    t.colmask = colmask;
    t.d_cols = d_cols;
    t.Z = Z;
    t.ldz = ldz;
    t.side = side ? *side : psd_bf16_side{nullptr, 0, nullptr, 0, nullptr};
    t.ntiles = (int)((n + PSD_TALL_RT - 1) / PSD_TALL_RT);
    // four tiles (128 rows) per block: the block's copy of B is read once per four
    t.nb = (t.ntiles + 3) / 4;
    return t;
}

// The tables of every grouped launch of the batch, uploaded to ctx->g_tabs[w]
int grouped_tables(psdproj_ctx *ctx, int w, grouped_plan &gp)
{
    const int count = (int)gp.pc.size();
    const int sms = ctx->persist_sms;
    table_blob tb;
    struct qr_off { int count, count2; gram_off g1, g2; size_t c1, c2; tall_off t1, t2; };
    std::vector<qr_off> qo;
    for (int st = 0; st <= 2 * gp.qmax; ++st) {
        std::vector<psd_g_gram> g1, g2;
        std::vector<psd_g_chol> c1, c2;
        std::vector<psd_g_tall> t1, t2;
        for (int i = 0; i < count; ++i) {
            const proj_call &pc = gp.pc[i];
            if (st > 0 && st > 2 * pc.q) continue;      // product st - 1 is not one of this problem's
            const psd_workspace &ws = gp.slot[i].ws;
            const int64_t n = pc.n;
            const int m = pc.m;
            float2 *gdf = reinterpret_cast<float2 *>(ws.cholscr);
            // the side outputs of the pass that reads Q next: a power product
            // (shifted) while product st is one of the problem's, else the
            // core; before a power product the first half alone (cholqr2's
            // passes = 1) writes Q
            const bool one = st < 2 * pc.q;
            const psd_bf16_side sd{ws.Xhi, ws.ld, ws.Y, ws.ld, one ? proj_shift(pc, ws) : nullptr};
            const psd_bf16_side *sdp = proj_fuse(pc) ? &sd : nullptr;
            g1.push_back(gram_entry(ws, ws.Y, ws.Y, n, m, ws.G, gdf, sms));
            c1.push_back(psd_g_chol{gdf, m, ws.Rinv, ws.dead, one ? ws.ints + IN_QRANK : nullptr});
            t1.push_back(one ? tall_entry(ws.Y, ws.ld, n, m, ws.Rinv, ws.dead, nullptr, ws.Q, ws.ld, sdp)
                             : tall_entry(ws.Y, ws.ld, n, m, ws.Rinv, ws.dead, nullptr, ws.T, ws.ld, nullptr));
            if (one) continue;
            g2.push_back(gram_entry(ws, ws.T, ws.T, n, m, ws.G, gdf, sms));
            c2.push_back(psd_g_chol{gdf, m, ws.Rinv, ws.dead, ws.ints + IN_QRANK});
            t2.push_back(tall_entry(ws.T, ws.ld, n, m, ws.Rinv, ws.dead, nullptr, ws.Q, ws.ld, sdp));
        }
        qr_off o;
        o.count = (int)c1.size();
        o.count2 = (int)c2.size();
        o.g1 = put_gram(tb, g1);
        o.g2 = put_gram(tb, g2);
        o.c1 = tb.put(c1);
        o.c2 = tb.put(c2);
        o.t1 = put_tall(tb, t1);
        o.t2 = put_tall(tb, t2);
        qo.push_back(o);
    }
    std::vector<psd_g_gram> cg;
    std::vector<psd_g_eig> ce;
    std::vector<psd_g_factor> cf;
    std::vector<psd_g_tall> ct;
    std::vector<int2> bns, bray;
    for (int i = 0; i < count; ++i) {
        const proj_call &pc = gp.pc[i];
        const psd_workspace &ws = gp.slot[i].ws;
        const int m = pc.m;
        float2 *cdf = reinterpret_cast<float2 *>(core_gdf(ws, m));
        cg.push_back(gram_entry(ws, ws.Q, ws.Y, pc.n, m, ws.C, cdf, sms));
        ce.push_back(psd_g_eig{ws.C, cdf, m, ws.V, ws.d, ws.eigscr, ws.ints + IN_EIGFAIL});
        cf.push_back(psd_g_factor{ws.V, ws.d, m, ws.M, ws.ints + IN_RANK, pc.rank_written ? pc.d_rank : nullptr});
        float *Wd = pc.dW ? pc.dW : ws.W;
        const int64_t ldwd = pc.dW ? pc.ldw : ws.ld;
        // the split-BF16 SYRK's operands written with W
        psd_bf16_side wsd{ws.Xhi, ws.ld, nullptr, 0, nullptr, ws.Xlo};
        ct.push_back(tall_entry(ws.Q, ws.ld, pc.n, m, ws.M, nullptr, ws.ints + IN_RANK, Wd, ldwd,
                                pc.w_split ? &wsd : nullptr));
        for (int b = 0; b < psd_eig_ns_blocks(m); ++b) bns.push_back(make_int2(i, b));
        for (int b = 0; b < psd_eig_ray_blocks(m); ++b) bray.push_back(make_int2(i, b));
    }
    const gram_off cgo = put_gram(tb, cg);
    const size_t ceo = tb.put(ce), cfo = tb.put(cf), bnso = tb.put(bns), brayo = tb.put(bray);
    const tall_off cto = put_tall(tb, ct);
    // the grouped power iterations: run 1 with A, run 2 with A - sigma_1 I
    // (Alg. 5), then alpha = |sigma_1 - sigma_2| and the shift
    std::vector<psd_g_pi> p1, p2;
    std::vector<psd_g_alpha> al;
    std::vector<int2> bpi;
    for (int i = 0; i < count; ++i) {
        if (!gp.galpha[i]) continue;
        const proj_call &pc = gp.pc[i];
        const grouped_slot &sl = gp.slot[i];
        const psd_workspace &ws = sl.ws;
        double *sc = ws.scal;
        psd_g_pi e;
        e.Ab = sl.Ab;
        e.n = pc.n;
        e.v0 = ws.pv0;
        e.v1 = ws.pv1;
        e.v2 = ws.pv2;
        e.scal = sc;
        e.shift_neg = nullptr;
        e.sigma = sc + SC_SIGMA1;
        e.seed = pc.seed;
        // one CTA per 16 tiles: a small product is dominated by each CTA's
        // fixed costs (its barriers, the norm of x), not by its tiles
        const int64_t tiles = psd_tile_count(pc.n);
        e.nb = (int)((tiles + 15) / 16);
        for (int b = 0; b < e.nb; ++b) bpi.push_back(make_int2((int)p1.size(), b));
        p1.push_back(e);
        e.shift_neg = sc + SC_SIGMA1;
        e.sigma = sc + SC_SIGMA2;
        p2.push_back(e);
        al.push_back(psd_g_alpha{sc + SC_SIGMA1, sc + SC_SIGMA2, pc.alpha_in,
                                 pc.d_alpha_out ? pc.d_alpha_out : sc + SC_ALPHA, sc + SC_SHIFT,
                                 pc.d_info ? pc.d_info : ws.ints + IN_INFO});
    }
    const size_t p1o = tb.put(p1), p2o = tb.put(p2), alo = tb.put(al), bpio = tb.put(bpi);
    // images: the blocks of each upper block triangle
    std::vector<psd_g_pack> pk, pkl;
    std::vector<int2> bpk;
    if (gp.gpack) {
        for (int i = 0; i < count; ++i) {
            const proj_call &pc = gp.pc[i];
            const int nbr = (int)((pc.n + PSD_TILE_M - 1) / PSD_TILE_M);
            psd_g_pack e;
            e.A = pc.dA;
            e.n = pc.n;
            e.lda = pc.lda;
            e.Ab = gp.slot[i].Ab;
            e.nbc = nbr * PSD_TILE_R;
            e.vec = (pc.lda % 4) == 0 && (reinterpret_cast<uintptr_t>(pc.dA) & 15) == 0;
            const int64_t nblocks = (int64_t)e.nbc * nbr * (PSD_TILE_M / 64);
            for (int64_t b = 0; b < nblocks; ++b) {
                const int J = (int)(b % e.nbc);
                const int I = (int)((b / e.nbc) * 64 / PSD_TILE_M);
                if (J >= PSD_TILE_R * I) bpk.push_back(make_int2((int)pk.size(), (int)b));
            }
            pk.push_back(e);
            e.Ab = gp.slot[i].Ab_lo;
            pkl.push_back(e);
        }
    }
    const size_t pko = tb.put(pk), pklo = tb.put(pkl), bpko = tb.put(bpk);
    // test matrices (with the BF16 pass's side outputs where the form fuses them)
    std::vector<psd_g_gauss> gs;
    std::vector<int2> bgs;
    for (int i = 0; i < count; ++i) {
        const proj_call &pc = gp.pc[i];
        if (!pc.omega_prepared) continue;
        const psd_workspace &ws = gp.slot[i].ws;
        psd_g_gauss e;
        e.seed = pc.seed;
        e.n = pc.n;
        e.m = pc.m;
        e.mpad = psd_lpad(pc.m);
        e.rows_pad = ws.ld;
        e.X = ws.Om;
        e.ldx = ws.ld;
        e.side = proj_fuse(pc) ? psd_bf16_side{ws.Xhi, ws.ld, ws.Y, ws.ld, proj_shift(pc, ws)}
                               : psd_bf16_side{nullptr, 0, nullptr, 0, nullptr};
        const int64_t vals = e.rows_pad * e.mpad;
        e.nb = (int)((vals + 2047) / 2048);      // eight values per thread
        for (int b = 0; b < e.nb; ++b) bgs.push_back(make_int2((int)gs.size(), b));
        gs.push_back(e);
    }
    const size_t gso = tb.put(gs), bgso = tb.put(bgs);
    const size_t bytes = align_up(tb.h.size(), 256);
    if (ctx->g_tabs_bytes[w] < bytes) {
        PSD_TRY(psd_budget_check(ctx, ctx->g_tabs_bytes[w], bytes));
        if (ctx->g_tabs[w]) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->g_tabs[w]);
            ctx->g_tabs[w] = nullptr;
            ctx->g_tabs_bytes[w] = 0;
        }
        PSD_CK(cudaMalloc(&ctx->g_tabs[w], bytes));
        ctx->g_tabs_bytes[w] = bytes;
    }
    // the previous plan's launches may still read the tables: upload in order
    PSD_CK(cudaStreamSynchronize(ctx->stream));
    PSD_CK(cudaMemcpy(ctx->g_tabs[w], tb.h.data(), tb.h.size(), cudaMemcpyHostToDevice));
    const char *d = static_cast<const char *>(ctx->g_tabs[w]);
    auto gram_at = [&](const gram_off &o) {
        gl_gram g;
        g.tab = reinterpret_cast<const psd_g_gram *>(d + o.tab);
        g.bm = reinterpret_cast<const int2 *>(d + o.bm);
        g.bm_red = reinterpret_cast<const int2 *>(d + o.bm_red);
        g.nb = o.nb;
        g.nb_red = o.nb_red;
        return g;
    };
    auto tall_at = [&](const tall_off &o) {
        gl_tall t;
        t.tab = reinterpret_cast<const psd_g_tall *>(d + o.tab);
        t.bm = reinterpret_cast<const int2 *>(d + o.bm);
        t.nb = o.nb;
        return t;
    };
    gp.qr.clear();
    for (const qr_off &o : qo) {
        gl_qr q;
        q.count = o.count;
        q.count2 = o.count2;
        q.g1 = gram_at(o.g1);
        q.g2 = gram_at(o.g2);
        q.c1 = reinterpret_cast<const psd_g_chol *>(d + o.c1);
        q.c2 = reinterpret_cast<const psd_g_chol *>(d + o.c2);
        q.t1 = tall_at(o.t1);
        q.t2 = tall_at(o.t2);
        gp.qr.push_back(q);
    }
    gp.core.count = count;
    gp.core.g = gram_at(cgo);
    gp.core.eig = reinterpret_cast<const psd_g_eig *>(d + ceo);
    gp.core.fac = reinterpret_cast<const psd_g_factor *>(d + cfo);
    gp.core.bm_ns = reinterpret_cast<const int2 *>(d + bnso);
    gp.core.bm_ray = reinterpret_cast<const int2 *>(d + brayo);
    gp.core.nb_ns = (int)bns.size();
    gp.core.nb_ray = (int)bray.size();
    gp.core.t = tall_at(cto);
    gp.pi1 = reinterpret_cast<const psd_g_pi *>(d + p1o);
    gp.pi2 = reinterpret_cast<const psd_g_pi *>(d + p2o);
    gp.al = reinterpret_cast<const psd_g_alpha *>(d + alo);
    gp.bm_pi = reinterpret_cast<const int2 *>(d + bpio);
    gp.nb_pi = (int)bpi.size();
    gp.pk = reinterpret_cast<const psd_g_pack *>(d + pko);
    gp.pk_lo = reinterpret_cast<const psd_g_pack *>(d + pklo);
    gp.bm_pk = reinterpret_cast<const int2 *>(d + bpko);
    gp.nb_pk = (int)bpk.size();
    gp.gs = reinterpret_cast<const psd_g_gauss *>(d + gso);
    gp.bm_gs = reinterpret_cast<const int2 *>(d + bgso);
    gp.nb_gs = (int)bgs.size();
    return PSDPROJ_OK;
}

// alpha of the grouped-alpha problems: the two power iterations (Alg. 4 in
// Alg. 5) of all of them as grouped launches, then alpha and the shift
int grouped_alpha_issue(psdproj_ctx *ctx, const grouped_plan &gp, const psdproj_opts &opts)
{
    cudaStream_t s = ctx->stream;
    const long long wl = (long long)opts.spin_limit;
    PSD_KL(launch_pi_start_grouped(s, gp.pi1, gp.bm_pi, gp.nb_pi, 3u), 1);
    PSD_KL(launch_power_iteration_grouped(s, gp.pi1, gp.n_galpha, gp.bm_pi, gp.nb_pi, gp.N, ctx->d_status, wl),
           gp.N + 2);
    PSD_KL(launch_pi_start_grouped(s, gp.pi2, gp.bm_pi, gp.nb_pi, 4u), 1);
    PSD_KL(launch_power_iteration_grouped(s, gp.pi2, gp.n_galpha, gp.bm_pi, gp.nb_pi, gp.N, ctx->d_status, wl),
           gp.N + 2);
    PSD_KL(launch_alpha_finish_grouped(s, gp.al, gp.n_galpha), 1);
    return PSDPROJ_OK;
}

// A lane running one problem's phase: the lane's workspace and image are
// those of the problem's slot until the binding ends
struct slot_binding {
    psdproj_ctx *c;
    psd_workspace ws;
    uint16_t *Ab, *Ab_lo;
    size_t Ab_bytes, Ab_lo_bytes;
    slot_binding(psdproj_ctx *lane, const grouped_slot &sl)
        : c(lane), ws(lane->ws), Ab(lane->Ab), Ab_lo(lane->Ab_lo), Ab_bytes(lane->Ab_bytes),
          Ab_lo_bytes(lane->Ab_lo_bytes)
    {
        lane->ws = sl.ws;
        lane->Ab = sl.Ab;
        lane->Ab_lo = sl.Ab_lo;
        lane->Ab_bytes = sl.Ab_bytes;
        lane->Ab_lo_bytes = sl.Ab_lo_bytes;
    }
    ~slot_binding()
    {
        c->ws = ws;
        c->Ab = Ab;
        c->Ab_lo = Ab_lo;
        c->Ab_bytes = Ab_bytes;
        c->Ab_lo_bytes = Ab_lo_bytes;
    }
};

int grouped_qr(psdproj_ctx *ctx, const grouped_plan &gp, const gl_qr &q)
{
    cudaStream_t s = ctx->stream;
    const double tau = 1e-10;     // the dependent-column threshold of cholqr2
    PSD_KL(launch_gram_grouped(s, q.g1.tab, 0, q.g1.bm, q.g1.nb, q.g1.bm_red, q.g1.nb_red, gp.mp_max), 2);
    PSD_KL(launch_cholesky_grouped(s, q.c1, q.count, gp.m_max, 1, tau, ctx->d_status), 1);
    PSD_KL(launch_tall_small_grouped(s, q.t1.tab, q.t1.bm, q.t1.nb, gp.m_max), 1);
    if (q.count2 == 0) return PSDPROJ_OK;
    PSD_KL(launch_gram_grouped(s, q.g2.tab, 0, q.g2.bm, q.g2.nb, q.g2.bm_red, q.g2.nb_red, gp.mp_max), 2);
    PSD_KL(launch_cholesky_grouped(s, q.c2, q.count2, gp.m_max, 0, tau, ctx->d_status), 1);
    PSD_KL(launch_tall_small_grouped(s, q.t2.tab, q.t2.bm, q.t2.nb, gp.m_max), 1);
    return PSDPROJ_OK;
}

int grouped_core(psdproj_ctx *ctx, const grouped_plan &gp, const psdproj_opts &opts)
{
    cudaStream_t s = ctx->stream;
    const gl_core &c = gp.core;
    PSD_KL(launch_gram_grouped(s, c.g.tab, 1, c.g.bm, c.g.nb, c.g.bm_red, c.g.nb_red, gp.mp_max), 2);
    PSD_KL(launch_eig_grouped(s, c.eig, c.count, c.bm_ns, c.nb_ns, c.bm_ray, c.nb_ray, gp.m_max, ctx->d_status,
                              opts.eig),
           psd_eig_launches(opts.eig));
    PSD_KL(launch_factor_prep_grouped(s, c.fac, c.count), 1);
    PSD_KL(launch_tall_small_grouped(s, c.t.tab, c.t.bm, c.t.nb, gp.m_max), 1);
    return PSDPROJ_OK;
}

// Issue a planned grouped batch on the context's stream
int grouped_issue(psdproj_ctx *ctx, grouped_plan &gp, const psdproj_opts &opts)
{
    const int S = gp.lanes.S;
    psdproj_ctx **ln = ctx->lane + gp.lane0;
    // the lanes run with this call's settings
    struct lane_settings {
        psdproj_ctx **ln;
        int S;
        ~lane_settings()
        {
            for (int j = 0; j < S; ++j) {
                ln[j]->wait_limit = 0;
                ln[j]->det = false;
            }
        }
    } settings_scope{ln, S};
    for (int j = 0; j < S; ++j) {
        ln[j]->wait_limit = (long long)opts.spin_limit;
        ln[j]->det = false;
    }
    // one phase of every problem with `take(i)` on the lanes, forked from and
    // joined back to the context's stream (also after an error)
    auto on_lanes = [&](auto take, auto phase) -> int {
        cudaEvent_t fork = ctx->lane_ev[PSD_MAX_LANES];
        PSD_CK(cudaEventRecord(fork, ctx->stream));
        for (int j = 0; j < S; ++j) PSD_CK(cudaStreamWaitEvent(ln[j]->stream, fork, 0));
        int rc = PSDPROJ_OK;
        for (int i : gp.lanes.order) {
            if (!take(i)) continue;
            psdproj_ctx *lane = ln[gp.lanes.lane_of[i]];
            slot_binding bind(lane, gp.slot[i]);
            rc = phase(lane, gp.pc[i], i);
            if (rc != PSDPROJ_OK) break;
        }
        for (int j = 0; j < S; ++j) {
            cudaEventRecord(ctx->lane_ev[gp.lane0 + j], ln[j]->stream);
            cudaStreamWaitEvent(ctx->stream, ctx->lane_ev[gp.lane0 + j], 0);
        }
        return rc;
    };
    auto all = [](int) { return true; };
    // the images (grouped in the BF16 forms), alpha (grouped power
    // iterations where they apply, else per problem), the test matrices
    // (grouped for the Gaussian sketch), then the first products
    if (gp.gpack) {
        PSD_KL(launch_pack_grouped(ctx->stream, gp.pk, gp.bm_pk, gp.nb_pk, 0), 1);
        if (gp.gpack_lo) PSD_KL(launch_pack_grouped(ctx->stream, gp.pk_lo, gp.bm_pk, gp.nb_pk, 1), 1);
    }
    auto lane_first = [&](int i) {
        const proj_call &pc = gp.pc[i];
        return (!gp.gpack && pc.opts.prec != PSDPROJ_PREC_FP32) ||
               (!gp.galpha[i] && pc.scaled && !proj_ritz(pc));
    };
    bool any_first = false;
    for (int i = 0; i < (int)gp.pc.size(); ++i) any_first = any_first || lane_first(i);
    if (any_first)
        PSD_TRY(on_lanes(lane_first, [&](psdproj_ctx *c, proj_call &pc, int i) {
            if (!gp.gpack) PSD_TRY(proj_pack(c, pc));
            return gp.galpha[i] ? PSDPROJ_OK : proj_alpha(c, pc);
        }));
    if (gp.n_galpha > 0) PSD_TRY(grouped_alpha_issue(ctx, gp, opts));
    if (gp.nb_gs > 0) PSD_KL(launch_gaussian_grouped(ctx->stream, gp.gs, gp.bm_gs, gp.nb_gs, 0u), 1);
    PSD_TRY(on_lanes(all, [](psdproj_ctx *c, proj_call &pc, int) { return proj_sketch(c, pc); }));
    PSD_TRY(grouped_qr(ctx, gp, gp.qr[0]));
    for (int t = 0; t < 2 * gp.qmax; ++t) {
        PSD_TRY(on_lanes([&](int i) { return t < 2 * gp.pc[i].q; },
                         [](psdproj_ctx *c, proj_call &pc, int) { return proj_power_pass(c, pc); }));
        PSD_TRY(grouped_qr(ctx, gp, gp.qr[t + 1]));
    }
    PSD_TRY(on_lanes(all, [](psdproj_ctx *c, proj_call &pc, int) { return proj_core_pass(c, pc); }));
    PSD_TRY(grouped_core(ctx, gp, opts));
    return on_lanes(all, [](psdproj_ctx *c, proj_call &pc, int) { return proj_finish(c, pc); });
}

// The plan of (part of) a grouped batch: its problems, lanes lane0 ..
// lane0 + lanes - 1, slots and tables in ctx->g_slots[w] / g_tabs[w]
int grouped_make(psdproj_ctx *ctx, const psdproj_opts &opts, int count, const psdproj_problem *probs, int lanes,
                 int lane0, int w, grouped_plan &gp)
{
    gp.lanes = batch_make_plan(ctx, opts, count, probs, lanes);
    if (gp.lanes.S < 1) gp.lanes.S = 1;
    gp.lane0 = lane0;
    for (int j = 0; j < gp.lanes.S; ++j) PSD_TRY(ensure_lane(ctx, lane0 + j));
    gp.pc.resize(count);
    for (int i = 0; i < count; ++i) {
        const psdproj_problem &pb = probs[i];
        proj_call &pc = gp.pc[i];
        pc.dA = pb.dA;
        pc.n = pb.n;
        pc.lda = pb.lda;
        pc.k = pb.k;
        pc.p = pb.p;
        pc.q = pb.q;
        pc.m = pb.k + pb.p;
        pc.seed = pb.seed;
        pc.scaled = pb.algorithm == 2;
        pc.alpha_in = pb.alpha_in;
        pc.d_alpha_out = pb.d_alpha_out;
        pc.d_info = pb.d_info;
        pc.dP = pb.dP;
        pc.ldp = pb.ldp;
        pc.dW = pb.dW;
        pc.ldw = pb.ldw;
        pc.d_rank = pb.d_rank;
        pc.opts = opts;
        if (pb.q > gp.qmax) gp.qmax = pb.q;
        if (pc.m > gp.m_max) gp.m_max = pc.m;
    }
    gp.mp_max = (int)psd_round_up(gp.m_max, 8);
    gp.N = opts.N;
    gp.galpha.assign(count, 0);
    for (int i = 0; i < count; ++i)
        if (grouped_alpha(gp.pc[i])) {
            gp.galpha[i] = 1;
            ++gp.n_galpha;
        }
    gp.gpack = opts.prec == PSDPROJ_PREC_BF16 || opts.prec == PSDPROJ_PREC_BF16X3;
    gp.gpack_lo = opts.prec == PSDPROJ_PREC_BF16X3;
    for (int i = 0; i < count; ++i) {
        proj_call &pc = gp.pc[i];
        pc.omega_prepared = opts.sketch == PSDPROJ_SKETCH_GAUSS;
        // the tensor-core SYRK (m <= 128 here) reads the split W
        pc.w_split = opts.out_mode != PSDPROJ_OUT_FACTOR && opts.syrk_prec == PSDPROJ_PREC_BF16X3;
        pc.rank_written = pc.d_rank != nullptr;
    }
    PSD_TRY(grouped_slots(ctx, w, opts, count, probs, gp.slot));
    return grouped_tables(ctx, w, gp);
}

void grouped_graph_free(psdproj_ctx *ctx)
{
    if (ctx->g_exec) cudaGraphExecDestroy(ctx->g_exec);
    ctx->g_exec = nullptr;
    ctx->g_probs.clear();
    ctx->g_launches = 0;
}

}  // namespace

extern "C" {

int psdproj_batched(psdproj_ctx *ctx, int count, const psdproj_problem *probs,
                    const psdproj_opts *opts_in)
{
    if (!ctx || count < 0 || (count > 0 && !probs)) return PSDPROJ_EINVAL;
    psdproj_opts opts;
    if (opts_in) opts = *opts_in; else psdproj_default_opts(&opts);
    PSD_TRY(check_opts(&opts));
    int64_t nmax = 0;
    int mmax = 0;
    PSD_TRY(batch_validate(opts, count, probs, nmax, mmax));
    if (count == 0) return PSDPROJ_OK;
    device_guard g(ctx->device);
    const batch_plan pl = batch_make_plan(ctx, opts, count, probs, batch_lanes(ctx, count, probs));
    if (pl.S <= 1) {
        // one workspace for the whole batch, problems one after another
        PSD_TRY(psd_ensure_workspace(ctx, nmax, mmax));
    } else {
        for (int j = 0; j < pl.S; ++j) PSD_TRY(ensure_lane(ctx, j));
    }
    return batch_issue(ctx, pl, opts, count, probs);
}

int psdproj_batched_graph(psdproj_ctx *ctx, int count, const psdproj_problem *probs,
                          const psdproj_opts *opts_in)
{
    if (!ctx || count < 0 || (count > 0 && !probs)) return PSDPROJ_EINVAL;
    psdproj_opts opts;
    if (opts_in) opts = *opts_in; else psdproj_default_opts(&opts);
    PSD_TRY(check_opts(&opts));
    int64_t nmax = 0;
    int mmax = 0;
    PSD_TRY(batch_validate(opts, count, probs, nmax, mmax));
    if (count == 0) return PSDPROJ_OK;
    device_guard g(ctx->device);
    // the same table, options and lane settings as the recorded graph: replay
    const int lanes = batch_lanes(ctx, count, probs);
    const bool same = ctx->graph_exec && (int)ctx->graph_probs.size() == count &&
                      memcmp(ctx->graph_probs.data(), probs, sizeof(psdproj_problem) * (size_t)count) == 0 &&
                      memcmp(&ctx->graph_opts, &opts, sizeof(opts)) == 0 &&
                      ctx->graph_streams == lanes && ctx->graph_persist == ctx->persist_sms;
    if (!same) {
        batch_graph_free(ctx);
        const batch_plan pl = batch_make_plan(ctx, opts, count, probs, lanes);
        if (pl.S > 1)
            for (int j = 0; j < pl.S; ++j) PSD_TRY(ensure_lane(ctx, j));
        PSD_TRY(batch_presize(ctx, pl, opts, count, probs));
        // record with the stage timers off (events inside a graph are not read back)
        int timing_was = ctx->timing.on;
        ctx->timing.on = 0;
        int lane_timing[PSD_MAX_LANES] = {};
        for (int j = 0; j < PSD_MAX_LANES; ++j)
            if (ctx->lane[j]) {
                lane_timing[j] = ctx->lane[j]->timing.on;
                ctx->lane[j]->timing.on = 0;
            }
        // record on a stream of the context's own (the caller's stream may be
        // the legacy default stream, which cannot be captured); the graph is
        // then launched into the caller's stream
        if (!ctx->capture_stream)
            PSD_CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaStream_t user = ctx->stream;
        const uint64_t l0 = g_launches.load();
        PSD_CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed));
        ctx->stream = ctx->capture_stream;
        const int rc = batch_issue(ctx, pl, opts, count, probs);
        ctx->stream = user;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->capture_stream, &graph);
        const uint64_t nk = g_launches.load() - l0;
        ctx->timing.on = timing_was;
        for (int j = 0; j < PSD_MAX_LANES; ++j)
            if (ctx->lane[j]) ctx->lane[j]->timing.on = lane_timing[j];
        if (rc != PSDPROJ_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            g_launches.fetch_sub(nk);
            return rc != PSDPROJ_OK ? rc : cuda_status(ec, __LINE__);
        }
        g_launches.fetch_sub(nk);      // recorded, not launched: counted on each replay
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return cuda_status(ei, __LINE__);
        ctx->graph_exec = exec;
        ctx->graph_probs.assign(probs, probs + count);
        ctx->graph_opts = opts;
        ctx->graph_streams = lanes;
        ctx->graph_persist = ctx->persist_sms;
        ctx->graph_launches = nk;
    }
    PSD_CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    g_launches.fetch_add(ctx->graph_launches);
    return PSDPROJ_OK;
}

int psdproj_batched_grouped(psdproj_ctx *ctx, int count, const psdproj_problem *probs,
                            const psdproj_opts *opts_in)
{
    if (!ctx || count < 0 || (count > 0 && !probs)) return PSDPROJ_EINVAL;
    psdproj_opts opts;
    if (opts_in) opts = *opts_in; else psdproj_default_opts(&opts);
    PSD_TRY(check_opts(&opts));
    int64_t nmax = 0;
    int mmax = 0;
    PSD_TRY(batch_validate(opts, count, probs, nmax, mmax));
    // the grouped small steps are the shared-memory kernels (m <= 128); the
    // fixed-order products of the deterministic form are not grouped
    if (mmax > 128 || opts.deterministic) return PSDPROJ_ENOTSUP;
    if (count == 0) return PSDPROJ_OK;
    device_guard g(ctx->device);
    const int lanes = batch_lanes(ctx, count, probs);
    const bool same = ctx->g_exec && (int)ctx->g_probs.size() == count &&
                      memcmp(ctx->g_probs.data(), probs, sizeof(psdproj_problem) * (size_t)count) == 0 &&
                      memcmp(&ctx->g_opts, &opts, sizeof(opts)) == 0 && ctx->g_streams == lanes &&
                      ctx->g_persist == ctx->persist_sms;
    if (!same) {
        grouped_graph_free(ctx);
        // a batch of 32 problems or more runs as two halves, each with half
        // of the lanes and its own chain of grouped launches on a stream of
        // its own (two branches of the graph): the latency-bound grouped
        // steps of one half overlap the per-problem products of the other
        const char *env = getenv("PSDPROJ_GROUPED_SPLIT");
        const int G = (env && atoi(env) == 1) || count < 32 || lanes < 2 ? 1 : 2;
        std::vector<psdproj_problem> half[2];
        {
            // alternate in decreasing cost, so that the halves weigh alike
            const batch_plan byc = batch_make_plan(ctx, opts, count, probs, 1);
            int r = 0;
            for (int i : byc.order) half[r++ % G].push_back(probs[i]);
        }
        std::vector<grouped_plan> gps(G);
        for (int w = 0; w < G; ++w)
            PSD_TRY(grouped_make(ctx, opts, (int)half[w].size(), half[w].data(), lanes / G, w * (lanes / G), w,
                                 gps[w]));
        if (G == 2) {
            if (!ctx->g_stream2) PSD_CK(cudaStreamCreateWithFlags(&ctx->g_stream2, cudaStreamNonBlocking));
            for (int w = 0; w < 2; ++w)
                if (!ctx->g_ev[w]) PSD_CK(cudaEventCreateWithFlags(&ctx->g_ev[w], cudaEventDisableTiming));
        }
        // record with the stage timers off (events inside a graph are not read back)
        int timing_was = ctx->timing.on;
        ctx->timing.on = 0;
        int lane_timing[PSD_MAX_LANES] = {};
        for (int j = 0; j < PSD_MAX_LANES; ++j)
            if (ctx->lane[j]) {
                lane_timing[j] = ctx->lane[j]->timing.on;
                ctx->lane[j]->timing.on = 0;
            }
        if (!ctx->capture_stream)
            PSD_CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        // the slots' zeroing (on the context's stream) ends before the recorded work
        PSD_CK(cudaStreamSynchronize(ctx->stream));
        cudaStream_t user = ctx->stream;
        const uint64_t l0 = g_launches.load();
        PSD_CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed));
        ctx->stream = ctx->capture_stream;
        int rc = PSDPROJ_OK;
        if (G == 1) {
            rc = grouped_issue(ctx, gps[0], opts);
        } else {
            cudaStream_t s0 = ctx->stream;
            cudaError_t ef = cudaEventRecord(ctx->g_ev[0], s0);
            if (ef == cudaSuccess) ef = cudaStreamWaitEvent(ctx->g_stream2, ctx->g_ev[0], 0);
            rc = ef != cudaSuccess ? cuda_status(ef, __LINE__) : grouped_issue(ctx, gps[0], opts);
            if (rc == PSDPROJ_OK) {
                ctx->stream = ctx->g_stream2;
                rc = grouped_issue(ctx, gps[1], opts);
                ctx->stream = s0;
            }
            // joined back also after an error, so that the capture ends
            cudaEventRecord(ctx->g_ev[1], ctx->g_stream2);
            cudaStreamWaitEvent(s0, ctx->g_ev[1], 0);
        }
        ctx->stream = user;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->capture_stream, &graph);
        const uint64_t nk = g_launches.load() - l0;
        g_launches.fetch_sub(nk);      // recorded, not launched: counted on each replay
        ctx->timing.on = timing_was;
        for (int j = 0; j < PSD_MAX_LANES; ++j)
            if (ctx->lane[j]) ctx->lane[j]->timing.on = lane_timing[j];
        if (rc != PSDPROJ_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != PSDPROJ_OK ? rc : cuda_status(ec, __LINE__);
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return cuda_status(ei, __LINE__);
        ctx->g_exec = exec;
        ctx->g_probs.assign(probs, probs + count);
        ctx->g_opts = opts;
        ctx->g_streams = lanes;
        ctx->g_persist = ctx->persist_sms;
        ctx->g_launches = nk;
    }
    PSD_CK(cudaGraphLaunch(ctx->g_exec, ctx->stream));
    g_launches.fetch_add(ctx->g_launches);
    return PSDPROJ_OK;
}

int psdproj_tune_batch(psdproj_ctx *ctx, int count, const psdproj_problem *probs, const psdproj_opts *opts,
                       int reps, int *best_streams, double *best_ms)
{
    if (!ctx || count < 1 || !probs || reps < 1) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    static const int trial[] = {2, 4, 8, 16, 32, 64};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PSD_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PSDPROJ_ECUDA;
    }
    int best = 0, rc = PSDPROJ_OK;
    float best_t = 0.0f;
    for (int S : trial) {
        if (S > PSD_MAX_LANES) continue;
        ctx->tune_force = S;
        rc = psdproj_batched_graph(ctx, count, probs, opts);          // records the graph, one warm-up run
        if (rc == PSDPROJ_OK && cudaEventRecord(e0, ctx->stream) != cudaSuccess) rc = PSDPROJ_ECUDA;
        for (int r = 0; r < reps && rc == PSDPROJ_OK; ++r) rc = psdproj_batched_graph(ctx, count, probs, opts);
        if (rc == PSDPROJ_OK && cudaEventRecord(e1, ctx->stream) != cudaSuccess) rc = PSDPROJ_ECUDA;
        if (rc == PSDPROJ_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = PSDPROJ_ECUDA;
        if (rc == PSDPROJ_OK) rc = psdproj_sync_status(ctx);
        if (rc != PSDPROJ_OK) break;
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        t /= (float)reps;
        if (best == 0 || t < best_t) {
            best = S;
            best_t = t;
        }
    }
    ctx->tune_force = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PSDPROJ_OK) return rc;
    ctx->batch_streams = best;
    ctx->lanes_explicit = true;
    const dev_ident d = device_ident(ctx->device);
    PSD_TRY(psdproj_tune_store(d.name, d.sms, median_side(count, probs), count, best));
    if (best_streams) *best_streams = best;
    if (best_ms) *best_ms = (double)best_t;
    return PSDPROJ_OK;
}

int psdproj_sdls_dual_gd(psdproj_ctx *ctx, const psdproj_sdls *pr, double *y, float *dX, int64_t ldx,
                         int *iters_out, double *gnorm_out, double *ghist, const psdproj_opts *opts_in)
{
    if (!ctx || !pr || !y || !pr->dC || !pr->dA || !pr->b || pr->mc < 1 || pr->mc > 4096) return PSDPROJ_EINVAL;
    if (!(pr->rho > 0.0) || !(pr->beta > 0.0) || !(pr->eps >= 0.0) || pr->max_iter < 1) return PSDPROJ_EINVAL;
    if (pr->algorithm != 1 && pr->algorithm != 2) return PSDPROJ_EINVAL;
    if (pr->n > 65535) return PSDPROJ_ETOOLARGE;
    for (int i = 0; i < pr->mc; ++i)
        if (!pr->dA[i]) return PSDPROJ_EINVAL;
    if (dX && ldx < pr->n) return PSDPROJ_EINVAL;
    psdproj_opts opts;
    if (opts_in) opts = *opts_in; else psdproj_default_opts(&opts);
    PSD_TRY(check_opts(&opts));
    PSD_TRY(validate(pr->n, pr->ld, pr->k, pr->p, pr->q, pr->dC));
    const int64_t n = pr->n;
    const int m = pr->k + pr->p, mc = pr->mc;
    device_guard g(ctx->device);
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    psd_workspace &ws = ctx->ws;
    cudaStream_t s = ctx->stream;
    // X = C / rho + sum y_i A_i lives in the host-API staging buffer (n x n)
    const int64_t ldX = (n + 3) / 4 * 4;
    PSD_TRY(ensure_stage(ctx, &ctx->dA_stage, &ctx->dA_stage_bytes, sizeof(float) * (size_t)n * ldX, s));
    // device scratch: y (mc doubles), g (mc doubles), the mc pointers to A_i
    const size_t scratch = sizeof(double) * 2 * mc + sizeof(float *) * mc;
    PSD_TRY(ensure_stage(ctx, &ctx->dP_stage, &ctx->dP_stage_bytes, scratch + 256, s));
    double *d_y = reinterpret_cast<double *>(ctx->dP_stage);
    double *d_g = d_y + mc;
    const float **d_A = reinterpret_cast<const float **>(d_g + mc);
    std::vector<double> neg_b(mc), gh(mc);
    for (int i = 0; i < mc; ++i) neg_b[i] = -pr->b[i];
    PSD_CK(cudaMemcpyAsync(d_A, pr->dA, sizeof(float *) * mc, cudaMemcpyHostToDevice, s));
    psdproj_opts po = opts;
    po.out_mode = PSDPROJ_OUT_FACTOR;
    double gn = 0.0;
    int t = 0;
    for (; t < pr->max_iter; ++t) {
        PSD_CK(cudaMemcpyAsync(d_y, y, sizeof(double) * mc, cudaMemcpyHostToDevice, s));
        PSD_CK(cudaMemcpyAsync(d_g, neg_b.data(), sizeof(double) * mc, cudaMemcpyHostToDevice, s));
        PSD_KL(launch_sdls_combine(s, pr->dC, d_A, mc, d_y, pr->rho, n, pr->ld, ctx->dA_stage, ldX), 1);
        const uint64_t seed_t = pr->seed + (uint64_t)t;
        bool warm = false;
        if (pr->warm_start && t > 0) {
            // the previous iterate's basis, with fresh Gaussian columns where
            // the orthonormalisation dropped one
            PSD_KL(launch_gaussian(s, seed_t, 0u, n, m, psd_lpad(m), ws.ld, ws.Om, ws.ld), 1);
            PSD_KL(launch_sdls_warm_omega(s, ws.Om, ws.Q, ws.dead, n, m, ws.ld), 1);
            warm = true;
        }
        PSD_TRY(run_projection(ctx, ctx->dA_stage, n, ldX, pr->k, pr->p, pr->q, seed_t, pr->algorithm == 2, 0.0,
                               nullptr, nullptr, nullptr, 0, nullptr, 0, nullptr, &po, warm));
        // grad_i = <A_i, W W^T> - b_i = sum_c w_c^T (A_i w_c) - b_i
        for (int i = 0; i < mc; ++i) {
            PSD_TRY(sym_pass(ctx, pr->dA[i], n, pr->ld, ws.W, ws.ld, m, nullptr, ws.Y, ws.ld, PSDPROJ_PREC_FP32));
            PSD_KL(launch_sdls_dot(s, ws.W, ws.Y, n, m, ws.ld, d_g + i), 1);
        }
        PSD_CK(cudaMemcpyAsync(gh.data(), d_g, sizeof(double) * mc, cudaMemcpyDeviceToHost, s));
        PSD_CK(cudaStreamSynchronize(s));
        int st = 0;
        PSD_CK(cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st) {
            cudaMemset(ctx->d_status, 0, sizeof(int));
            return st;
        }
        gn = 0.0;
        for (int i = 0; i < mc; ++i) gn += gh[i] * gh[i];
        gn = sqrt(gn);
        if (ghist) ghist[t] = gn;
        for (int i = 0; i < mc; ++i) y[i] -= pr->beta * gh[i];
        if (gn <= pr->eps) {
            ++t;
            break;
        }
    }
    if (iters_out) *iters_out = t;
    if (gnorm_out) *gnorm_out = gn;
    if (dX) {
        // the last iterate's projection: X_hat = W W^T
        stage_scope st(ctx, PSDPROJ_STAGE_SYRK);
        if (opts.syrk_prec == PSDPROJ_PREC_FP32 || m > 128)
            PSD_KL(launch_syrk_simt(s, ws.W, ws.ld, n, m, ws.ints + IN_RANK, dX, ldx, 0), 1);
        else
            PSD_KL(launch_syrk_tc(s, ctx->persist_sms, ws.W, ws.ld, n, m, ws.ints + IN_RANK, dX, ldx, 0, ws.Xhi,
                                  ws.Xlo, ws.ld, ctx->d_status), 2);
    }
    return PSDPROJ_OK;
}

int psdproj_alg1_host(psdproj_ctx *ctx, const float *hA, int64_t n, int64_t lda, int k, int p,
                      int q, uint64_t seed, float *hP, int64_t ldp, float *hW, int64_t ldw,
                      int *h_rank, const psdproj_opts *opts)
{
    return run_host(ctx, hA, n, lda, k, p, q, seed, false, 0.0, nullptr, hP, ldp, hW, ldw, h_rank,
                    opts);
}

int psdproj_alg2_host(psdproj_ctx *ctx, const float *hA, int64_t n, int64_t lda, int k, int p,
                      int q, uint64_t seed, double alpha_in, double *h_alpha_out, float *hP,
                      int64_t ldp, float *hW, int64_t ldw, int *h_rank, const psdproj_opts *opts)
{
    return run_host(ctx, hA, n, lda, k, p, q, seed, true, alpha_in, h_alpha_out, hP, ldp, hW, ldw,
                    h_rank, opts);
}

int psdproj_gaussian(psdproj_ctx *ctx, uint64_t seed, uint32_t stream, int64_t n, int m,
                     float *dX, int64_t ldx)
{
    if (!ctx || !dX || n < 1 || m < 1 || ldx < n) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_KL(launch_gaussian(ctx->stream, seed, stream, n, m, m, n, dX, ldx), 1);
    return PSDPROJ_OK;
}

int psdproj_srht(psdproj_ctx *ctx, uint64_t seed, int64_t n, int m, float *dX, int64_t ldx)
{
    if (!ctx || !dX || n < 1 || m < 1 || m > PSD_MAX_M || m > n || ldx < n) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    PSD_KL(launch_srht(ctx->stream, seed, n, m, m, n, ctx->ws.picks, ctx->d_status, dX, ldx), 2);
    return PSDPROJ_OK;
}

int psdproj_sym_pass(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda, const float *dX,
                     int64_t ldx, int m, const double *d_shift, float *dY, int64_t ldy, int prec)
{
    if (!ctx || !dA || !dX || !dY || n < 1 || m < 1 || lda < n || ldx < n || ldy < n)
        return PSDPROJ_EINVAL;
    if (prec < PSDPROJ_PREC_FP32 || prec > PSDPROJ_PREC_BF16X3) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    if (prec == PSDPROJ_PREC_FP32) return sym_pass(ctx, dA, n, lda, dX, ldx, m, d_shift, dY, ldy, prec);
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    PSD_TRY(pack_image(ctx, dA, n, lda, prec));
    return sym_pass(ctx, dA, n, lda, dX, ldx, m, d_shift, dY, ldy, prec);
}

int psdproj_cholqr2(psdproj_ctx *ctx, const float *dY, int64_t n, int64_t ldy, int m, float *dQ,
                    int64_t ldq, int *d_qrank)
{
    if (!ctx || !dY || !dQ || n < 1 || m < 1 || m > PSD_MAX_M || ldy < n || ldq < n)
        return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    return cholqr2(ctx, dY, ldy, n, m, dQ, ldq, d_qrank);
}

int psdproj_core(psdproj_ctx *ctx, const float *dX, int64_t ldx, const float *dZ, int64_t ldz,
                 int64_t n, int m, double *dC)
{
    if (!ctx || !dX || !dZ || !dC || n < 1 || m < 1 || m > PSD_MAX_M || ldx < n || ldz < n)
        return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    stage_scope st(ctx, PSDPROJ_STAGE_CORE);
    PSD_KL(launch_gram(ctx->stream, dX, ldx, dZ, ldz, n, m, ctx->ws.gpart, dC, 2, nullptr, ctx->persist_sms), 2);
    return PSDPROJ_OK;
}

int psdproj_eig_method(psdproj_ctx *ctx, const double *dC, int m, float *dV, double *dd,
                       int method)
{
    if (!ctx || !dC || !dV || !dd || m < 1 || m > PSD_MAX_M) return PSDPROJ_EINVAL;
    if (method < PSDPROJ_EIG_AUTO || method > PSDPROJ_EIG_TRIDIAG) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_TRY(psd_ensure_workspace(ctx, 1, m));
    stage_scope st(ctx, PSDPROJ_STAGE_EIG);
    PSD_KL(launch_eig(ctx->stream, dC, m, dV, dd, ctx->ws.eigscr, ctx->d_status, method,
                      ctx->ws.ints + IN_EIGFAIL), psd_eig_launches(method));
    return PSDPROJ_OK;
}

int psdproj_eig(psdproj_ctx *ctx, const double *dC, int m, float *dV, double *dd)
{
    return psdproj_eig_method(ctx, dC, m, dV, dd, PSDPROJ_EIG_AUTO);
}

int psdproj_factor(psdproj_ctx *ctx, const float *dQ, int64_t ldq, int64_t n, int m,
                   const float *dV, const double *dd, float *dW, int64_t ldw, int *d_rank)
{
    if (!ctx || !dQ || !dV || !dd || !dW || n < 1 || m < 1 || m > PSD_MAX_M || ldq < n || ldw < n)
        return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    psd_workspace &ws = ctx->ws;
    int *rk = ws.ints + IN_RANK;
    stage_scope st(ctx, PSDPROJ_STAGE_FACTOR);
    PSD_KL(launch_factor_prep(ctx->stream, dV, dd, m, ws.M, rk), 1);
    PSD_KL(launch_tall_small(ctx->stream, dQ, ldq, n, m, ws.M, m, nullptr, rk, dW, ldw, nullptr, ctx->persist_sms), 1);
    if (d_rank)
        PSD_CK(cudaMemcpyAsync(d_rank, rk, sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
    return PSDPROJ_OK;
}

int psdproj_syrk(psdproj_ctx *ctx, const float *dW, int64_t ldw, int64_t n, int m,
                 const int *d_rank, float *dP, int64_t ldp, int out_mode, int prec)
{
    if (!ctx || !dW || !dP || n < 1 || m < 1 || ldw < n || ldp < n) return PSDPROJ_EINVAL;
    if (out_mode != PSDPROJ_OUT_FULL && out_mode != PSDPROJ_OUT_UPPER) return PSDPROJ_EINVAL;
    if (prec != PSDPROJ_PREC_FP32 && prec != PSDPROJ_PREC_BF16X3) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    const int upper = out_mode == PSDPROJ_OUT_UPPER;
    if (prec == PSDPROJ_PREC_FP32) {
        stage_scope st(ctx, PSDPROJ_STAGE_SYRK);
        PSD_KL(launch_syrk_simt(ctx->stream, dW, ldw, n, m, d_rank, dP, ldp, upper), 1);
        return PSDPROJ_OK;
    }
    if (m > PSD_MAX_M) return PSDPROJ_ENOTSUP;
    PSD_TRY(psd_ensure_workspace(ctx, n, m));
    stage_scope st(ctx, PSDPROJ_STAGE_SYRK);
    PSD_KL(launch_syrk_tc(ctx->stream, ctx->persist_sms, dW, ldw, n, m, d_rank, dP, ldp, upper,
                          ctx->ws.Xhi, ctx->ws.Xlo, ctx->ws.ld, ctx->d_status), 2);
    return PSDPROJ_OK;
}

int psdproj_min_eig(psdproj_ctx *ctx, const float *dA, int64_t n, int64_t lda, int N,
                    uint64_t seed, double *d_alpha, double *d_sigma1, double *d_sigma2)
{
    if (!ctx || !dA || !d_alpha || n < 1 || lda < n || N < 0) return PSDPROJ_EINVAL;
    device_guard g(ctx->device);
    PSD_TRY(psd_ensure_workspace(ctx, n, 1));
    psd_workspace &ws = ctx->ws;
    cudaStream_t s = ctx->stream;
    double *sc = ws.scal;
    stage_scope st(ctx, PSDPROJ_STAGE_GEMV);
    PSD_KL(launch_power_iteration(s, dA, n, lda, N, seed, 3u, nullptr, ws.pv0, ws.pv1, sc,
                                  sc + SC_SIGMA1), 2 * N + 4);
    PSD_KL(launch_power_iteration(s, dA, n, lda, N, seed, 4u, sc + SC_SIGMA1, ws.pv0, ws.pv1, sc,
                                  sc + SC_SIGMA2), 2 * N + 4);
    PSD_KL(launch_alpha_finish(s, sc + SC_SIGMA1, sc + SC_SIGMA2, 0.0, d_alpha, sc + SC_SHIFT,
                               ws.ints + IN_INFO), 1);
    if (d_sigma1)
        PSD_CK(cudaMemcpyAsync(d_sigma1, sc + SC_SIGMA1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (d_sigma2)
        PSD_CK(cudaMemcpyAsync(d_sigma2, sc + SC_SIGMA2, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return PSDPROJ_OK;
}

}  // extern "C"
