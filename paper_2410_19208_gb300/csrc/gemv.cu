// power_iteration (Alg. 4) and min_eig (Alg. 5) on the device.
//
// One launch per product w = (A + shift I) (s * v): A is streamed once, upper
// triangle only, in 32 x 128 tiles.  A thread block owns a segment of one
// block row: the row sums accumulate in registers, the transposed
// contributions of each tile are summed over the block's 8 warps and added
// with atomics.  The last block to finish (atomic ticket) forms ||w|| in
// FP64, stores the scale 1/||w|| that the next product applies on load,
// clears the other vector for the next product, and resets the ticket.
// sigma = ||A v|| after the N normalised steps is written to *d_sigma.
#include "ctx.h"

namespace {

constexpr int TRW = 32;    // rows per tile
constexpr int TCW = 128;   // columns per tile
constexpr int SEGW = 8;    // tiles per block
constexpr int NTW = 256;

// scal[0]: scale of the input vector; scal[1]: norm of the last output.
// A block owns a segment of SEGW tiles (32 rows x 128 columns each) of one
// block row.  Warp w holds rows 4w..4w+3, lane l columns 4l..4l+3 of every
// tile; the loads of the whole segment are independent, and the column
// partial sums stay in registers until the segment ends (one barrier).
__global__ void __launch_bounds__(NTW)
sym_gemv_kernel(const float *__restrict__ A, int64_t n, int64_t lda,
                const float *__restrict__ x, float *__restrict__ y, float *__restrict__ other,
                double *scal, unsigned *counter, const double *d_shift_neg, double *d_sigma,
                unsigned nactive, int vec)
{
    __shared__ float colsum[8][SEGW * TCW];
    __shared__ double red[NTW / 32];
    __shared__ bool s_last;
    // grid: x = segment within the block row, y = block row; segments past
    // the end of a row exit at once (and take no completion ticket)
    const int I = blockIdx.y;
    const int64_t row0 = (int64_t)I * TRW;
    const int tiles = (int)((n - row0 + TCW - 1) / TCW);
    const int t0 = (int)blockIdx.x * SEGW;
    if (t0 >= tiles) return;
    const float sc = (float)scal[0];
    const float shift = d_shift_neg ? (float)(-(*d_shift_neg)) : 0.0f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    float rowacc[4] = {0.f, 0.f, 0.f, 0.f};
    float xr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = row0 + warp * 4 + i;
        xr[i] = gr < n ? x[gr] * sc : 0.0f;
    }
    // Interior tiles (strictly above the diagonal block, not past column n)
    // take an unmasked path: per row one float4 load, 4 FMAs into the row sum
    // and 4 into the column partials.  The diagonal tile, the ragged last
    // tile and unaligned rows take the masked path.
    const float *rowp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = row0 + warp * 4 + i;
        rowp[i] = A + (gr < n ? gr : 0) * lda;
    }
    auto is_interior = [&](int tt) {
        const int64_t cb = row0 + (int64_t)tt * TCW;
        return vec && tt > 0 && tt < tiles && cb + TCW <= n && row0 + 32 <= n;
    };
    // software pipeline: the loads of tile t+1 are issued before tile t is used
    float4 nxt[4];
    bool nxt_int = is_interior(t0);
    if (nxt_int) {
        const int64_t c0 = row0 + (int64_t)t0 * TCW + lane * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) nxt[i] = __ldcs(reinterpret_cast<const float4 *>(rowp[i] + c0));
    }
#pragma unroll 1
    for (int t = 0; t < SEGW; ++t) {
        const int tt = t0 + t;
        const int64_t c0 = row0 + (int64_t)tt * TCW + lane * 4;
        float colacc[4] = {0.f, 0.f, 0.f, 0.f};
        const bool interior = nxt_int;
        float4 a4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a4[i] = nxt[i];
        nxt_int = (t + 1 < SEGW) && is_interior(tt + 1);
        if (nxt_int) {
            const int64_t c1 = c0 + TCW;
#pragma unroll
            for (int i = 0; i < 4; ++i) nxt[i] = __ldcs(reinterpret_cast<const float4 *>(rowp[i] + c1));
        }
        if (interior) {
            const float4 xv = __ldg(reinterpret_cast<const float4 *>(x + c0));
            const float xc[4] = {xv.x * sc, xv.y * sc, xv.z * sc, xv.w * sc};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float a[4] = {a4[i].x, a4[i].y, a4[i].z, a4[i].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    rowacc[i] = fmaf(a[j], xc[j], rowacc[i]);
                    colacc[j] = fmaf(a[j], xr[i], colacc[j]);
                }
            }
        } else if (tt < tiles) {
            float xc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) xc[j] = (c0 + j < n) ? x[c0 + j] * sc : 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t gr = row0 + warp * 4 + i;
                if (gr >= n) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // strictly-lower entries of the diagonal tile are never loaded
                    const float a = (c0 + j < n && c0 + j >= gr) ? rowp[i][c0 + j] : 0.0f;
                    rowacc[i] = fmaf(a, xc[j], rowacc[i]);
                    if (c0 + j > gr) colacc[j] = fmaf(a, xr[i], colacc[j]);
                }
            }
        }
        // this thread's column partials of tile t (one owner per slot)
#pragma unroll
        for (int j = 0; j < 4; ++j) colsum[warp][t * TCW + lane * 4 + j] = colacc[j];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < SEGW * TCW; c += NTW) {
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += colsum[w][c];
        const int64_t gc = row0 + (int64_t)t0 * TCW + c;
        if (gc < n && s != 0.0f) atomicAdd(&y[gc], s);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s = rowacc[i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int64_t gr = row0 + warp * 4 + i;
        if (lane == 0 && gr < n) {
            if (t0 == 0) s = fmaf(shift, xr[i], s);  // the segment holding the diagonal
            atomicAdd(&y[gr], s);
        }
    }

    // ticket: the last block finishes the product
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == nactive - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NTW) {
        const double v = (double)__ldcg(&y[i]);
        acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < NTW / 32; ++w) s += red[w];
        const double nrm = sqrt(s);
        scal[1] = nrm;
        scal[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
        if (d_sigma) *d_sigma = nrm;
        *counter = 0u;
    }
    for (int64_t i = threadIdx.x; i < n; i += NTW) other[i] = 0.0f;
}

// The same product on the BF16 image A' of the block upper triangle
// (A = A' + A'^T; written by the tensor-core pass's pack kernel, zero padded
// to npad = a multiple of 256).  Block row of 32 rows from row0: its tiles
// start at the first column of its 256 x 256 diagonal block and are 256
// columns wide (lane l: columns 8l..8l+7, one 16-byte load per row); no
// entry needs masking, and the diagonal block's halved diagonal enters once
// through the row sums and once through the column sums.
constexpr int TCB = 256;   // columns per BF16 tile
constexpr int SEGB = 4;    // tiles per block

__device__ __forceinline__ void bf16x8_to_f32(const uint4 u, float (&a)[8])
{
    a[0] = __uint_as_float(u.x << 16); a[1] = __uint_as_float(u.x & 0xFFFF0000u);
    a[2] = __uint_as_float(u.y << 16); a[3] = __uint_as_float(u.y & 0xFFFF0000u);
    a[4] = __uint_as_float(u.z << 16); a[5] = __uint_as_float(u.z & 0xFFFF0000u);
    a[6] = __uint_as_float(u.w << 16); a[7] = __uint_as_float(u.w & 0xFFFF0000u);
}

__global__ void __launch_bounds__(NTW)
sym_gemv_bf16_kernel(const uint16_t *__restrict__ Ab, int64_t ldb, int64_t n, int64_t npad,
                     const float *__restrict__ x, float *__restrict__ y, float *__restrict__ other,
                     double *scal, unsigned *counter, const double *d_shift_neg, double *d_sigma,
                     unsigned nactive)
{
    __shared__ float colsum[8][SEGB * TCB];
    __shared__ double red[NTW / 32];
    __shared__ bool s_last;
    const int64_t row0 = (int64_t)blockIdx.y * TRW;
    const int64_t cs = (row0 / 256) * 256;
    const int tiles = (int)((npad - cs) / TCB);
    const int t0 = (int)blockIdx.x * SEGB;
    if (t0 >= tiles) return;
    const float sc = (float)scal[0];
    const float shift = d_shift_neg ? (float)(-(*d_shift_neg)) : 0.0f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    float rowacc[4] = {0.f, 0.f, 0.f, 0.f};
    float xr[4];
    const uint16_t *rowp[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gr = row0 + warp * 4 + i;      // < npad
        xr[i] = gr < n ? x[gr] * sc : 0.0f;
        rowp[i] = Ab + gr * ldb;
    }
    const int nt = min(SEGB, tiles - t0);
    uint4 nxt[4];
    {
        const int64_t c0 = cs + (int64_t)t0 * TCB + lane * 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) nxt[i] = __ldcs(reinterpret_cast<const uint4 *>(rowp[i] + c0));
    }
#pragma unroll 1
    for (int t = 0; t < nt; ++t) {
        const int64_t c0 = cs + (int64_t)(t0 + t) * TCB + lane * 8;
        uint4 cur[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) cur[i] = nxt[i];
        if (t + 1 < nt) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                nxt[i] = __ldcs(reinterpret_cast<const uint4 *>(rowp[i] + c0 + TCB));
        }
        float xc[8];
        if (c0 + 8 <= n) {
            const float4 x0 = __ldg(reinterpret_cast<const float4 *>(x + c0));
            const float4 x1 = __ldg(reinterpret_cast<const float4 *>(x + c0 + 4));
            xc[0] = x0.x * sc; xc[1] = x0.y * sc; xc[2] = x0.z * sc; xc[3] = x0.w * sc;
            xc[4] = x1.x * sc; xc[5] = x1.y * sc; xc[6] = x1.z * sc; xc[7] = x1.w * sc;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) xc[j] = (c0 + j < n) ? x[c0 + j] * sc : 0.0f;
        }
        float colacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float a[8];
            bf16x8_to_f32(cur[i], a);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                rowacc[i] = fmaf(a[j], xc[j], rowacc[i]);
                colacc[j] = fmaf(a[j], xr[i], colacc[j]);
            }
        }
        float4 *dst = reinterpret_cast<float4 *>(&colsum[warp][t * TCB + lane * 8]);
        dst[0] = make_float4(colacc[0], colacc[1], colacc[2], colacc[3]);
        dst[1] = make_float4(colacc[4], colacc[5], colacc[6], colacc[7]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nt * TCB; c += NTW) {
        float sacc = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) sacc += colsum[w][c];
        const int64_t gc = cs + (int64_t)t0 * TCB + c;
        if (gc < n && sacc != 0.0f) atomicAdd(&y[gc], sacc);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float sacc = rowacc[i];
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        const int64_t gr = row0 + warp * 4 + i;
        if (lane == 0 && gr < n) {
            if (t0 == 0) sacc = fmaf(shift, xr[i], sacc);  // the segment holding the diagonal
            atomicAdd(&y[gr], sacc);
        }
    }

    // ticket: the last block finishes the product
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == nactive - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NTW) {
        const double v = (double)__ldcg(&y[i]);
        acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sacc = 0.0;
        for (int w = 0; w < NTW / 32; ++w) sacc += red[w];
        const double nrm = sqrt(sacc);
        scal[1] = nrm;
        scal[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
        if (d_sigma) *d_sigma = nrm;
        *counter = 0u;
    }
    for (int64_t i = threadIdx.x; i < n; i += NTW) other[i] = 0.0f;
}

__global__ void pi_init_kernel(double *scal, float *v1, int64_t n)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) { scal[0] = 1.0; scal[1] = 0.0; }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v1[i] = 0.0f;
}

// alpha = alpha_in if alpha_in > 0, else |sigma1 - sigma2|.  The shift used by
// the range finder is alpha when alpha is finite and > 1e-300; otherwise 0
// and bit 0 of *d_info is set (the call degrades to Alg. 2).
__global__ void alpha_finish_kernel(const double *d_s1, const double *d_s2, double alpha_in,
                                    double *d_alpha, double *d_shift, int *d_info)
{
    double a = alpha_in;
    if (!(alpha_in > 0.0)) a = fabs(*d_s1 - *d_s2);
    const bool ok = isfinite(a) && a > 1e-300;
    if (d_alpha) *d_alpha = a;
    *d_shift = ok ? a : 0.0;
    if (d_info) *d_info = ok ? 0 : 1;
}

}  // namespace

cudaError_t launch_power_iteration(cudaStream_t s, const float *A, int64_t n, int64_t lda, int N,
                                   uint64_t seed, uint32_t stream_id, const double *d_shift_neg,
                                   float *v0, float *v1, double *scal, unsigned *counter,
                                   double *d_sigma)
{
    cudaError_t e = launch_gaussian(s, seed, stream_id, n, 1, 1, n, v0, n);
    if (e != cudaSuccess) return e;
    pi_init_kernel<<<64, 256, 0, s>>>(scal, v1, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = (int)((n + TRW - 1) / TRW);
    int64_t blocks = 0;
    for (int I = 0; I < nb; ++I) {
        const int tiles = (int)((n - (int64_t)I * TRW + TCW - 1) / TCW);
        blocks += (tiles + SEGW - 1) / SEGW;
    }
    const int maxseg = (int)(((n + TCW - 1) / TCW + SEGW - 1) / SEGW);  // row 0 has the most
    const dim3 grid((unsigned)maxseg, (unsigned)nb);
    const int vec = ((lda % 4) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    float *in = v0, *out = v1;
    for (int it = 0; it <= N; ++it) {
        sym_gemv_kernel<<<grid, NTW, 0, s>>>(A, n, lda, in, out, in, scal, counter, d_shift_neg,
                                             it == N ? d_sigma : nullptr, (unsigned)blocks, vec);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float *t = in; in = out; out = t;
    }
    return cudaSuccess;
}

cudaError_t launch_power_iteration_bf16(cudaStream_t s, const uint16_t *Ab, int64_t ldb, int64_t n,
                                        int N, uint64_t seed, uint32_t stream_id,
                                        const double *d_shift_neg, float *v0, float *v1, double *scal,
                                        unsigned *counter, double *d_sigma)
{
    const int64_t npad = psd_round_up(n, 256);
    if (ldb < npad || (ldb % 8) != 0 || (reinterpret_cast<uintptr_t>(Ab) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(v0) & 15) != 0 || (reinterpret_cast<uintptr_t>(v1) & 15) != 0)
        return cudaErrorInvalidValue;
    cudaError_t e = launch_gaussian(s, seed, stream_id, n, 1, 1, n, v0, n);
    if (e != cudaSuccess) return e;
    pi_init_kernel<<<64, 256, 0, s>>>(scal, v1, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = (int)((n + TRW - 1) / TRW);   // block rows holding rows < n
    int64_t blocks = 0;
    for (int I = 0; I < nb; ++I) {
        const int64_t cs = ((int64_t)I * TRW / 256) * 256;
        const int tiles = (int)((npad - cs) / TCB);
        blocks += (tiles + SEGB - 1) / SEGB;
    }
    const int maxseg = (int)((npad / TCB + SEGB - 1) / SEGB);
    const dim3 grid((unsigned)maxseg, (unsigned)nb);
    float *in = v0, *out = v1;
    for (int it = 0; it <= N; ++it) {
        sym_gemv_bf16_kernel<<<grid, NTW, 0, s>>>(Ab, ldb, n, npad, in, out, in, scal, counter,
                                                  d_shift_neg, it == N ? d_sigma : nullptr,
                                                  (unsigned)blocks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float *t = in; in = out; out = t;
    }
    return cudaSuccess;
}

cudaError_t launch_alpha_finish(cudaStream_t s, const double *d_s1, const double *d_s2,
                                double alpha_in, double *d_alpha, double *d_shift, int *d_info)
{
    alpha_finish_kernel<<<1, 1, 0, s>>>(d_s1, d_s2, alpha_in, d_alpha, d_shift, d_info);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of min_eig.
//
// For callers that cannot call cudaMalloc: code running inside another
// library's memory manager or a custom allocator that forbids allocations in
// its hot path, plug-ins whose host cannot grant device allocations, or
// contexts whose memory is capped and fully reserved up front.  Its scratch
// (the two power-iteration vectors, the norms and the completion ticket) is a
// fixed file-scope device array, present on every GPU that loads this
// library until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NOALLOC_MAX_N = PSDPROJ_NOALLOC_MAX_N;
constexpr size_t NOALLOC_VEC_BYTES = sizeof(float) * (size_t)NOALLOC_MAX_N;
constexpr size_t NOALLOC_BYTES = 2 * NOALLOC_VEC_BYTES + 32 * sizeof(double) + 16 * sizeof(unsigned);

// the shared scratch: v0, v1, then 32 doubles (scales, sigmas, shift, info), then tickets
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

__global__ void noalloc_reset_kernel(unsigned *counter) { if (threadIdx.x < 16) counter[threadIdx.x] = 0u; }

__global__ void noalloc_copy_kernel(const double *s1, const double *s2, double *d1, double *d2)
{
    if (d1) *d1 = *s1;
    if (d2) *d2 = *s2;
}

}  // namespace

#include <mutex>

extern "C" int psdproj_min_eig_noalloc(const float *dA, int64_t n, int64_t lda, int N, uint64_t seed,
                                       double *d_alpha, double *d_sigma1, double *d_sigma2,
                                       void *stream)
{
    if (!dA || !d_alpha || n < 1 || lda < n || N < 0) return PSDPROJ_EINVAL;
    if (n > NOALLOC_MAX_N) return PSDPROJ_ETOOLARGE;
    // set-up, once per device, with that device current: the device address
    // of the scratch array (its name in host code is only a host-side stand-in)
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PSDPROJ_ECUDA;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PSDPROJ_ECUDA;
            addr[dev] = p;
        }
        base = static_cast<unsigned char *>(addr[dev]);
    }
    float *v0 = reinterpret_cast<float *>(base);
    float *v1 = reinterpret_cast<float *>(base + NOALLOC_VEC_BYTES);
    double *scal = reinterpret_cast<double *>(base + 2 * NOALLOC_VEC_BYTES);
    unsigned *counter = reinterpret_cast<unsigned *>(base + 2 * NOALLOC_VEC_BYTES + 32 * sizeof(double));
    double *sig1 = scal + 16, *sig2 = scal + 17, *shift = scal + 18;
    int *info = reinterpret_cast<int *>(scal + 19);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the ticket must start at zero whatever an earlier call left behind
    noalloc_reset_kernel<<<1, 32, 0, s>>>(counter);
    if (cudaGetLastError() != cudaSuccess) return PSDPROJ_ECUDA;
    if (launch_power_iteration(s, dA, n, lda, N, seed, 3u, nullptr, v0, v1, scal, counter, sig1) != cudaSuccess)
        return PSDPROJ_ECUDA;
    if (launch_power_iteration(s, dA, n, lda, N, seed, 4u, sig1, v0, v1, scal, counter, sig2) != cudaSuccess)
        return PSDPROJ_ECUDA;
    if (launch_alpha_finish(s, sig1, sig2, 0.0, d_alpha, shift, info) != cudaSuccess) return PSDPROJ_ECUDA;
    if (d_sigma1 || d_sigma2) {
        noalloc_copy_kernel<<<1, 1, 0, s>>>(sig1, sig2, d_sigma1, d_sigma2);
        if (cudaGetLastError() != cudaSuccess) return PSDPROJ_ECUDA;
    }
    return PSDPROJ_OK;
}
