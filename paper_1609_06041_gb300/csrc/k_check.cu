// k_check.cu -- input checks of a solve and its optional per-iteration trace.
//
// Checks: the weights W = diag(w) of Eq. 1 must be positive and finite
// (W^-1 enters every dual step of Algorithm 1), and the data b finite.  A
// device pass sets bits of a flag word in the solve's scalar block, which
// the host reads when it synchronises (the report, ct_pdtv_status); the
// final image gets the same finiteness check.
//
// Trace: after iteration k the cost f(x^{k+1}) = beta psi(x^{k+1}) +
// 1/2 ||A x^{k+1} - b||_W^2 of Eq. 1 (Algorithm 1), or the residual
// ||A x^{k+1} - b|| of the constraint of Eq. 25 (Algorithm 2), from the
// projector's band partial sums of A x^{k+1}.  Per-thread float sums, block
// sums in a fixed shuffle order, and the block sums added in order in
// double by one thread: deterministic.
#include <math.h>

#include "ctpd_internal.cuh"

namespace ctpd {

constexpr int CHK_THREADS = 256;

static int chk_grid(size_t n)
{
    const size_t b = (n + CHK_THREADS - 1) / CHK_THREADS;
    return (int)(b == 0 ? 1 : (b < 152 * 8 ? b : 152 * 8));
}

__global__ void __launch_bounds__(CHK_THREADS)
k_check_inputs(const float *__restrict__ b, const float *__restrict__ w, size_t n, unsigned *flags)
{
    unsigned f = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (!isfinite(b[i])) f |= CHK_NONFINITE_INPUT;
        if (w) {
            const float wi = w[i];
            if (!isfinite(wi)) f |= CHK_NONFINITE_INPUT;
            else if (!(wi > 0.0f)) f |= CHK_WEIGHT_NOT_POSITIVE;
        }
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

void launch_check_inputs(const float *b, const float *w, size_t n, unsigned *flags, cudaStream_t st)
{
    counted();
    k_check_inputs<<<chk_grid(n), CHK_THREADS, 0, st>>>(b, w, n, flags);
}

__global__ void __launch_bounds__(CHK_THREADS)
k_check_finite(const float *__restrict__ x, size_t n, unsigned *flags, unsigned bit)
{
    unsigned f = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) f = bit;
    f = __reduce_or_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

void launch_check_finite(const float *x, size_t n, unsigned *flags, unsigned bit, cudaStream_t st)
{
    counted();
    k_check_finite<<<chk_grid(n), CHK_THREADS, 0, st>>>(x, n, flags, bit);
}

// ---- trace ----
constexpr int TR_BLOCKS = 304;   // per part (data term, penalty)

size_t trace_scratch_doubles() { return 2 * TR_BLOCKS; }

__device__ __forceinline__ float chk_block_sum(float v)
{
    __shared__ float ws[CHK_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int i = 0; i < CHK_THREADS / 32; ++i) t += ws[i];
    return t;
}

// blocks [0, TR_BLOCKS): sum_i wt_i (A x - b)_i^2 with A x = scale_v sum_bands
// partial (wt = w, or 1 without weights); blocks [TR_BLOCKS, 2 TR_BLOCKS):
// psi(x) of Eq. 2 with forward differences, zero across the last column / row
__global__ void __launch_bounds__(CHK_THREADS)
k_trace_parts(const float *__restrict__ partial, int nb, const ViewP *__restrict__ views, const float *__restrict__ b,
              const float *__restrict__ w, int V, int B, const float *__restrict__ x, int N, double *part)
{
    float acc = 0.0f;
    if (blockIdx.x < TR_BLOCKS) {
        const size_t I = (size_t)V * B;
        for (size_t i = blockIdx.x * (size_t)CHK_THREADS + threadIdx.x; i < I; i += (size_t)TR_BLOCKS * CHK_THREADS) {
            float s = 0.0f;
            for (int k = 0; k < nb; ++k) s += partial[k * I + i];
            const float e = s * views[i / B].scale - b[i];
            acc = fmaf(w ? w[i] * e : e, e, acc);
        }
    } else {
        const size_t J = (size_t)N * N;
        for (size_t j = (blockIdx.x - TR_BLOCKS) * (size_t)CHK_THREADS + threadIdx.x; j < J;
             j += (size_t)TR_BLOCKS * CHK_THREADS) {
            const int r = (int)(j / N), c = (int)(j - (size_t)r * N);
            const float xv = x[j];
            const float dx = c + 1 < N ? x[j + 1] - xv : 0.0f;
            const float dy = r + 1 < N ? x[j + N] - xv : 0.0f;
            acc += sqrtf(fmaf(dx, dx, dy * dy));
        }
    }
    const float t = chk_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = (double)t;
}

// out = beta psi + fid / 2 (lowdose) or sqrt(fid)
__global__ void k_trace_final(const double *part, double beta, int lowdose, double *out)
{
    double fid = 0.0, tv = 0.0;
    for (int i = 0; i < TR_BLOCKS; ++i) fid += part[i];
    for (int i = 0; i < TR_BLOCKS; ++i) tv += part[TR_BLOCKS + i];
    *out = lowdose ? beta * tv + 0.5 * fid : sqrt(fid);
}

void launch_trace(const Geometry *g, const float *partial, const float *b, const float *w, const float *x,
                  double beta, int lowdose, double *part, double *out, cudaStream_t st)
{
    counted(2);
    k_trace_parts<<<2 * TR_BLOCKS, CHK_THREADS, 0, st>>>(partial, proj_bands(g->n), g->d_views, b,
                                                         lowdose ? w : nullptr, g->n_views, g->n_bins, x, g->n,
                                                         part);
    k_trace_final<<<1, 1, 0, st>>>(part, beta, lowdose, out);
}

}  // namespace ctpd
