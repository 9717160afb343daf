// k_grad.cu -- reductions used by the adjoint of the unrolled solve.
#include "ctpd_internal.cuh"

namespace ctpd {

constexpr int TC_VIEWS = 64;    // views per correlation block

// partial[lag][chunk] = sum over the chunk's views of sum_d g[v][d] s[v][d - k],
// k = lag - (half - 1), |k| < half: the derivative of <g, D s> with respect
// to the tap t[k] of D (out[d] = sum_e t[d - e] in[e]).  Float products
// summed per thread, double across the block.
__global__ void __launch_bounds__(256)
k_tapcorr(const float *__restrict__ g, const float *__restrict__ s, int nviews, int B, int half,
          double *__restrict__ partial)
{
    __shared__ double red[256];
    const int lag = blockIdx.x, chunk = blockIdx.y, k = lag - (half - 1);
    const int v0 = chunk * TC_VIEWS, v1 = min(nviews, v0 + TC_VIEWS);
    float acc = 0.0f;
    for (int v = v0; v < v1; ++v) {
        const float *gv = g + (size_t)v * B, *sv = s + (size_t)v * B;
        for (int d = threadIdx.x; d < B; d += blockDim.x) {
            const int e = d - k;
            if (e >= 0 && e < B) acc = fmaf(gv[d], sv[e], acc);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)lag * gridDim.y + chunk] = red[0];
}

// acc[lag] += coef * sum_chunk partial[lag][chunk] (chunks in order)
__global__ void k_tapcorr_acc(const double *__restrict__ partial, int nchunks, int nlags, double coef,
                              double *__restrict__ acc)
{
    const int lag = blockIdx.x * blockDim.x + threadIdx.x;
    if (lag >= nlags) return;
    double t = 0.0;
    for (int c = 0; c < nchunks; ++c) t += partial[(size_t)lag * nchunks + c];
    acc[lag] += coef * t;
}

size_t tapcorr_partials(int nviews, int half) { return (size_t)(2 * half - 1) * ((nviews + TC_VIEWS - 1) / TC_VIEWS); }

void launch_tapcorr_acc(const float *g, const float *s, int nviews, int B, int half, double coef,
                        double *partial, double *acc, cudaStream_t st)
{
    const int nl = 2 * half - 1, nc = (nviews + TC_VIEWS - 1) / TC_VIEWS;
    counted(2);
    k_tapcorr<<<dim3(nl, nc), 256, 0, st>>>(g, s, nviews, B, half, partial);
    k_tapcorr_acc<<<(nl + 127) / 128, 128, 0, st>>>(partial, nc, nl, coef, acc);
}

// scal[slot] += coef * sum(partials[0..n)), in order
__global__ void k_sum_partials(const double *__restrict__ partials, size_t n, double *scal, int slot, double coef)
{
    __shared__ double red[256];
    double t = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) t += partials[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[slot] += coef * red[0];
}

void launch_sum_partials(const double *partials, size_t n, double *scal, int slot, double coef, cudaStream_t st)
{
    counted();
    k_sum_partials<<<1, 256, 0, st>>>(partials, n, scal, slot, coef);
}

// grad[0 .. nl) = (float) tap accumulators; grad[nl] = (float) scal[slot] * fac
__global__ void k_grad_out(const double *__restrict__ acc, int nl, const double *__restrict__ scal, int slot,
                           double fac, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nl) grad[i] = (float)acc[i];
    if (i == nl) grad[nl] = (float)(scal[slot] * fac);
}

void launch_grad_out(const double *acc, int nl, const double *scal, int slot, double fac, float *grad,
                     cudaStream_t st)
{
    counted();
    k_grad_out<<<(nl + 1 + 127) / 128, 128, 0, st>>>(acc, nl, scal, slot, fac, grad);
}

}  // namespace ctpd
