// k_misc.cu -- element-wise helpers, deterministic reductions and the
// scalar program of the step-size setup (Alg. 1 / Alg. 2 boxes).
#include <math.h>

#include <algorithm>

#include "ctpd_internal.cuh"

namespace ctpd {

static int grid_for(size_t n, int threads)
{
    size_t b = (n + threads - 1) / threads;
    return (int)(b < 152 * 16 ? (b == 0 ? 1 : b) : 152 * 16);
}

__global__ void k_fill(float *p, float v, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

void launch_fill(float *p, float v, size_t n, cudaStream_t st)
{
    counted();
    k_fill<<<grid_for(n, 256), 256, 0, st>>>(p, v, n);
}

__global__ void k_recip(const float *w, float *winv, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        winv[i] = 1.0f / w[i];
}

void launch_recip(const float *w, float *winv, size_t n, cudaStream_t st)
{
    counted();
    k_recip<<<grid_for(n, 256), 256, 0, st>>>(w, winv, n);
}

__global__ void k_sqrt(const float *a, float *out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = sqrtf(a[i]);
}

void launch_sqrt(const float *a, float *out, size_t n, cudaStream_t st)
{
    counted();
    k_sqrt<<<grid_for(n, 256), 256, 0, st>>>(a, out, n);
}

// s = sqrt(kappa w): the diagonal of the shift-variant preconditioner
__global__ void k_sv_scale(const float *w, const double *scal, float *s, size_t n)
{
    const float kappa = (float)scal[S_KAPPA];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s[i] = sqrtf(kappa * w[i]);
}

void launch_sv_scale(const float *w, const double *scal, float *s, size_t n, cudaStream_t st)
{
    counted();
    k_sv_scale<<<grid_for(n, 256), 256, 0, st>>>(w, scal, s, n);
}

// out[i] = +-1 from a 32-bit integer hash of i (the lowbias32 mixing of
// C. Wellons): a start vector with components in every symmetry class
__global__ void k_fill_sign(float *out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned x = (unsigned)i * 2654435761u + 12345u;
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        out[i] = (x & 1u) ? 1.0f : -1.0f;
    }
}

void launch_fill_sign(float *out, size_t n, cudaStream_t st)
{
    counted();
    k_fill_sign<<<grid_for(n, 256), 256, 0, st>>>(out, n);
}

// out = in * s (sqrt_s: in * sqrt(s))
__global__ void k_scale_by(const float *in, const float *s, int sqrt_s, float *out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i] * (sqrt_s ? sqrtf(s[i]) : s[i]);
}

void launch_scale_by(const float *in, const float *s, int sqrt_s, float *out, size_t n, cudaStream_t st)
{
    counted();
    k_scale_by<<<grid_for(n, 256), 256, 0, st>>>(in, s, sqrt_s, out, n);
}

// Deterministic reductions: a fixed grid of DOT_BLOCKS blocks; each thread
// sums its grid-stride elements in float, warps add their lanes by a fixed
// shuffle tree, the warp sums of a block are added in order, and the block
// partials the same way.  Everything is float (FP64 arithmetic is slow on
// this GPU); the relative error stays near 1e-6, well inside what the
// step-size setup needs.
constexpr int DOT_BLOCKS = 1216;   // 8 blocks per SM of 152: one element group per thread
constexpr int DOT_THREADS = 256;
size_t dot_partials_doubles() { return DOT_BLOCKS + 64; }   // + room for the ticket counter

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block total (valid in thread 0) of the float per-thread sums: warp trees,
// then the warp sums in order
__device__ __forceinline__ float block_sum(float v)
{
    __shared__ float wsum[DOT_THREADS / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < DOT_THREADS / 32; ++k) t += wsum[k];
    }
    return t;
}

// sum of the np block partials (strided runs per thread, then block_sum),
// valid in thread 0; every thread of the block calls it.  The partials are
// read from L2 (written by other blocks before their fence).
__device__ __forceinline__ float partials_sum(const double *partials, int np)
{
    float t = 0.0f;
    for (int i = threadIdx.x; i < np; i += blockDim.x) t += (float)__ldcg(partials + i);
    return block_sum(t);
}

__global__ void __launch_bounds__(DOT_THREADS)
k_dot_partial(const float *a, const float *b, size_t n, double *partials)
{
    float acc = 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc = fmaf(a[i], b ? b[i] : 1.0f, acc);
    const float t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = (double)t;
}

__global__ void __launch_bounds__(DOT_THREADS) k_dot_final(const double *partials, int np, double *scal, int slot)
{
    const float t = partials_sum(partials, np);
    if (threadIdx.x == 0) scal[slot] = (double)t;
}

void launch_dot(const float *a, const float *b, size_t n, double *scal, int slot,
                double *partials, cudaStream_t st)
{
    counted();
    k_dot_partial<<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(a, b, n, partials);
    counted();
    k_dot_final<<<1, DOT_THREADS, 0, st>>>(partials, DOT_BLOCKS, scal, slot);
}

// One-thread scalar program (keeps the whole setup on the device, so a
// solve needs no host round trip).
__global__ void k_scalars(double *s, int op, double a0, double a1, double a2, int i0)
{
    switch (op) {
    case SC_KAPPA_FROM_SUM:             // kappa = mean(1/w), a0 = count (Eq. 24)
        s[S_KAPPA] = s[S_RED0] / a0;
        break;
    case SC_TAU:                        // a0 = given tau (> 0) ; a1 = m ; i0 = mode
        if (a0 > 0.0) s[S_TAU] = a0;
        else s[S_TAU] = (i0 == CT_LOWDOSE) ? 3.14159265358979323846 * s[S_KAPPA] / (2.0 * a1) : 0.01;
        break;
    case SC_NORM_FROM_DOT:              // s[i0] = Rayleigh quotient <v, Mv>, |v| = 1
        s[i0] = s[S_RED0];
        break;
    case SC_SIGMA: {                    // a0 = given sigma ; a1 = rho ; i0 = mode
        if (a0 > 0.0) { s[S_SIGMA] = a0; break; }
        double bound = 1.0 / (s[S_TAU] * s[S_NADA]);
        if (i0 == CT_LOWDOSE && s[S_NWDW] > 0.0) bound = fmin(bound, 2.0 / s[S_NWDW]);
        s[S_SIGMA] = a1 * bound;
        break;
    }
    case SC_LAMBDA: {                   // a0 = beta ; i0 = mode
        double lam = (i0 == CT_LOWDOSE) ? s[S_TAU] * a0 : s[S_TAU];
        s[S_LAMBDA] = lam;
        s[S_INV8LAM] = lam > 0.0 ? 1.0 / (8.0 * lam) : 0.0;
        break;
    }
    case SC_SET:
        s[i0] = a0;
        break;
    case SC_COPY:                       // s[i0] = s[(int)a0]
        s[i0] = s[(int)a0];
        break;
    case SC_NORM_SQRT:                  // s[i0] = sqrt(s[(int)a0])
        s[i0] = sqrt(s[(int)a0]);
        break;
    case SC_AXPY_SLOT:                  // s[i0] += a0 * s[(int)a1]
        s[i0] += a0 * s[(int)a1];
        break;
    }
    float *f = reinterpret_cast<float *>(s + S_F32);
    f[F_TAU] = (float)s[S_TAU];
    f[F_SIGMA] = (float)s[S_SIGMA];
    f[F_LAMBDA] = (float)s[S_LAMBDA];
    f[F_INV8LAM] = (float)s[S_INV8LAM];
}

// Largest eigenvalue of the Lanczos tridiagonal T_k (diagonal s[base + 2j],
// off-diagonal s[base + 2j + 1]) into s[out]: multisection on the Sturm
// count of T - x I (the number of negative pivots of its LDL^T is the
// number of eigenvalues below x), 32 points per round.  The count runs in
// float on T scaled by its Gershgorin bound (backward stable: the count is
// exact for a matrix within a few float ulps of T); the result is the upper
// end of the final bracket, so it errs high.
__global__ void k_lanczos_max(double *s, int base, int k, int out)
{
    __shared__ float ta[LANCZOS_MAX], tb[LANCZOS_MAX];
    const int lane = threadIdx.x;
    for (int j = lane; j < k; j += 32) {
        ta[j] = (float)s[base + 2 * j];
        tb[j] = (float)s[base + 2 * j + 1];
    }
    __syncwarp();
    float glo = 0.0f, ghi = 0.0f;
    for (int j = 0; j < k; ++j) {   // Gershgorin interval
        const float rad = (j > 0 ? fabsf(tb[j - 1]) : 0.0f) + (j + 1 < k ? fabsf(tb[j]) : 0.0f);
        glo = j == 0 ? ta[j] - rad : fminf(glo, ta[j] - rad);
        ghi = j == 0 ? ta[j] + rad : fmaxf(ghi, ta[j] + rad);
    }
    const float big = fmaxf(fabsf(glo), fabsf(ghi));
    if (!(big > 0.0f)) {
        if (lane == 0) s[out] = 0.0;
        return;
    }
    const float inv = 1.0f / big;
    float lo = glo * inv, hi = ghi * inv;
    for (int round = 0; round < 8 && hi - lo > 4e-7f * fmaxf(fabsf(hi), 1e-30f); ++round) {
        const float x = lo + (hi - lo) * (float)(lane + 1) * (1.0f / 33.0f);
        int below = 0;
        float d = 1.0f;
        for (int j = 0; j < k; ++j) {
            const float b = j > 0 ? tb[j - 1] * inv : 0.0f;
            d = (ta[j] * inv - x) - (j > 0 ? b * b / d : 0.0f);
            if (d == 0.0f) d = -1e-30f;
            if (d < 0.0f) ++below;
        }
        // lowest point with all k eigenvalues below it bounds lambda_max from above
        const unsigned all = __ballot_sync(0xffffffffu, below == k);
        const int first = all ? __ffs(all) - 1 : 32;     // lanes >= first have below == k
        const float nlo = first == 0 ? lo : lo + (hi - lo) * (float)first * (1.0f / 33.0f);
        const float nhi = first == 32 ? hi : lo + (hi - lo) * (float)(first + 1) * (1.0f / 33.0f);
        lo = nlo;
        hi = fmaxf(nhi, nlo);
    }
    if (lane != 0) return;
    // theta = the upper end of the bracket; the estimate is theta + beta_k |y_k|,
    // the Ritz value plus its residual norm (y the unit eigenvector of T for
    // theta, beta_k the norm left after the last step), so that it lies above
    // lambda_max once the Ritz vector has found the top of the spectrum.
    // y by two steps of inverse iteration with theta I - T (positive definite,
    // as theta is above every eigenvalue of T): tridiagonal elimination in
    // double on this one thread.
    const double theta = (double)(hi * big) * (1.0 + 1e-6);
    double y[LANCZOS_MAX], cp[LANCZOS_MAX];
    for (int j = 0; j < k; ++j) y[j] = 1.0;
    for (int itr = 0; itr < 2; ++itr) {
        double m = theta - s[base];
        if (!(m > 0.0)) m = 1e-300;
        cp[0] = k > 1 ? -s[base + 1] / m : 0.0;
        y[0] = y[0] / m;
        for (int j = 1; j < k; ++j) {
            const double sub = -s[base + 2 * j - 1];
            double d = (theta - s[base + 2 * j]) - sub * cp[j - 1];
            if (!(d > 0.0)) d = 1e-300;
            cp[j] = j + 1 < k ? -s[base + 2 * j + 1] / d : 0.0;
            y[j] = (y[j] - sub * y[j - 1]) / d;
        }
        for (int j = k - 2; j >= 0; --j) y[j] -= cp[j] * y[j + 1];
        double nrm = 0.0;
        for (int j = 0; j < k; ++j) nrm += y[j] * y[j];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0) || !isfinite(nrm)) break;
        for (int j = 0; j < k; ++j) y[j] /= nrm;
    }
    const double res = fabs(s[base + 2 * (k - 1) + 1] * y[k - 1]);
    s[out] = isfinite(res) ? theta + res : theta;
}

void launch_lanczos_max(double *scal, int base, int k, int out, cudaStream_t st)
{
    counted();
    k_lanczos_max<<<1, 32, 0, st>>>(scal, base, k, out);
}

// One half of a Lanczos step on unnormalised vectors (t_j = n_j q_j with
// n_0 = s[n0slot] and n_j = beta_{j-1} = s[base + 2j - 1]):
//   phase 0:  w = w / n_j - (n_j / n_{j-1}) t_{j-1}   (w held op(t_j));
//             alpha_j = <w, t_j> / n_j                 -> s[base + 2j]
//   phase 1:  w -= (alpha_j / n_j) t_j;  beta_j = |w|  -> s[base + 2j + 1]
// The dot is the deterministic reduction above; the last block to finish
// (ticket counter) adds the partials in block order and resets the counter.
__global__ void __launch_bounds__(DOT_THREADS)
k_lanczos_step(float *__restrict__ w, const float *__restrict__ tp, const float *__restrict__ tc, size_t n,
               double *s, int base, int n0slot, int j, int phase, double *partials, unsigned *ticket)
{
    __shared__ bool last;
    __shared__ float coef[3];
    const float *x2 = phase == 0 ? tp : tc;
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(tc) |
                       reinterpret_cast<uintptr_t>(x2)) & 15) == 0;
    const size_t n4 = vec ? n / 4 : 0;   // four elements per load
    float4 *w4 = reinterpret_cast<float4 *>(w);
    const float4 *x4 = reinterpret_cast<const float4 *>(x2), *t4 = reinterpret_cast<const float4 *>(tc);
    // the first group's loads go out before the coefficients are known
    const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float4 a0 = zero, xa = zero, ta = zero;
    if (tid < n4) {
        a0 = w4[tid];
        xa = x4[tid];
        if (phase == 0) ta = t4[tid];
    }
    // coefficients from the double slots, once per block (FP64 is slow here)
    if (threadIdx.x == 0) {
        const float nj = (float)(j == 0 ? s[n0slot] : s[base + 2 * j - 1]);
        float c1 = 1.0f, c2 = 0.0f;
        if (phase == 0) {
            const float njm1 = (float)(j <= 1 ? s[n0slot] : s[base + 2 * j - 3]);
            c1 = nj > 0.0f ? 1.0f / nj : 0.0f;
            c2 = (j > 0 && njm1 > 0.0f) ? nj / njm1 : 0.0f;
        } else {
            c2 = nj > 0.0f ? (float)s[base + 2 * j] / nj : 0.0f;
        }
        coef[0] = c1;
        coef[1] = c2;
        coef[2] = nj;
    }
    __syncthreads();
    const float c1 = coef[0], c2 = coef[1];
    float acc = 0.0f;
    auto group = [&](float4 a, float4 x, float4 t, size_t i) {
        if (c2 == 0.0f) x = zero;   // t_{-1} is never read (it may hold anything)
        a.x = fmaf(-c2, x.x, a.x * c1);
        a.y = fmaf(-c2, x.y, a.y * c1);
        a.z = fmaf(-c2, x.z, a.z * c1);
        a.w = fmaf(-c2, x.w, a.w * c1);
        w4[i] = a;
        const float4 d = phase == 0 ? t : a;
        acc = fmaf(a.x, d.x, acc);
        acc = fmaf(a.y, d.y, acc);
        acc = fmaf(a.z, d.z, acc);
        acc = fmaf(a.w, d.w, acc);
    };
    if (tid < n4) group(a0, xa, ta, tid);
    for (size_t i = tid + stride; i < n4; i += stride) group(w4[i], x4[i], phase == 0 ? t4[i] : zero, i);
    const size_t done = n4 * 4;
    for (size_t i = done + tid; i < n; i += stride) {
        float wi = w[i] * c1;
        if (c2 != 0.0f) wi = fmaf(-c2, x2[i], wi);
        w[i] = wi;
        acc = fmaf(wi, phase == 0 ? tc[i] : wi, acc);
    }
    const float t = block_sum(acc);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = (double)t;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const float tf = partials_sum(partials, gridDim.x);
    if (threadIdx.x == 0) {
        const float nj = coef[2];
        if (phase == 0) s[base + 2 * j] = nj > 0.0f ? (double)(tf / nj) : 0.0;
        else s[base + 2 * j + 1] = (double)sqrtf(fmaxf(tf, 0.0f));
        *ticket = 0u;
    }
}

void launch_lanczos_step(float *w, const float *tp, const float *tc, size_t n, double *scal, int base, int n0slot,
                         int j, int phase, double *partials, unsigned *ticket, cudaStream_t st)
{
    // one four-element group per thread: no block without elements, so the
    // ticket sees only as many arrivals as the vector needs (256 blocks for
    // a 512^2 image instead of the full reduction grid)
    const size_t groups = (n + 4 * (size_t)DOT_THREADS - 1) / (4 * (size_t)DOT_THREADS);
    const int blocks = (int)std::min<size_t>(std::max<size_t>(groups, 1), DOT_BLOCKS);
    counted();
    k_lanczos_step<<<blocks, DOT_THREADS, 0, st>>>(w, tp, tc, n, scal, base, n0slot, j, phase, partials, ticket);
}

__global__ void k_axpy_neg(float *w, const float *q, size_t n, const double *scal, int slot)
{
    const float c = (float)scal[slot];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        w[i] = fmaf(-c, q[i], w[i]);
}

void launch_axpy_neg(float *w, const float *q, size_t n, const double *scal, int slot, cudaStream_t st)
{
    counted();
    k_axpy_neg<<<grid_for(n, 256), 256, 0, st>>>(w, q, n, scal, slot);
}

void launch_scalars(double *scal, int op, double a0, double a1, double a2, int i0, cudaStream_t st)
{
    counted();
    k_scalars<<<1, 1, 0, st>>>(scal, op, a0, a1, a2, i0);
}

}  // namespace ctpd
