// k_misc.cu -- element-wise helpers, deterministic reductions and the
// scalar program of the step-size setup (Alg. 1 / Alg. 2 boxes).
#include <math.h>

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

// Deterministic dot product: a fixed grid of DOT_BLOCKS blocks writes one
// double partial each (fixed grid-stride order, fixed tree), then one block
// adds the partials in a fixed order.
constexpr int DOT_BLOCKS = 304;
size_t dot_partials_doubles() { return DOT_BLOCKS + 64; }   // + room for the ticket counter

__global__ void __launch_bounds__(256)
k_dot_partial(const float *a, const float *b, size_t n, double *partials)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (b ? (double)b[i] : 1.0);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_dot_final(const double *partials, int np, double *scal, int slot)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) scal[slot] = red[0];
}

void launch_dot(const float *a, const float *b, size_t n, double *scal, int slot,
                double *partials, cudaStream_t st)
{
    counted();
    k_dot_partial<<<DOT_BLOCKS, 256, 0, st>>>(a, b, n, partials);
    counted();
    k_dot_final<<<1, 256, 0, st>>>(partials, DOT_BLOCKS, scal, slot);
}

__global__ void k_normalize(const float *in, float *out, size_t n, const double *scal, int slot)
{
    const float s2 = (float)scal[slot];
    const float inv = s2 > 0.0f ? rsqrtf(s2) : 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i] * inv;
}

void launch_normalize(const float *in, float *out, size_t n, const double *scal, int slot,
                      cudaStream_t st)
{
    counted();
    k_normalize<<<grid_for(n, 256), 256, 0, st>>>(in, out, n, scal, slot);
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
}

// Largest eigenvalue of the Lanczos tridiagonal T_k (diagonal s[S_LZ + 2j],
// off-diagonal s[S_LZ + 2j + 1]) into s[out]: multisection on the Sturm
// count of T - x I (the number of negative pivots of its LDL^T is the
// number of eigenvalues below x), 32 points per round, in double precision.
__global__ void k_lanczos_max(double *s, int k, int out)
{
    const int lane = threadIdx.x;
    double lo = 0.0, hi = 0.0;
    for (int j = 0; j < k; ++j) {   // Gershgorin interval
        const double al = s[S_LZ + 2 * j];
        const double rad = (j > 0 ? fabs(s[S_LZ + 2 * j - 1]) : 0.0) + (j + 1 < k ? fabs(s[S_LZ + 2 * j + 1]) : 0.0);
        lo = j == 0 ? al - rad : fmin(lo, al - rad);
        hi = j == 0 ? al + rad : fmax(hi, al + rad);
    }
    for (int round = 0; round < 12 && hi - lo > 1e-13 * fmax(fabs(hi), 1e-300); ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        int below = 0;
        double d = 1.0;
        for (int j = 0; j < k; ++j) {
            const double b = j > 0 ? s[S_LZ + 2 * j - 1] : 0.0;
            d = (s[S_LZ + 2 * j] - x) - (j > 0 ? b * b / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++below;
        }
        // lowest point with all k eigenvalues below it bounds lambda_max from above
        const unsigned all = __ballot_sync(0xffffffffu, below == k);
        const int first = all ? __ffs(all) - 1 : 32;     // lanes >= first have below == k
        const double nlo = first == 0 ? lo : lo + (hi - lo) * (double)first / 33.0;
        const double nhi = first == 32 ? hi : lo + (hi - lo) * (double)(first + 1) / 33.0;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) s[out] = hi;
}

void launch_lanczos_max(double *scal, int k, int out, cudaStream_t st)
{
    counted();
    k_lanczos_max<<<1, 32, 0, st>>>(scal, k, out);
}

// w -= c q (c = scal[cslot], skipped when cslot < 0), then scal[dslot] =
// <w, v> (v = w when NULL): a fixed grid writes per-block partials; the
// last block to finish (ticket counter) adds them in block order and
// resets the counter, so the sum is deterministic and nothing waits.
constexpr int AXD_BLOCKS = 304;
__global__ void __launch_bounds__(256)
k_axpy_dot(float *w, const float *q, size_t n, double *scal, int cslot, const float *v, int dslot,
           double *partials, unsigned *ticket, int sqrt_out)
{
    __shared__ double red[256];
    __shared__ bool last;
    const float c = cslot >= 0 ? (float)scal[cslot] : 0.0f;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float wi = w[i];
        if (cslot >= 0) {
            wi = fmaf(-c, q[i], wi);
            w[i] = wi;
        }
        acc += (double)wi * (double)(v ? v[i] : wi);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += ((volatile double *)partials)[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scal[dslot] = red[0];
        if (sqrt_out >= 0) scal[sqrt_out] = sqrt(red[0]);
        *ticket = 0u;
    }
}

void launch_axpy_dot(float *w, const float *q, size_t n, double *scal, int cslot, const float *v, int dslot,
                     double *partials, unsigned *ticket, int sqrt_out, cudaStream_t st)
{
    counted();
    k_axpy_dot<<<AXD_BLOCKS, 256, 0, st>>>(w, q, n, scal, cslot, v, dslot, partials, ticket, sqrt_out);
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
