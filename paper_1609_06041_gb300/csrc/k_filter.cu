// k_filter.cu -- the preconditioner D (Eq. 24 / Eq. 32) as a per-view
// linear convolution along the detector, its taps, and the fused dual step
// (Step 3 of Algorithm 1 / 2 followed by Step 1 of the next iteration).
#include "ctpd_internal.cuh"

namespace ctpd {

constexpr int FT = 256;      // threads per view block
constexpr int FR = 4;        // outputs per thread, strided by FT

// Convolve the view held in shared memory `s_in` (B values) with the taps in
// `s_t` (index k + half - 1, zero padded so that every |k| <= B-1 is valid)
// for the outputs d = threadIdx.x + i*FT, i < FR (plus further rounds when
// B > FT*FR, handled by the caller's loop over `base`).
__device__ __forceinline__ void conv_view(const float *s_in, const float *s_t, int B, int tpad,
                                          int base, float acc[FR])
{
#pragma unroll
    for (int i = 0; i < FR; ++i) acc[i] = 0.0f;
    const int d0 = base + threadIdx.x;
    // s_t holds t[k] at index k + tpad; every output needs all e in [0, B)
    for (int e = 0; e < B; ++e) {
        const float xe = s_in[e];
#pragma unroll
        for (int i = 0; i < FR; ++i) acc[i] = fmaf(s_t[d0 + i * FT - e + tpad], xe, acc[i]);
    }
}

// Stage taps of half length `half` into shared memory padded to |k| <= B-1+FT*FR.
__device__ __forceinline__ int stage_taps(float *s_t, const float *taps, int half, int B)
{
    const int tpad = B - 1 + FT * FR;          // index of k = 0
    const int len = 2 * tpad + 1;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        int k = i - tpad;
        s_t[i] = (k > -half && k < half) ? taps[half - 1 + k] : 0.0f;
    }
    return tpad;
}

static size_t filter_smem(int B) { return sizeof(float) * (size_t)(2 * B + 2 * (B - 1 + FT * FR) + 1); }

__global__ void __launch_bounds__(FT)
k_filter(const float *__restrict__ taps, int half, const float *__restrict__ in,
         float *__restrict__ out, const float *__restrict__ pre, const float *__restrict__ post,
         int mode, const double *__restrict__ scal, int V, int B)
{
    extern __shared__ float sm[];
    float *s_in = sm;
    float *s_t = sm + B;
    const size_t off = ((size_t)blockIdx.y * V + blockIdx.x) * B;
    const int tpad = stage_taps(s_t, taps, half, B);
    for (int e = threadIdx.x; e < B; e += blockDim.x) {
        float val = in[off + e];
        if (pre) val *= pre[off + e];
        s_in[e] = val;
    }
    __syncthreads();
    const float sc = (mode == 1) ? -fscal(scal, F_SIGMA) : 1.0f;
    for (int base = 0; base < B; base += FT * FR) {
        float acc[FR];
        conv_view(s_in, s_t, B, tpad, base, acc);
#pragma unroll
        for (int i = 0; i < FR; ++i) {
            int d = base + threadIdx.x + i * FT;
            if (d < B) {
                float val = acc[i];
                if (post) val *= post[off + d];
                out[off + d] = sc * val;
            }
        }
    }
}

void launch_filter(const Geometry *g, const float *taps, int half, const float *in,
                   float *out, const float *pre, const float *post, int mode,
                   const double *scal, int batch, cudaStream_t st)
{
    size_t smem = filter_smem(g->n_bins);
    dim3 grd(g->n_views, batch);
    counted();
    k_filter<<<grd, FT, smem, st>>>(taps, half, in, out, pre, post, mode, scal, g->n_views, g->n_bins);
}

// Fused dual step for view v (one block per view):
//   mu' = mu + sigma D r                                  (Step 3)
//   mu_bar = 2 mu' - mu - sigma D (winv .* (mu' - mu))    (Step 1, Alg. 1)
//   mu_bar = 2 mu' - mu                                   (Step 1, Alg. 2)
// mu is updated in place; the view's values are read before any write.
__global__ void __launch_bounds__(FT)
k_dual(const float *__restrict__ taps, int half, const float *__restrict__ partial, int nb,
       const float *__restrict__ b, float *__restrict__ mu, float *__restrict__ mu_bar,
       const float *__restrict__ winv, int lowdose, const ViewP *__restrict__ views,
       const double *__restrict__ scal, int V, int B)
{
    extern __shared__ float sm[];
    float *s_in = sm;
    float *s_t = sm + B;
    const size_t off = (size_t)blockIdx.x * B;
    const size_t VB = (size_t)V * B;
    const float scale = views[blockIdx.x].scale;
    const int tpad = stage_taps(s_t, taps, half, B);
    // residual r = A x - b [- winv mu] from the projector's band partial sums
    for (int e = threadIdx.x; e < B; e += blockDim.x) {
        float acc = 0.0f;
        for (int k = 0; k < nb; ++k) acc += partial[k * VB + off + e];
        float r = acc * scale - b[off + e];
        if (lowdose) r -= winv[off + e] * mu[off + e];
        s_in[e] = r;
    }
    __syncthreads();
    const float sigma = fscal(scal, F_SIGMA);
    // B <= FT*FR*MAXR handled by keeping the per-round results in registers
    constexpr int MAXR = 8;
    float mun[MAXR][FR], mo[MAXR][FR];
    const int rounds = (B + FT * FR - 1) / (FT * FR);
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
        if (q >= rounds) break;
        float acc[FR];
        conv_view(s_in, s_t, B, tpad, q * FT * FR, acc);
#pragma unroll
        for (int i = 0; i < FR; ++i) {
            int d = q * FT * FR + threadIdx.x + i * FT;
            float m0 = d < B ? mu[off + d] : 0.0f;
            mo[q][i] = m0;
            mun[q][i] = m0 + sigma * acc[i];
        }
    }
    if (!lowdose) {
#pragma unroll
        for (int q = 0; q < MAXR; ++q) {
            if (q >= rounds) break;
#pragma unroll
            for (int i = 0; i < FR; ++i) {
                int d = q * FT * FR + threadIdx.x + i * FT;
                if (d < B) {
                    mu[off + d] = mun[q][i];
                    mu_bar[off + d] = 2.0f * mun[q][i] - mo[q][i];
                }
            }
        }
        return;
    }
    __syncthreads();   // everyone is done reading s_in
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
        if (q >= rounds) break;
#pragma unroll
        for (int i = 0; i < FR; ++i) {
            int d = q * FT * FR + threadIdx.x + i * FT;
            if (d < B) s_in[d] = winv[off + d] * (mun[q][i] - mo[q][i]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
        if (q >= rounds) break;
        float acc[FR];
        conv_view(s_in, s_t, B, tpad, q * FT * FR, acc);
#pragma unroll
        for (int i = 0; i < FR; ++i) {
            int d = q * FT * FR + threadIdx.x + i * FT;
            if (d < B) {
                mu[off + d] = mun[q][i];
                mu_bar[off + d] = 2.0f * mun[q][i] - mo[q][i] - sigma * acc[i];
            }
        }
    }
}

void launch_dual_update(const Geometry *g, const float *taps, int half, const float *partial,
                        const float *b, float *mu, float *mu_bar, const float *winv, int lowdose,
                        const double *scal, cudaStream_t st)
{
    size_t smem = filter_smem(g->n_bins);
    counted();
    k_dual<<<g->n_views, FT, smem, st>>>(taps, half, partial, proj_bands(g->n), b, mu, mu_bar, winv,
                                         lowdose, g->d_views, scal, g->n_views, g->n_bins);
}

void kernel_attrs_filter()
{
    cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filter_smem(8192));
    cudaFuncSetAttribute(k_dual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filter_smem(8192));
}

// Taps t[k] = (1/P) sum_j H(w_j) cos(2 pi j k / P), k = 0..B-1, written
// mirrored into taps[B-1 +- k].  One warp per k; the cosine argument is
// reduced exactly in integers ((j*k) mod P) and evaluated with cospif;
// compensated summation keeps the float sum at full precision.
// H(w) = |w|/(2 m tau + kappa |w|) (mode 0, Eq. 24) or |w|/(2 m tau) (mode 1, Eq. 32);
// modes 2 and 3 split mode 0 into the low band 2 m tau |w| / (2 m tau + kappa |w|)^2
// and the high band kappa w^2 / (2 m tau + kappa |w|)^2 of the shift-variant D.
__global__ void k_taps(int mode, int m, int P, int B, const double *__restrict__ scal,
                       float tau_h, float kappa_h, float *__restrict__ taps)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= B) return;
    const int k = warp;
    const float tau = scal ? fscal(scal, F_TAU) : tau_h;
    const float kappa = scal ? (float)scal[S_KAPPA] : kappa_h;
    const float two_m_tau = 2.0f * (float)m * tau;
    float sum = 0.0f, comp = 0.0f;
    for (int j = lane; j < P; j += 32) {
        const int jj = j < P - j ? j : P - j;
        const float w = 6.28318530717958647692f * (float)jj / (float)P;
        const float den = two_m_tau + kappa * w;
        // modes 2, 3: the low and high bands of mode 0 (shift-variant preconditioner)
        const float Hj = (mode == 0) ? w / den
                       : (mode == 1) ? w / two_m_tau
                       : (mode == 2) ? two_m_tau * w / (den * den) : kappa * w * w / (den * den);
        const int ph = (int)(((unsigned)j * (unsigned)k) & (unsigned)(P - 1));   // j k mod P, P a power of two
        const float term = Hj * cospif(2.0f * (float)ph / (float)P);
        const float y = term - comp;
        const float t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
        const float tk = sum / (float)P;
        taps[B - 1 + k] = tk;
        taps[B - 1 - k] = tk;
    }
}

void launch_taps(const Geometry *g, int mode, const double *scal, double tau, double kappa,
                 float *taps, cudaStream_t st)
{
    int threads = 256, warps_per = threads / 32;
    int blocks = (g->n_bins + warps_per - 1) / warps_per;
    counted();
    k_taps<<<blocks, threads, 0, st>>>(mode, g->n_views, g->n_fft, g->n_bins, scal,
                                       (float)tau, (float)kappa, taps);
}

}  // namespace ctpd
