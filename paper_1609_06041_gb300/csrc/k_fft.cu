// k_fft.cu -- the preconditioner D as a frequency-domain filter.
//
// D applies, along the detector of every view, the linear (zero-padded)
// convolution with the taps t[k], |k| < half (Eq. 24 / Eq. 32 give the
// taps from H).  With the view zero-padded to the period P >= 2B, the
// circular convolution with the taps placed at k mod P equals that linear
// convolution on bins 0..B-1, so D = IFFT_P(Hhat . FFT_P(.)) with Hhat the
// P-point DFT of the circularly placed taps.  The taps are real, so two
// views travel as the real and imaginary parts of one complex sequence.
//
// FFTs run in shared memory as Stockham autosort stages (radix 8, then a
// radix-4 or radix-2 stage for the remaining factor), twiddles from a
// table built in double precision on the host.
#include "body_fft.cuh"

namespace ctpd {

// Hhat = DFT_P of the taps placed circularly (t[k] at k mod P).
__global__ void __launch_bounds__(FFT_T)
k_hhat(const float *__restrict__ taps, int half, int P, const float2 *__restrict__ tw, float2 *__restrict__ hhat)
{
    extern __shared__ float2 fsm[];
    float2 *a = fsm, *b = fsm + fft_elems(P);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        // index i holds t[k] with k = i (i < half) or k = i - P (i > P - half)
        float v = 0.0f;
        if (i < half) v = taps[half - 1 + i];
        else if (i > P - half) v = taps[half - 1 + (i - P)];
        a[fp(i)] = make_float2(v, 0.0f);
    }
    const float2 *res = fft_block(whole_block(), a, b, P, tw, false);
    for (int i = threadIdx.x; i < P; i += blockDim.x) hhat[i] = res[fp(i)];
}

void launch_hhat(const Geometry *g, const float *taps, int half, float2 *hhat, cudaStream_t st)
{
    const int P = g->n_fft;
    counted();
    k_hhat<<<1, FFT_T, sizeof(float2) * 2 * fft_elems(P), st>>>(taps, half, P, g->d_tw, hhat);
}

// out = post .* D(pre .* in) * sc, sc = 1 (mode 0) or -sigma (mode 1);
// one block per pair of views (v, v+1) of image `blockIdx.y`.  BANDS: the
// input is A x given as band partial sums (in = partial, nb bands), added
// in band order and scaled by the views' path lengths.
template <bool BANDS>
__global__ void __launch_bounds__(FFT_T)
k_filter_fft(const float2 *__restrict__ hhat, const float *__restrict__ in, float *__restrict__ out,
             const float *__restrict__ pre, const float *__restrict__ post, int mode,
             const double *__restrict__ scal, int V, int B, int P, const float2 *__restrict__ tw, int nb,
             const ViewP *__restrict__ views)
{
    extern __shared__ float2 fsm[];
    float2 *a = fsm, *b = fsm + fft_elems(P);
    const int v0 = 2 * blockIdx.x, v1 = v0 + 1;
    const bool has1 = v1 < V;
    const size_t base = (size_t)blockIdx.y * V * B;
    const size_t o0 = base + (size_t)v0 * B, o1 = base + (size_t)v1 * B;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        float x0 = 0.0f, x1 = 0.0f;
        if (i < B) {
            if (BANDS) {
                const size_t VB = (size_t)V * B;
                const float *p0 = in + (size_t)blockIdx.y * nb * VB + (size_t)v0 * B + i;
                const float *p1 = in + (size_t)blockIdx.y * nb * VB + (size_t)(has1 ? v1 : v0) * B + i;
                float s0, s1;
                band_sum2(p0, p1, VB, nb, s0, s1);
                x0 = s0 * views[v0].scale;
                x1 = has1 ? s1 * views[v1].scale : 0.0f;
            } else {
                x0 = in[o0 + i];
                if (pre) x0 *= pre[o0 + i];
                if (has1) {
                    x1 = in[o1 + i];
                    if (pre) x1 *= pre[o1 + i];
                }
            }
        }
        a[fp(i)] = make_float2(x0, x1);
    }
    // the response and the output scaling fused into the transforms' last stages
    auto mul_h = [&](int d, float2 v, float2 *dst) { dst[fp(d)] = cmul(v, hhat[d]); };
    float2 *f = fft_block_out(whole_block(), a, b, P, tw, false, mul_h);
    const float sc = ((mode == 1) ? -fscal(scal, F_SIGMA) : 1.0f) / (float)P;
    auto outp = [&](int d, float2 v, float2 *) {
        if (d < B) {
            float y0 = v.x * sc, y1 = v.y * sc;
            if (post) {
                y0 *= post[o0 + d];
                if (has1) y1 *= post[o1 + d];
            }
            out[o0 + d] = y0;
            if (has1) out[o1 + d] = y1;
        }
    };
    fft_block_out(whole_block(), f, f == a ? b : a, P, tw, true, outp);
}

// out = D (A x) from the projector's band partial sums
void launch_filter_fft_bands(const Geometry *g, const float2 *hhat, const float *partial, float *out, int batch,
                             cudaStream_t st)
{
    const int P = g->n_fft;
    dim3 grd((g->n_views + 1) / 2, batch);
    counted();
    k_filter_fft<true><<<grd, FFT_T, sizeof(float2) * 2 * fft_elems(P), st>>>(hhat, partial, out, nullptr, nullptr, 0, nullptr,
                                                                   g->n_views, g->n_bins, P, g->d_tw,
                                                                   proj_bands(g->n), g->d_views);
}

void launch_filter_fft(const Geometry *g, const float2 *hhat, const float *in, float *out,
                       const float *pre, const float *post, int mode, const double *scal, int batch,
                       cudaStream_t st)
{
    const int P = g->n_fft;
    dim3 grd((g->n_views + 1) / 2, batch);
    counted();
    k_filter_fft<false><<<grd, FFT_T, sizeof(float2) * 2 * fft_elems(P), st>>>(hhat, in, out, pre, post, mode, scal,
                                                                    g->n_views, g->n_bins, P, g->d_tw, 0, nullptr);
}

__global__ void __launch_bounds__(FFT_T, 4)
k_dual_fft(const float2 *__restrict__ hhat, const float *__restrict__ partial, int nb,
           const float *b, const float *mu_in, float *mu, float *mu_bar,
           const float *winv, int lowdose, const ViewP *__restrict__ views,
           const double *__restrict__ scal, int V, int B, int P, const float2 *__restrict__ tw)
{
    extern __shared__ float2 fsm[];
    pdl_wait();
    dual_fft_body(whole_block(), blockIdx.x, blockIdx.y, fsm, hhat, partial, nb, b, mu_in, mu, mu_bar, winv, lowdose,
                  views, scal, V, B, P, tw);
}

// =====================================================================
// The shift-variant preconditioner D = T_lo + S T_hi S (S = diag(s),
// s_i = sqrt(kappa w_i)): T_lo and T_hi are the convolutions with the taps
// of the low and high bands H_lo + H_hi = H of Eq. 24, so that D tends to
// the pure ramp of Eq. 32 at low frequency and to W at high frequency, the
// two limits of D = (tau A A^T + W^-1)^-1 (Eq. 23).  One view y per block:
// the real sequences y and S y travel as one complex sequence,
//     Z = FFT(y + i S y),  F y = (Z + conj Z(-k)) / 2,  F(S y) = (Z - conj Z(-k)) / 2i,
// and one inverse transform of
//     Y = H_lo F y + i H_hi F(S y) = hs Z + hd conj Z(-k),   hs, hd = (H_lo +- H_hi) / 2,
// returns u + i v with u = P T_lo y and v = P T_hi S y (both real, as
// H_lo and H_hi are Hermitian), so D y = (u + s v) / P.
// =====================================================================
__global__ void k_sv_combine(float2 *__restrict__ hs, float2 *__restrict__ hd, int P)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const float2 lo = hs[k], hi = hd[k];
    hs[k] = make_float2(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y));
    hd[k] = make_float2(0.5f * (lo.x - hi.x), 0.5f * (lo.y - hi.y));
}

void launch_sv_hhat(const Geometry *g, const float *taps_lo, const float *taps_hi, int half, float2 *hs, float2 *hd,
                    cudaStream_t st)
{
    launch_hhat(g, taps_lo, half, hs, st);
    launch_hhat(g, taps_hi, half, hd, st);
    counted();
    k_sv_combine<<<(g->n_fft + 255) / 256, 256, 0, st>>>(hs, hd, g->n_fft);
}

// Y(k) = hs(k) Z(k) + hd(k) conj Z(P-k), in place: each thread takes the pair (k, P-k)
__device__ __forceinline__ void sv_spectrum(float2 *f, const float2 *__restrict__ hs, const float2 *__restrict__ hd,
                                            int P)
{
    for (int k = threadIdx.x; k <= P / 2; k += blockDim.x) {
        const int k2 = (P - k) & (P - 1);
        const float2 z1 = f[fp(k)], z2 = f[fp(k2)];
        const float2 c1 = make_float2(z1.x, -z1.y), c2 = make_float2(z2.x, -z2.y);
        f[fp(k)] = cadd(cmul(hs[k], z1), cmul(hd[k], c2));
        if (k2 != k) f[fp(k2)] = cadd(cmul(hs[k2], z2), cmul(hd[k2], c1));
    }
}

// out = post .* D(pre .* in) * sc, sc = 1 (mode 0) or -sigma (mode 1), D the
// shift-variant form; one block per view v = blockIdx.x of image blockIdx.y.
// BANDS: the input is A x as the projector's nb band partial sums.
template <bool BANDS>
__global__ void __launch_bounds__(FFT_T)
k_filter_sv(const float2 *__restrict__ hs, const float2 *__restrict__ hd, const float *__restrict__ sv,
            const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ pre,
            const float *__restrict__ post, int mode, const double *__restrict__ scal, int V, int B, int P,
            const float2 *__restrict__ tw, int nb, const ViewP *__restrict__ views)
{
    extern __shared__ float2 fsm[];
    float2 *a = fsm, *b = fsm + fft_elems(P);
    const int v = blockIdx.x;
    const size_t VB = (size_t)V * B;
    const size_t o = (size_t)blockIdx.y * VB + (size_t)v * B;
    const float *s = sv + (size_t)v * B;   // the weights, so S, are one slice's
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        float y = 0.0f, sy = 0.0f;
        if (i < B) {
            if (BANDS) {
                const float *pp = in + (size_t)blockIdx.y * nb * VB + (size_t)v * B + i;
                float acc = 0.0f;
                for (int q = 0; q < nb; ++q) acc += pp[q * VB];
                y = acc * views[v].scale;
            } else {
                y = in[o + i];
                if (pre) y *= pre[o + i];
            }
            sy = s[i] * y;
        }
        a[fp(i)] = make_float2(y, sy);
    }
    float2 *f = fft_block(whole_block(), a, b, P, tw, false);
    sv_spectrum(f, hs, hd, P);
    const float sc = ((mode == 1) ? -fscal(scal, F_SIGMA) : 1.0f) / (float)P;
    auto outp = [&](int d, float2 uv, float2 *) {   // fused into the inverse transform's last stage
        if (d < B) {
            float y = fmaf(s[d], uv.y, uv.x) * sc;
            if (post) y *= post[o + d];
            out[o + d] = y;
        }
    };
    fft_block_out(whole_block(), f, f == a ? b : a, P, tw, true, outp);
}

void launch_filter_sv(const Geometry *g, const float2 *hs, const float2 *hd, const float *sv, const float *in,
                      float *out, const float *pre, const float *post, int mode, const double *scal, int batch,
                      cudaStream_t st)
{
    counted();
    k_filter_sv<false><<<dim3(g->n_views, batch), FFT_T, sizeof(float2) * 2 * fft_elems(g->n_fft), st>>>(
        hs, hd, sv, in, out, pre, post, mode, scal, g->n_views, g->n_bins, g->n_fft, g->d_tw, 0, nullptr);
}

void launch_filter_sv_bands(const Geometry *g, const float2 *hs, const float2 *hd, const float *sv,
                            const float *partial, float *out, int batch, cudaStream_t st)
{
    counted();
    k_filter_sv<true><<<dim3(g->n_views, batch), FFT_T, sizeof(float2) * 2 * fft_elems(g->n_fft), st>>>(
        hs, hd, sv, partial, out, nullptr, nullptr, 0, nullptr, g->n_views, g->n_bins, g->n_fft, g->d_tw,
        proj_bands(g->n), g->d_views);
}

// Fused Step 3 and next Step 1 of Algorithm 1 with the shift-variant D, one
// view per block (the form of k_dual_fft):
//   r = scale_v sum_b partial[b] - b - winv mu;  mu' = mu + sigma D r;
//   mubar = 2 mu' - mu - sigma D (winv .* (mu' - mu)).
__global__ void __launch_bounds__(FFT_T)
k_dual_sv(const float2 *__restrict__ hs, const float2 *__restrict__ hd, const float *__restrict__ sv,
          const float *__restrict__ partial, int nb, const float *__restrict__ b, float *mu,
          float *__restrict__ mu_bar, const float *__restrict__ winv, const ViewP *__restrict__ views,
          const double *__restrict__ scal, int V, int B, int P, const float2 *__restrict__ tw)
{
    extern __shared__ float2 fsm[];
    float2 *a = fsm, *bb = fsm + fft_elems(P);
    float *m_old = reinterpret_cast<float *>(fsm + 2 * fft_elems(P));   // B
    float *m_new = m_old + B;                                          // B
    const int v = blockIdx.x;
    const size_t VB = (size_t)V * B, o = (size_t)v * B;
    const float *s = sv + o;
    const float sc = views[v].scale;
    const float sigma = fscal(scal, F_SIGMA);
    const float invP = 1.0f / (float)P;

    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        float r = 0.0f, sr = 0.0f;
        if (i < B) {
            const float *pp = partial + o + i;
            float acc = 0.0f;
            for (int q = 0; q < nb; ++q) acc += pp[q * VB];
            const float m0 = mu[o + i];
            m_old[i] = m0;
            r = acc * sc - b[o + i] - winv[o + i] * m0;
            sr = s[i] * r;
        }
        a[fp(i)] = make_float2(r, sr);
    }
    float2 *f = fft_block(whole_block(), a, bb, P, tw, false);
    sv_spectrum(f, hs, hd, P);
    // the dual update fused into the inverse transform's last stage, which
    // also stages the second filter's input (d, s d) in the buffer it writes
    auto upd = [&](int i, float2 uv, float2 *dst) {
        float d = 0.0f, sd = 0.0f;
        if (i < B) {
            const float n0 = m_old[i] + sigma * (fmaf(s[i], uv.y, uv.x) * invP);
            m_new[i] = n0;
            d = winv[o + i] * (n0 - m_old[i]);
            sd = s[i] * d;
        }
        dst[fp(i)] = make_float2(d, sd);
    };
    f = fft_block_out(whole_block(), f, f == a ? bb : a, P, tw, true, upd);
    f = fft_block(whole_block(), f, f == a ? bb : a, P, tw, false);
    sv_spectrum(f, hs, hd, P);
    auto fin = [&](int i, float2 uv, float2 *) {
        if (i < B) {
            const float n0 = m_new[i];
            mu[o + i] = n0;
            mu_bar[o + i] = 2.0f * n0 - m_old[i] - sigma * (fmaf(s[i], uv.y, uv.x) * invP);
        }
    };
    fft_block_out(whole_block(), f, f == a ? bb : a, P, tw, true, fin);
}

void launch_dual_sv(const Geometry *g, const float2 *hs, const float2 *hd, const float *sv, const float *partial,
                    const float *b, float *mu, float *mu_bar, const float *winv, const double *scal,
                    cudaStream_t st)
{
    counted();
    const size_t smem = sizeof(float2) * 2 * fft_elems(g->n_fft) + sizeof(float) * 2 * g->n_bins;
    k_dual_sv<<<g->n_views, FFT_T, smem, st>>>(hs, hd, sv, partial, proj_bands(g->n), b, mu, mu_bar, winv,
                                               g->d_views, scal, g->n_views, g->n_bins, g->n_fft, g->d_tw);
}

size_t dual_fft_smem(const Geometry *g) { return sizeof(float2) * 2 * fft_elems(g->n_fft) + sizeof(float) * 4 * g->n_bins; }

void launch_dual_fft(const Geometry *g, const float2 *hhat, const float *partial, const float *b, float *mu,
                     float *mu_bar, const float *winv, int lowdose, const double *scal, cudaStream_t st)
{
    launch_dual_fft_batched(g, hhat, partial, b, mu, mu, mu_bar, winv, lowdose, scal, 1, st);
}

void launch_dual_fft_batched(const Geometry *g, const float2 *hhat, const float *partial, const float *b,
                             const float *mu_in, float *mu_out, float *mu_bar, const float *winv, int lowdose,
                             const double *scal, int batch, cudaStream_t st)
{
    counted();
    launch_kernel(k_dual_fft, dim3((g->n_views + 1) / 2, batch), dim3(FFT_T), dual_fft_smem(g), st, hhat, partial,
                  proj_bands(g->n), b, mu_in, mu_out, mu_bar, winv, lowdose, g->d_views, scal, g->n_views, g->n_bins,
                  g->n_fft, g->d_tw);
}

// Adjoint of one dual step (Step 3 and the next Step 1) for the pair of
// views (v, v+1) of slice blockIdx.y.  Forward (W = diag(winv), low-dose):
//   r      = A x' - b - W mu
//   mu'    = mu + sigma D r
//   mubar' = 2 mu' - mu - sigma D W (mu' - mu)
// Given gm = dL/dmu' and gmb = dL/dmubar', with D^T applied through the
// conjugate response:
//   h   = D^T gmb
//   gm1 = gm + 2 gmb - sigma W h          (total dL/dmu')
//   gr  = sigma D^T gm1                   (dL/dr)
//   gmu = gm1 - W gr - gmb + sigma W h    (dL/dmu)
// and writes r and v = W (mu' - mu) for the tap correlations
// dL/dt += sigma (gm1 * r) - sigma (gmb * v).  Few-view drops every W term.
__global__ void __launch_bounds__(FFT_T)
k_dual_bwd_fft(const float2 *__restrict__ hhat, const float *__restrict__ partial, int nb,
               const float *__restrict__ b, const float *__restrict__ winv, const float *__restrict__ mu,
               const float *__restrict__ mu1, const float *__restrict__ gm, const float *__restrict__ gmb,
               float *__restrict__ gmu_out, float *__restrict__ gr_out, float *__restrict__ gm1_out,
               float *__restrict__ r_out, float *__restrict__ v_out, int lowdose,
               const ViewP *__restrict__ views, const double *__restrict__ scal, int V, int B, int P,
               const float2 *__restrict__ tw)
{
    extern __shared__ float2 fsm[];
    float2 *a = fsm, *bb = fsm + fft_elems(P);
    float *h_s = reinterpret_cast<float *>(fsm + 2 * fft_elems(P));   // 2 x B: D^T gmb
    float *g1_s = h_s + 2 * B;                             // 2 x B: gm1
    const size_t so = (size_t)blockIdx.y * V * B;
    partial += (size_t)blockIdx.y * nb * V * B;
    const int v0 = 2 * blockIdx.x, v1 = v0 + 1;
    const bool has1 = v1 < V;
    const size_t VB = (size_t)V * B;
    const size_t o0 = so + (size_t)v0 * B, o1 = so + (size_t)(has1 ? v1 : v0) * B;
    const float sigma = fscal(scal, F_SIGMA);
    const float invP = 1.0f / (float)P;

    // h = D^T gmb
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        a[fp(i)] = i < B ? make_float2(gmb[o0 + i], has1 ? gmb[o1 + i] : 0.0f) : make_float2(0.0f, 0.0f);
    float2 *f = fft_block(whole_block(), a, bb, P, tw, false);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float2 h = hhat[i];
        f[fp(i)] = cmul(f[fp(i)], make_float2(h.x, -h.y));
    }
    float2 *res = fft_block(whole_block(), f, f == a ? bb : a, P, tw, true);
    float2 *other = res == a ? bb : a;
    // gm1 = gm + 2 gmb - sigma W h ; stage gm1 for D^T
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        float g0 = 0.0f, g1v = 0.0f;
        if (i < B) {
            const float h0 = res[fp(i)].x * invP, h1 = res[fp(i)].y * invP;
            h_s[i] = h0;
            h_s[B + i] = h1;
            g0 = gm[o0 + i] + 2.0f * gmb[o0 + i];
            g1v = has1 ? gm[o1 + i] + 2.0f * gmb[o1 + i] : 0.0f;
            if (lowdose) {
                g0 -= sigma * winv[o0 + i] * h0;
                if (has1) g1v -= sigma * winv[o1 + i] * h1;
            }
            g1_s[i] = g0;
            g1_s[B + i] = g1v;
        }
        other[fp(i)] = make_float2(g0, g1v);
    }
    f = fft_block(whole_block(), other, res, P, tw, false);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float2 h = hhat[i];
        f[fp(i)] = cmul(f[fp(i)], make_float2(h.x, -h.y));
    }
    res = fft_block(whole_block(), f, f == a ? bb : a, P, tw, true);
    const float sc0 = views[v0].scale, sc1 = has1 ? views[v1].scale : 0.0f;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        // two views: k = 0 -> v0, k = 1 -> v1
        for (int k = 0; k < (has1 ? 2 : 1); ++k) {
            const size_t o = (k == 0 ? o0 : o1) + i;
            const float gr = sigma * ((k == 0 ? res[fp(i)].x : res[fp(i)].y) * invP);
            const float g1v = g1_s[k * B + i], hv = h_s[k * B + i];
            float gmu = g1v - gmb[o];
            float acc = 0.0f;
            const float *pp = partial + (o - so);
            for (int q = 0; q < nb; ++q) acc += pp[q * VB];
            float r = acc * (k == 0 ? sc0 : sc1) - b[o];
            float vv = 0.0f;
            if (lowdose) {
                gmu += -winv[o] * gr + sigma * winv[o] * hv;
                r -= winv[o] * mu[o];
                vv = winv[o] * (mu1[o] - mu[o]);
            }
            gmu_out[o] = gmu;
            gr_out[o] = gr;
            gm1_out[o] = g1v;
            r_out[o] = r;
            v_out[o] = vv;
        }
    }
}

size_t dual_bwd_smem(const Geometry *g) { return sizeof(float2) * 2 * fft_elems(g->n_fft) + sizeof(float) * 4 * g->n_bins; }

void launch_dual_bwd_fft(const Geometry *g, const float2 *hhat, const float *partial, const float *b,
                         const float *winv, const float *mu, const float *mu1, const float *gm, const float *gmb,
                         float *gmu, float *gr, float *gm1, float *r, float *v, int lowdose, const double *scal,
                         int batch, cudaStream_t st)
{
    counted();
    k_dual_bwd_fft<<<dim3((g->n_views + 1) / 2, batch), FFT_T, dual_bwd_smem(g), st>>>(
        hhat, partial, proj_bands(g->n), b, winv, mu, mu1, gm, gmb, gmu, gr, gm1, r, v, lowdose, g->d_views,
        scal, g->n_views, g->n_bins, g->n_fft, g->d_tw);
}

bool fft_supported(const Geometry *g) { return g->n_fft <= FFT_MAX_P; }

void kernel_attrs_fft()
{
    const int smax = (int)(sizeof(float2) * 2 * fft_elems(FFT_MAX_P) + sizeof(float) * 4 * (FFT_MAX_P / 2));
    cudaFuncSetAttribute(k_hhat, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_filter_fft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_filter_fft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_dual_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_dual_bwd_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_filter_sv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_filter_sv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_dual_sv, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
}

}  // namespace ctpd
