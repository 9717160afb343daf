// body_fft.cuh -- shared-memory FFT building blocks of the frequency-domain
// preconditioner D (k_fft.cu) and the body of the fused dual step, shared by
// its kernel and the persistent batched kernel (persist.cu).
//
// D applies, along the detector of every view, the linear (zero-padded)
// convolution with the taps t[k], |k| < half.  With the view zero-padded to
// the period P >= 2B, the circular convolution with the taps placed at k
// mod P equals that linear convolution on bins 0..B-1, so D =
// IFFT_P(Hhat . FFT_P(.)) with Hhat the P-point DFT of the circularly placed
// taps.  FFTs run in shared memory as Stockham autosort stages (radix 8, then
// a radix-4 or radix-2 stage for the remaining factor), twiddles from a table
// built in double precision on the host.  A BlockCtx names the threads that
// run one transform (a whole block, or a group of a persistent block).
#pragma once

#include "ctpd_internal.cuh"

namespace ctpd {

constexpr int FFT_T = 256;    // threads per block

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ float2 rot(float2 a, bool inv) { return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }

__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3, bool inv)
{
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = rot(csub(a1, a3), inv);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

__device__ __forceinline__ void dft8(float2 *v, bool inv)
{
    // even / odd 4-point DFTs, then the radix-2 combination with w8^k
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3, inv);
    dft4(o0, o1, o2, o3, inv);
    const float c = 0.70710678118654752440f;
    // w8^1 = c(1 -+ i), w8^2 = -+i, w8^3 = c(-1 -+ i)
    const float2 w1o = inv ? make_float2(c * (o1.x - o1.y), c * (o1.x + o1.y))
                           : make_float2(c * (o1.x + o1.y), c * (o1.y - o1.x));
    const float2 w2o = rot(o2, inv);
    const float2 w3o = inv ? make_float2(-c * (o3.x + o3.y), c * (o3.x - o3.y))
                           : make_float2(c * (o3.y - o3.x), -c * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1o);
    v[5] = csub(e1, w1o);
    v[2] = cadd(e2, w2o);
    v[6] = csub(e2, w2o);
    v[3] = cadd(e3, w3o);
    v[7] = csub(e3, w3o);
}

// Shared-memory FFT buffers hold element i at fp(i) = i + i/16: one pad slot
// per 16 elements makes the strided stores of the first stages (stride R
// and R Ns) and the contiguous loads free of bank conflicts.
__host__ __device__ __forceinline__ int fp(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int fft_elems(int P) { return P + (P >> 4); }

// One radix-R Stockham stage: butterfly j reads src[j + r P/R], applies the
// twiddles w^(r k P/(Ns R)) (k = j mod Ns) and writes dst[(j - k) R + k + r Ns].
template <int R, class Ctx>
__device__ __forceinline__ void fft_stage(const Ctx &c, const float2 *src, float2 *dst, int P, int Ns,
                                          const float2 *__restrict__ tw, bool inv)
{
    const int nb = P / R;
    for (int j = c.tid(); j < nb; j += c.nth()) {
        float2 v[R];
        const int k = j & (Ns - 1);
        const int step = (P / (Ns * R)) * k;
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[fp(j + r * nb)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(tw + r * step);
                if (inv) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (R == 8) dft8(v, inv);
        else if (R == 4) dft4(v[0], v[1], v[2], v[3], inv);
        else dft2(v[0], v[1]);
        const int d0 = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[fp(d0 + r * Ns)] = v[r];
    }
}

// Unnormalised DFT (forward: e^{-2 pi i jk/P}; inverse: e^{+...}) of the P
// values in a; b is scratch.  Returns the buffer holding the result.  All
// threads of the block (context c) must call it; it synchronises between
// stages.
template <class Ctx>
__device__ __noinline__ float2 *fft_block(const Ctx &c, float2 *a, float2 *b, int P,
                                                 const float2 *__restrict__ tw, bool inv)
{
    int Ns = 1;
    float2 *src = a, *dst = b;
    while (Ns < P) {
        const int rem = P / Ns;
        c.sync();
        if (rem >= 8) {
            fft_stage<8>(c, src, dst, P, Ns, tw, inv);
            Ns *= 8;
        } else if (rem == 4) {
            fft_stage<4>(c, src, dst, P, Ns, tw, inv);
            Ns *= 4;
        } else {
            fft_stage<2>(c, src, dst, P, Ns, tw, inv);
            Ns *= 2;
        }
        float2 *t = src;
        src = dst;
        dst = t;
    }
    c.sync();
    return src;
}

// fft_block with the work that follows the transform fused into its last
// stage: instead of storing output d, the last stage calls
// store(d, value, dst), dst being the buffer it would have written, which
// the call returns.  This saves one pass over shared memory and one block
// barrier per transform.
template <int R, class Store, class Ctx>
__device__ __forceinline__ void fft_stage_last(const Ctx &c, const float2 *src, float2 *dst, int P, int Ns,
                                               const float2 *__restrict__ tw, bool inv, Store store)
{
    const int nb = P / R;
    for (int j = c.tid(); j < nb; j += c.nth()) {
        float2 v[R];
        const int k = j & (Ns - 1);
        const int step = (P / (Ns * R)) * k;
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[fp(j + r * nb)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(tw + r * step);
                if (inv) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (R == 8) dft8(v, inv);
        else if (R == 4) dft4(v[0], v[1], v[2], v[3], inv);
        else dft2(v[0], v[1]);
        const int d0 = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) store(d0 + r * Ns, v[r], dst);
    }
}

template <class Store, class Ctx>
__device__ __forceinline__ float2 *fft_block_out(const Ctx &c, float2 *a, float2 *b, int P,
                                                 const float2 *__restrict__ tw, bool inv, Store store)
{
    int Ns = 1;
    float2 *src = a, *dst = b;
    while (Ns < P) {
        const int rem = P / Ns;
        const int R = rem >= 8 ? 8 : (rem == 4 ? 4 : 2);
        c.sync();
        if (Ns * R == P) {
            if (R == 8) fft_stage_last<8>(c, src, dst, P, Ns, tw, inv, store);
            else if (R == 4) fft_stage_last<4>(c, src, dst, P, Ns, tw, inv, store);
            else fft_stage_last<2>(c, src, dst, P, Ns, tw, inv, store);
        } else {
            if (R == 8) fft_stage<8>(c, src, dst, P, Ns, tw, inv);
            else if (R == 4) fft_stage<4>(c, src, dst, P, Ns, tw, inv);
            else fft_stage<2>(c, src, dst, P, Ns, tw, inv);
        }
        float2 *t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    c.sync();
    return src;
}

// Band partial sums of A x for two rays (p0[k VB], p1[k VB], k < nb),
// added in band order; the loads of 16 bands are issued together.
__device__ __forceinline__ void band_sum2(const float *__restrict__ p0, const float *__restrict__ p1, size_t VB,
                                          int nb, float &s0, float &s1)
{
    s0 = 0.0f;
    s1 = 0.0f;
    for (int kb = 0; kb < nb; kb += 16) {
        float a[16], c[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const bool ok = kb + k < nb;
            a[k] = ok ? p0[(size_t)(kb + k) * VB] : 0.0f;
            c[k] = ok ? p1[(size_t)(kb + k) * VB] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (kb + k < nb) {
                s0 += a[k];
                s1 += c[k];
            }
        }
    }
}

// Fused Step 3 and next Step 1 for the pair of views (v, v+1):
//   r     = scale_v sum_b partial[b] - b [- winv mu]     (A x^{k+1} - b [- W^-1 mu^k])
//   mu'   = mu + sigma D r                               (Step 3)
//   mubar = 2 mu' - mu [- sigma D (winv .* (mu' - mu))]  (Step 1, Alg. 1 / Alg. 2)
// Block (context c) `bx` handles views (2 bx, 2 bx + 1) of slice `by` of a
// batch; fsm: shared memory of dual_fft_smem bytes.
template <class Ctx>
__device__ __forceinline__ void dual_fft_body(const Ctx &c, int bx, int by, float2 *fsm, const float2 *hhat,
                                              const float *partial, int nb, const float *b, const float *mu_in,
                                              float *mu, float *mu_bar, const float *winv, int lowdose,
                                              const ViewP *views, const double *scal, int V, int B, int P,
                                              const float2 *tw)
{
    // mu_in may equal mu (each block reads its two views completely before
    // writing them)
    {
        const size_t so = (size_t)by * V * B;
        partial += (size_t)by * nb * V * B;
        b += so;
        mu_in += so;
        mu += so;
        mu_bar += so;
        if (winv) winv += so;
    }
    float2 *a = fsm, *bb = fsm + fft_elems(P);
    float *m_old = reinterpret_cast<float *>(fsm + 2 * fft_elems(P));   // 2 x B
    float *m_new = m_old + 2 * B;                            // 2 x B
    const int v0 = 2 * bx, v1 = v0 + 1;
    const bool has1 = v1 < V;
    const size_t VB = (size_t)V * B;
    const size_t o0 = (size_t)v0 * B, o1 = (size_t)v1 * B;
    const float sc0 = views[v0].scale, sc1 = has1 ? views[v1].scale : 0.0f;
    const float sigma = fscal(scal, F_SIGMA);
    const float invP = 1.0f / (float)P;

    for (int i = c.tid(); i < P; i += c.nth()) {
        float r0 = 0.0f, r1 = 0.0f;
        if (i < B) {
            // band partial sums of A x, added in band order
            float s0, s1;
            band_sum2(partial + o0 + i, partial + (has1 ? o1 : o0) + i, VB, nb, s0, s1);
            if (!has1) s1 = 0.0f;
            const float mu0 = mu_in[o0 + i], mu1 = has1 ? mu_in[o1 + i] : 0.0f;
            m_old[i] = mu0;
            m_old[B + i] = mu1;
            r0 = s0 * sc0 - b[o0 + i];
            if (lowdose) r0 -= winv[o0 + i] * mu0;
            if (has1) {
                r1 = s1 * sc1 - b[o1 + i];
                if (lowdose) r1 -= winv[o1 + i] * mu1;
            }
        }
        a[fp(i)] = make_float2(r0, r1);
    }
    // D r: forward transform with the response fused into its last stage,
    // inverse transform with the dual update fused into its last stage
    // (which also stages the second filter's input in the buffer it writes)
    auto mul_h = [&](int d, float2 v, float2 *dst) { dst[fp(d)] = cmul(v, hhat[d]); };
    float2 *f = fft_block_out(c, a, bb, P, tw, false, mul_h);   // H . FFT(r), in f
    auto upd = [&](int d, float2 v, float2 *dst) {
        float d0 = 0.0f, d1 = 0.0f;
        if (d < B) {
            const float n0 = m_old[d] + sigma * (v.x * invP);
            const float n1 = m_old[B + d] + sigma * (v.y * invP);
            if (lowdose) {
                m_new[d] = n0;
                m_new[B + d] = n1;
                d0 = winv[o0 + d] * (n0 - m_old[d]);
                if (has1) d1 = winv[o1 + d] * (n1 - m_old[B + d]);
            } else {
                // Alg. 2: mu_bar = 2 mu' - mu, no second filter
                mu[o0 + d] = n0;
                mu_bar[o0 + d] = 2.0f * n0 - m_old[d];
                if (has1) {
                    mu[o1 + d] = n1;
                    mu_bar[o1 + d] = 2.0f * n1 - m_old[B + d];
                }
            }
        }
        if (lowdose) dst[fp(d)] = make_float2(d0, d1);
    };
    f = fft_block_out(c, f, f == a ? bb : a, P, tw, true, upd);   // the second filter's input, in f
    if (!lowdose) return;
    f = fft_block_out(c, f, f == a ? bb : a, P, tw, false, mul_h);
    auto fin = [&](int d, float2 v, float2 *) {
        if (d < B) {
            const float n0 = m_new[d], n1 = m_new[B + d];
            mu[o0 + d] = n0;
            mu_bar[o0 + d] = 2.0f * n0 - m_old[d] - sigma * (v.x * invP);
            if (has1) {
                mu[o1 + d] = n1;
                mu_bar[o1 + d] = 2.0f * n1 - m_old[B + d] - sigma * (v.y * invP);
            }
        }
    };
    fft_block_out(c, f, f == a ? bb : a, P, tw, true, fin);
}

}  // namespace ctpd
