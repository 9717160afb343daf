// k_grad.cu -- reductions used by the adjoint of the unrolled solve.
#include <algorithm>

#include "ctpd_internal.cuh"

namespace ctpd {

// Tap correlations of the adjoint: the derivative of sum_p c_p <g_p, D s_p>
// with respect to the tap t[k] of D (out[d] = sum_e t[d - e] in[e]) is
// sum_p c_p sum_v sum_d g_p[v][d] s_p[v][d - k], |k| < half.
//
// One warp per (view, pair): the two rows are staged zero-padded in shared
// memory and lane l owns eight consecutive lags of a pass of 256.  The lane
// walks the bins with a register window of the eight s values its lags
// need, so each step loads one s and one g value for eight FMAs; lane l runs
// l / 4 bins ahead of lane 0, which puts the 32 lanes' s loads in 32
// different banks and their g loads in eight consecutive words.  A block
// adds its warps' results in order into partial[lag][block] (float);
// k_tapcorr_sum adds the blocks in order (compensated FP32).
constexpr int TC_PASS = 256;                  // lags per pass: 32 lanes x 8
constexpr int TC_MAXW = 8;                    // warps per block
constexpr int TC_SMEM = 112 * 1024;           // dynamic shared memory bound per block

struct TcPlan {
    int nl, npass, nlp, l8, off, ng, ns, wfl, nw;
};

// l8: loop steps (bins + 7 of lead, rounded to 8); off: the s row's zero
// padding in front; ng, ns: staged lengths; wfl: floats per warp (rows and
// the warp's results); nw: warps per block within TC_SMEM.
TcPlan tc_plan(int B, int half)
{
    TcPlan p;
    p.nl = 2 * half - 1;
    p.npass = (p.nl + TC_PASS - 1) / TC_PASS;
    p.nlp = p.npass * TC_PASS;
    p.l8 = (B + 7 + 7) / 8 * 8;
    p.off = 7 + p.nlp - half;
    p.ng = p.l8 + 8;
    p.ns = p.l8 + p.nlp + 8;
    p.wfl = p.ng + p.ns + p.nlp;
    p.nw = std::max(1, std::min(TC_MAXW, TC_SMEM / (int)(sizeof(float) * p.wfl)));
    return p;
}

__global__ void __launch_bounds__(TC_MAXW * 32)
k_tapcorr(const float *__restrict__ g0, const float *__restrict__ s0, float c0, const float *__restrict__ g1,
          const float *__restrict__ s1, float c1, int npairs, int nviews, int B, int half, TcPlan pl,
          float *__restrict__ partial)
{
    extern __shared__ float sm[];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    float *G = sm + (size_t)w * pl.wfl, *S = G + pl.ng, *res = S + pl.ns;
    const int u = blockIdx.x * nw + w, v = u / npairs, pr = u - v * npairs;
    if (v < nviews) {
        const float *gr = (pr == 0 ? g0 : g1) + (size_t)v * B, *sr = (pr == 0 ? s0 : s1) + (size_t)v * B;
        const float c = pr == 0 ? c0 : c1;
        for (int t = l; t < pl.ng; t += 32) G[t] = (t >= 7 && t - 7 < B) ? gr[t - 7] : 0.0f;
        for (int t = l; t < pl.ns; t += 32) S[t] = (t >= pl.off && t - pl.off < B) ? sr[t - pl.off] : 0.0f;
        __syncwarp();
        const int lead = l >> 2;
        const float *Gl = G + lead;
        for (int pass = 0; pass < pl.npass; ++pass) {
            const int k0 = pass * TC_PASS + 8 * l - (half - 1);
            const float *Sl = S + (pl.off - 7 + lead - k0);   // Sl[m] = s[d - k0] at bin d = m - 7 + lead
            float R[8], a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                a[j] = 0.0f;
                R[j] = j > 0 ? Sl[j - 8] : 0.0f;
            }
            for (int i = 0; i < pl.l8; i += 8) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    R[q] = Sl[i + q];
                    const float gv = Gl[i + q];
#pragma unroll
                    for (int j = 0; j < 8; ++j) a[j] = fmaf(gv, R[(q - j) & 7], a[j]);   // s[d - k0 - j]
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) res[pass * TC_PASS + 8 * l + j] = c * a[j];
        }
    } else {
        for (int t = l; t < pl.nlp; t += 32) res[t] = 0.0f;
    }
    __syncthreads();
    for (int li = threadIdx.x; li < pl.nl; li += blockDim.x) {
        float t = 0.0f;
        for (int k = 0; k < nw; ++k) t += sm[(size_t)k * pl.wfl + pl.ng + pl.ns + li];
        partial[(size_t)li * gridDim.x + blockIdx.x] = t;
    }
}

// acc[lag] += sum over blocks of partial[lag][block]: one warp per lag,
// lanes over strided blocks, then a fixed shuffle tree, all in compensated
// FP32 (acc holds value x + y)
__global__ void k_tapcorr_sum(const float *__restrict__ partial, int nblocks, int nl, float2 *__restrict__ acc)
{
    const int lag = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), l = threadIdx.x & 31;
    if (lag >= nl) return;
    const float *p = partial + (size_t)lag * nblocks;
    FSum t{0.0f, 0.0f};
    for (int b = l; b < nblocks; b += 32) fsum_add(t, p[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const FSum u{__shfl_down_sync(0xffffffffu, t.s, o), __shfl_down_sync(0xffffffffu, t.c, o)};
        fsum_merge(t, u);
    }
    if (l == 0) {
        FSum a{acc[lag].x, acc[lag].y};
        fsum_merge(a, t);
        acc[lag] = make_float2(a.s, a.c);
    }
}

size_t tapcorr_partial_bytes(int nviews, int B, int half)
{
    const TcPlan pl = tc_plan(B, half);
    const size_t nb = ((size_t)2 * nviews + pl.nw - 1) / pl.nw;
    return sizeof(float) * (size_t)pl.nl * nb;
}

void launch_tapcorr_acc(const float *g0, const float *s0, double c0, const float *g1, const float *s1, double c1,
                        int nviews, int B, int half, float *partial, float2 *acc, cudaStream_t st)
{
    const TcPlan pl = tc_plan(B, half);
    const int npairs = g1 ? 2 : 1;
    const int nb = (int)(((size_t)npairs * nviews + pl.nw - 1) / pl.nw);
    counted(2);
    k_tapcorr<<<nb, pl.nw * 32, sizeof(float) * (size_t)pl.nw * pl.wfl, st>>>(
        g0, s0, (float)c0, g1, s1, (float)c1, npairs, nviews, B, half, pl, partial);
    k_tapcorr_sum<<<(pl.nl + 7) / 8, 256, 0, st>>>(partial, nb, pl.nl, acc);
}

void kernel_attrs_grad() { cudaFuncSetAttribute(k_tapcorr, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM); }

// grad[0 .. nl) = the compensated tap accumulators; grad[nl] = scal[slot] * fac
// (one thread's scalar arithmetic)
__global__ void k_grad_out(const float2 *__restrict__ acc, int nl, const double *__restrict__ scal, int slot,
                           double fac, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nl) grad[i] = acc[i].x + acc[i].y;
    if (i == nl) grad[nl] = (float)(scal[slot] * fac);
}

void launch_grad_out(const float2 *acc, int nl, const double *scal, int slot, double fac, float *grad,
                     cudaStream_t st)
{
    counted();
    k_grad_out<<<(nl + 1 + 127) / 128, 128, 0, st>>>(acc, nl, scal, slot, fac, grad);
}

}  // namespace ctpd
