// body_joseph.cuh -- bodies of the Joseph projector (view pairs and mirrored
// bands) and of the rotation-orbit backprojector, shared by their kernels
// (k_joseph.cu) and the persistent batched kernel (persist.cu).  Each body
// takes its block index and shared memory explicitly and runs on the
// threads of a context (a whole block or a group of a persistent block).
#pragma once

#include "ctpd_internal.cuh"

namespace ctpd {

__device__ __forceinline__ float joseph_h(int n) { return 0.5f * (float)(n - 1); }
__device__ __forceinline__ float joseph_dp(int d, int B) { return __fsub_rn((float)d, 0.5f * (float)(B - 1)); }

constexpr int PG = 16;         // views per block
constexpr int MR = 16;         // steps per band (two bands per block)

// Conservative integer range [lo, hi] within [s_lo, s_hi] of the steps s
// for which u'(s) = q + (s - h) m can lie in [ulo, uhi] (empty if lo > hi).
__device__ __forceinline__ void step_range(float q, float m, float inv_m, float h, float ulo, float uhi,
                                           int s_lo, int s_hi, int &lo, int &hi)
{
    if (m == 0.0f) {
        lo = s_lo;
        hi = (q >= ulo && q <= uhi) ? s_hi : s_lo - 1;
        return;
    }
    // explicit roundings: every kernel that walks a ray finds the same range
    float sa = __fmaf_rn(__fsub_rn(ulo, q), inv_m, h), sb = __fmaf_rn(__fsub_rn(uhi, q), inv_m, h);
    float smin = fminf(sa, sb), smax = fmaxf(sa, sb);
    // clamp before converting: far-off rays give huge (or infinite) s
    smin = fminf(fmaxf(smin, (float)s_lo - 2.0f), (float)s_hi + 2.0f);
    smax = fminf(fmaxf(smax, (float)s_lo - 2.0f), (float)s_hi + 2.0f);
    lo = max(s_lo, (int)floorf(smin) - 1);
    hi = min(s_hi, (int)ceilf(smax) + 1);
}

// Shared memory of the view-pair projector's block at image side N.
__host__ __device__ __forceinline__ size_t quad_smem(int N) { return sizeof(float2) * (size_t)2 * MR * ((N + 3) | 1); }

// ---------------------------------------------------------------------
// Forward projection with the detector mirror and the view mirror (default
// angles t_v = v pi / V).  View V-v is view v reflected in the image's
// vertical axis: its a and m are those of view v with the signs a row view
// (a -> -a, m -> -m) or a column view (m -> -m) gets from t -> pi - t.
// For a row view that puts ray d of view V-v at coordinate N-1-u on the
// same row; for a column view ray d of view V-v meets column N-1-c where
// ray d of view v meets column c, i.e. the other band's line.  Either way
// the reflected sample sits at pair N-2-i0 of a staged line with weight
// -g: one evaluation of (u', g) at (d, s) yields four samples, two of view
// v (bands A, B as in k_project_mirror) and two of view V-v:
//     rows:    A[i0] (v, d)  B[i0] (v, B-1-d)  A[N-2-i0] (V-v, d)    B[N-2-i0] (V-v, B-1-d)
//     columns: A[i0] (v, d)  B[i0] (v, B-1-d)  A[N-2-i0] (V-v, B-1-d) B[N-2-i0] (V-v, d)
// Work items are view pairs (v, V-v) and the views without a partner
// (v = 0, and v = V/2 for even V), pg items per block, 64 threads per item.
// ---------------------------------------------------------------------
// Walks one ray through the staged steps lo..hi (ROWS steps per pass, one
// coordinate evaluation per step) and returns its four sums: band A and
// band B at the pair i0, and (PAIR) at the reflected pair N-2-i0.  Q holds
// per step and pair (A mid, B mid, A delta, B delta), so one 16-byte load
// serves both bands and the two bands' samples are one packed two-wide
// FMA, mid + g delta, into a pair accumulator (the reflected pair with -g).
// The coordinates of two steps are evaluated as one packed pair as well.
// A pass of ROWS = 4 is two passes of ROWS = 2 whose loads are issued
// together: the same coordinates (u' = (s - h) m + q for even steps,
// (s - 1 - h) m + (q + m) for odd ones), the same two accumulators (even
// and odd steps) updated in the same order and the same tail, so both
// give the same sums to the bit.
template <bool PAIR, int ROWS>
__device__ __forceinline__ float4 quad_walk(const float4 *__restrict__ Q, int SP, float q, float m, int lo, int hi,
                                            int s0, float h, unsigned top)
{
    static_assert(ROWS == 2 || ROWS == 4, "steps are evaluated in pairs, one or two pairs per pass");
    const float2 qk = pk(q, __fmaf_rn(1.0f, m, q));   // q + k m for the steps k = 0, 1 of a pair
    const float2 mm = pk(m, m), bias = pk(JOSEPH_BIAS, JOSEPH_BIAS);
    float spk = (float)lo - h;
    int ridx = (lo - s0) * SP;
    float2 ab[2], ce[2];   // (band A, band B) sums of the even and odd steps, at i0 and at the reflected pair
    ab[0] = ab[1] = ce[0] = ce[1] = pk(0.0f, 0.0f);
    // the samples of the steps s and s + 1, at (s - h) = sp
    auto pair_samples = [&](float sp, int rr, float4 &p0, float4 &p1, float4 &r0, float4 &r1, float2 &g) {
        const float2 up = pfma(pk(sp, sp), mm, qk);
        const float2 t = padd(up, bias);
        const float2 tb = psub(t, bias);
        g = psub(up, tb);
        const unsigned i0 = min((unsigned)(__float_as_int(t.x) - (JOSEPH_BIAS_BITS - 2)), top);
        const unsigned i1 = min((unsigned)(__float_as_int(t.y) - (JOSEPH_BIAS_BITS - 2)), top);
        p0 = Q[rr + (int)i0];
        p1 = Q[rr + SP + (int)i1];
        if (PAIR) {
            r0 = Q[rr + (int)(top - i0)];
            r1 = Q[rr + SP + (int)(top - i1)];
        }
    };
    auto pair_add = [&](const float4 &p0, const float4 &p1, const float4 &r0, const float4 &r1, float2 g) {
        ab[0] = pfma(pk(g.x, g.x), pk(p0.z, p0.w), padd(ab[0], pk(p0.x, p0.y)));
        ab[1] = pfma(pk(g.y, g.y), pk(p1.z, p1.w), padd(ab[1], pk(p1.x, p1.y)));
        if (PAIR) {
            ce[0] = pfma(pk(-g.x, -g.x), pk(r0.z, r0.w), padd(ce[0], pk(r0.x, r0.y)));
            ce[1] = pfma(pk(-g.y, -g.y), pk(r1.z, r1.w), padd(ce[1], pk(r1.x, r1.y)));
        }
    };
    int s = lo;
    for (; s + ROWS - 1 <= hi; s += ROWS) {
        float4 p[ROWS], r[ROWS];
        float2 g[ROWS / 2];
#pragma unroll
        for (int k = 0; k < ROWS / 2; ++k)
            pair_samples(k == 0 ? spk : __fadd_rn(spk, (float)(2 * k)), ridx + 2 * k * SP, p[2 * k], p[2 * k + 1],
                         r[2 * k], r[2 * k + 1], g[k]);
#pragma unroll
        for (int k = 0; k < ROWS / 2; ++k) pair_add(p[2 * k], p[2 * k + 1], r[2 * k], r[2 * k + 1], g[k]);
        spk = __fadd_rn(spk, (float)ROWS);
        ridx += ROWS * SP;
    }
    if (ROWS == 4 && s + 1 <= hi) {   // the pair ROWS = 2 would still take
        float4 p0, p1, r0, r1;
        float2 g;
        pair_samples(spk, ridx, p0, p1, r0, r1, g);
        pair_add(p0, p1, r0, r1, g);
        spk = __fadd_rn(spk, 2.0f);
        ridx += 2 * SP;
        s += 2;
    }
    if (s <= hi) {   // one step left
        const float up = joseph_u(spk, m, qk.x);
        const float t = __fadd_rn(up, JOSEPH_BIAS);
        const unsigned i = min((unsigned)(__float_as_int(t) - (JOSEPH_BIAS_BITS - 2)), top);
        const float g = __fsub_rn(up, __fsub_rn(t, JOSEPH_BIAS));
        const float4 pv = Q[ridx + (int)i];
        ab[0] = pfma(pk(g, g), pk(pv.z, pv.w), padd(ab[0], pk(pv.x, pv.y)));
        if (PAIR) {
            const float4 rv = Q[ridx + (int)(top - i)];
            ce[0] = pfma(pk(-g, -g), pk(rv.z, rv.w), padd(ce[0], pk(rv.x, rv.y)));
        }
    }
    ab[0] = padd(ab[0], ab[1]);
    ce[0] = padd(ce[0], ce[1]);
    return make_float4(ab[0].x, ab[0].y, ce[0].x, ce[0].y);
}

// Stages band pair s0 of image img into Q: pair i (stored at i + 2) of step
// t holds (A mid, B mid, A delta, B delta), band A the image line s0 + t
// and band B the line N-1-s0-t read backwards (image value at N-1-i); the
// lines are image rows (rows) or columns.  Runs on the threads of c and
// ends without a barrier.
template <bool DEEP, class Ctx>
__device__ __forceinline__ void quad_stage(const Ctx &c, float4 *Q, const float *img, int N, int s0, bool rows)
{
    static_assert(MR == 16, "column staging: a warp's lanes take the 16 steps of two pairs");
    const int CW = N + 3, SP = CW | 1;
    const int tid = c.tid(), nth = c.nth();
    // one thread forms both bands' pairs of (t, i) and stores them as one float4
    const int lx = tid & 31, nw = nth >> 5;
    if constexpr (DEEP) {
        // each thread issues the loads of SU pairs before it stores any, so
        // that SU L2 round trips overlap (grids of few blocks, whose threads
        // each stage many pairs)
        constexpr int SU = 4;
        float a0[SU], a1[SU], b0[SU], b1[SU];
        if (rows) {
            const int nch = (CW + 31) >> 5, nc = MR * nch;
            for (int c0 = tid >> 5; c0 < nc; c0 += SU * nw) {
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    const int ch = c0 + u * nw;
                    const int t = ch / nch, ii = ((ch - t * nch) << 5) + lx;
                    const bool ok = ch < nc && ii < CW;
                    const int i = ii - 2;
                    const float *ra = img + (size_t)(s0 + t) * N, *rb = img + (size_t)(N - 1 - s0 - t) * N;
                    a0[u] = (ok && i >= 0 && i < N) ? ra[i] : 0.0f;
                    a1[u] = (ok && i + 1 >= 0 && i + 1 < N) ? ra[i + 1] : 0.0f;
                    b0[u] = (ok && N - 1 - i >= 0 && N - 1 - i < N) ? rb[N - 1 - i] : 0.0f;
                    b1[u] = (ok && N - 2 - i >= 0 && N - 2 - i < N) ? rb[N - 2 - i] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    const int ch = c0 + u * nw;
                    const int t = ch / nch, ii = ((ch - t * nch) << 5) + lx;
                    if (ch < nc && ii < CW)
                        Q[t * SP + ii] = make_float4(0.5f * (a0[u] + a1[u]), 0.5f * (b0[u] + b1[u]), a1[u] - a0[u],
                                                     b1[u] - b0[u]);
                }
            }
        } else {
            const int t = lx & 15;
            const float *ia = img + (s0 + t), *ib = img + (N - 1 - s0 - t);   // columns of bands A, B
            const int nc = (CW + 1) >> 1;
            for (int c0 = tid >> 5; c0 < nc; c0 += SU * nw) {
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    const int ii = 2 * (c0 + u * nw) + (lx >> 4);
                    const bool ok = c0 + u * nw < nc && ii < CW;
                    const int i = ii - 2;   // rows i, i + 1 (band A), N-1-i, N-2-i (band B); N N < 2^31
                    a0[u] = (ok && i >= 0 && i < N) ? ia[i * N] : 0.0f;
                    a1[u] = (ok && i + 1 >= 0 && i + 1 < N) ? ia[(i + 1) * N] : 0.0f;
                    b0[u] = (ok && N - 1 - i >= 0 && N - 1 - i < N) ? ib[(N - 1 - i) * N] : 0.0f;
                    b1[u] = (ok && N - 2 - i >= 0 && N - 2 - i < N) ? ib[(N - 2 - i) * N] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    const int ii = 2 * (c0 + u * nw) + (lx >> 4);
                    if (c0 + u * nw < nc && ii < CW)
                        Q[t * SP + ii] = make_float4(0.5f * (a0[u] + a1[u]), 0.5f * (b0[u] + b1[u]), a1[u] - a0[u],
                                                     b1[u] - b0[u]);
                }
            }
        }
    } else if (rows) {
        // warps take 32-pair chunks of the 16 steps, lanes neighbouring pairs
        const int nch = (CW + 31) >> 5;
        for (int ch = tid >> 5; ch < MR * nch; ch += nw) {
            const int t = ch / nch, ii = ((ch - t * nch) << 5) + lx;
            if (ii < CW) {
                const int i = ii - 2;
                const float *ra = img + (size_t)(s0 + t) * N, *rb = img + (size_t)(N - 1 - s0 - t) * N;
                const float a0 = (i >= 0 && i < N) ? ra[i] : 0.0f;
                const float a1 = (i + 1 >= 0 && i + 1 < N) ? ra[i + 1] : 0.0f;
                const float b0 = (N - 1 - i >= 0 && N - 1 - i < N) ? rb[N - 1 - i] : 0.0f;
                const float b1 = (N - 2 - i >= 0 && N - 2 - i < N) ? rb[N - 2 - i] : 0.0f;
                Q[(size_t)t * SP + ii] = make_float4(0.5f * (a0 + a1), 0.5f * (b0 + b1), a1 - a0, b1 - b0);
            }
        }
    } else {
        // lanes take the 16 steps (columns) of two neighbouring pairs:
        // 64-byte row segments in, conflict-free float4 stores (odd SP)
        const int t = lx & 15, ca = s0 + t, cb = N - 1 - s0 - t;
        for (int ch = tid >> 5; 2 * ch < CW; ch += nw) {
            const int ii = 2 * ch + (lx >> 4);
            if (ii < CW) {
                const int i = ii - 2;
                const float a0 = (i >= 0 && i < N) ? img[(size_t)i * N + ca] : 0.0f;
                const float a1 = (i + 1 >= 0 && i + 1 < N) ? img[(size_t)(i + 1) * N + ca] : 0.0f;
                const float b0 = (N - 1 - i >= 0 && N - 1 - i < N) ? img[(size_t)(N - 1 - i) * N + cb] : 0.0f;
                const float b1 = (N - 2 - i >= 0 && N - 2 - i < N) ? img[(size_t)(N - 2 - i) * N + cb] : 0.0f;
                Q[(size_t)t * SP + ii] = make_float4(0.5f * (a0 + a1), 0.5f * (b0 + b1), a1 - a0, b1 - b0);
            }
        }
    }
}

// Walks ray position idx of view-pair item (v, vp) through the staged band
// pair (steps s0 .. s0 + MR - 1) and stores its band sums into the partial
// slot out (V x B): ray d and its detector mirror B-1-d of view v and, for
// vp >= 0, of view vp.  Positions map to rays in whole blocks of 8 cs
// positions, where the eight lanes of a quarter warp take rays cs apart,
// spreading their 16-byte loads over the bank groups; the last partial
// block maps to itself.
template <int ROWS>
__device__ __forceinline__ void quad_position(const float4 *Q, int SP, float a, float m, float inv_m, int cs, int v,
                                              int vp, bool rows, int idx, int npair, int N, int B, int s0, float h,
                                              float hq, unsigned top, float *out)
{
    int d = idx;
    {
        const int blk = 8 * cs, b = idx / blk, r = idx - b * blk;
        if ((b + 1) * blk <= npair) d = b * blk + (r & 7) * cs + (r >> 3);
    }
    const int dm = B - 1 - d;
    float ov[2] = {0.0f, 0.0f}, op[2] = {0.0f, 0.0f};   // view v / vp: [0] ray d, [1] ray dm
#pragma unroll
    for (int which = 0; which < 2; ++which) {
        if (which == 1 && dm == d) break;
        const int dd = which == 0 ? d : dm;
        const float q = joseph_q(joseph_dp(dd, B), a, hq);
        int lo, hi;
        step_range(q, m, inv_m, h, -2.5f, (float)N + 0.5f, s0, s0 + MR - 1, lo, hi);
        const float4 r = vp >= 0 ? quad_walk<true, ROWS>(Q, SP, q, m, lo, hi, s0, h, top)
                                 : quad_walk<false, ROWS>(Q, SP, q, m, lo, hi, s0, h, top);
        ov[which] += r.x;
        ov[1 - which] += r.y;
        if (rows) {
            op[which] += r.z;
            op[1 - which] += r.w;
        } else {
            op[1 - which] += r.z;
            op[which] += r.w;
        }
    }
    float *o = out + (size_t)v * B;
    if (dm == d) {
        o[d] = ov[0] + ov[1];
    } else {
        o[d] = ov[0];
        o[dm] = ov[1];
    }
    if (vp >= 0) {
        float *o2 = out + (size_t)vp * B;
        if (dm == d) {
            o2[d] = op[0] + op[1];
        } else {
            o2[d] = op[0];
            o2[dm] = op[1];
        }
    }
}

// Body of block (bx, by, bz) of a grid of nbp band pairs: smraw holds
// quad_smem(N) bytes, the block's c.nth() = 64 pg threads.  The block
// stages its band pair once and then walks gpb groups of pg view-pair
// items of one class (rows or columns) one after the other, so that the
// staging is spread over gpb groups.
template <int ROWS, bool DEEP, class Ctx>
__device__ __forceinline__ void quad_body(const Ctx &c, int bx, int by, int bz, int nbp, unsigned char *smraw,
                                          const float *x, const ViewP *views, const int2 *row_items, int n_row,
                                          const int2 *col_items, int n_col, int N, int V, int B, int pg, int gpb,
                                          float *partial)
{
    const int SP = (N + 3) | 1;
    float4 *Q = reinterpret_cast<float4 *>(smraw);   // [step][pair]: band A pair, band B pair

    const int bp = bx;
    const int row_groups = (n_row + pg - 1) / pg, col_groups = (n_col + pg - 1) / pg;
    const int row_blocks = (row_groups + gpb - 1) / gpb;
    const bool rows = by < row_blocks;
    const int grp0 = (rows ? by : by - row_blocks) * gpb;
    const int ngrp = min(gpb, (rows ? row_groups : col_groups) - grp0);
    const int2 *list = rows ? row_items : col_items;
    const int nl = rows ? n_row : n_col;
    float *out = partial + ((size_t)bz * nbp + bp) * V * B;
    const int s0 = bp * MR;
    const float h = joseph_h(N), hq = joseph_hq(N);
    const int tid = c.tid();

    quad_stage<DEEP>(c, Q, x + (size_t)bz * N * N, N, s0, rows);
    c.sync();
    const int npair = (B + 1) / 2;
    const unsigned top = (unsigned)(N + 2);
    const int vi = tid >> 6;
    for (int gi = 0; gi < ngrp; ++gi) {
        const int grp = grp0 + gi;
        if (vi >= min(pg, nl - grp * pg)) break;
        const int2 it = list[grp * pg + vi];
        const ViewP &vw = views[it.x];
        const float a = vw.a, m = vw.m, inv_m = vw.inv_m;
        const int cs = vw.stride;
        for (int idx = tid & 63; idx < npair; idx += 64)
            quad_position<ROWS>(Q, SP, a, m, inv_m, cs, it.x, it.y, rows, idx, npair, N, B, s0, h, hq, top, out);
    }
}

// Work-balanced form of the same projection.  The work of a batch is cut
// into units (slice, class, band pair, item, chunk of 64 ray positions),
// ordered so that the units of one staged band pair (a segment) are
// consecutive; each block takes the equal range [u0, u1) of units, stages
// each segment the range touches once, and its warps take the segment's
// units one at a time from a shared counter.  Blocks thus carry equal work
// whatever the number of items, and a block holds as many warps as its
// registers allow.  The sums are those of quad_body, unit for unit.
struct QuadUnits {
    int nch;        // 64-position chunks per item
    int u_rows;     // units of one row-class segment: n_row items x nch
    int u_cols;     // units of one column-class segment
    long long u_z;  // units per slice: nbp (u_rows + u_cols)
};

template <int ROWS, bool DEEP, class Ctx>
__device__ __forceinline__ void quad_balanced_body(const Ctx &c, long long u0, long long u1, const QuadUnits &U,
                                                   unsigned char *smraw, int *next, const float *x,
                                                   const ViewP *views, const int2 *row_items,
                                                   const int2 *col_items, int N, int V, int B, float *partial)
{
    const int SP = (N + 3) | 1, nbp = N / (2 * MR);
    float4 *Q = reinterpret_cast<float4 *>(smraw);
    const float h = joseph_h(N), hq = joseph_hq(N);
    const int npair = (B + 1) / 2;
    const unsigned top = (unsigned)(N + 2);
    const int tid = c.tid(), lane = tid & 31;
    const long long rows_all = (long long)nbp * U.u_rows;
    long long u = u0;
    while (u < u1) {
        // the segment of unit u: slice z, class, band pair bp
        const long long z = u / U.u_z, r = u - z * U.u_z;
        const bool rows = r < rows_all;
        const long long r2 = rows ? r : r - rows_all;
        const int per = rows ? U.u_rows : U.u_cols;
        const int bp = (int)(r2 / per);
        const long long seg0 = u - (r2 - (long long)bp * per);
        const long long e = min(u1, seg0 + per);
        const int s0 = bp * MR;
        quad_stage<DEEP>(c, Q, x + (size_t)z * N * N, N, s0, rows);
        if (tid == 0) *next = (int)(u - seg0);
        c.sync();
        const int2 *list = rows ? row_items : col_items;
        float *out = partial + ((size_t)z * nbp + bp) * V * B;
        const int n_units = (int)(e - seg0);
        for (;;) {
            int w = 0;
            if (lane == 0) w = atomicAdd(next, 1);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (w >= n_units) break;
            const int item = w / U.nch, chunk = w - item * U.nch;
            const int2 it = list[item];
            const ViewP &vw = views[it.x];
            const float a = vw.a, m = vw.m, inv_m = vw.inv_m;
            const int cs = vw.stride;
#pragma unroll 1
            for (int k = 0; k < 2; ++k) {
                const int idx = chunk * 64 + k * 32 + lane;
                if (idx < npair)
                    quad_position<ROWS>(Q, SP, a, m, inv_m, cs, it.x, it.y, rows, idx, npair, N, B, s0, h, hq, top,
                                        out);
            }
        }
        c.sync();
        u = e;
    }
}

// =====================================================================
// Backprojection by rotation orbits (default angles, V and N even).
// View v + V/2 is view v turned by 90 degrees and the detector mirror
// d -> B-1-d is the turn by 180 degrees, so for a pixel P the detector
// coordinate e of (P, view v) is also that of (R90 P, view v + V/2), and the
// mirrored coordinate B-1-e is that of (R180 P, v) and (R270 P, v + V/2).
// One weight evaluation (floor, fraction, two hat weights) therefore
// serves four pixel-views; a block takes a 16 x 16 tile of one image
// quadrant and evaluates, per base view v < V/2, the weights of P and of
// R90 P, which cover all eight (pixel, view) pairs of the orbit
// {P, R90 P, R180 P, R270 P} x {v, v + V/2}.  Each of the block's
// 16 ORB_TY threads takes the orbits of ORB_PX pixels of one tile column
// (rows r, r + ORB_TY, ..), so the per-view constants, window bases and
// loop control are shared by 8 ORB_PX pixel-views.  Base views are split into
// nsl slices (grid.z; 4 unless tuned, at most ORB_SL_MAX), added in slice
// order: in a thread-block cluster of the slices' blocks
// (k_backproject_orbit_cl), or from slice images (the persistent batched
// kernel's reduction phase).  The weights are the
// pixel-side Joseph weights of k_backproject_tiles, so both kernels compute
// the same A^T.
// =====================================================================
constexpr int ORB_T = 16;        // quadrant tile side
constexpr int ORB_TY = 8;        // thread rows of a block: tile rows r, r + ORB_TY, ... each
constexpr int ORB_TH = ORB_T * ORB_TY;
constexpr int ORB_PX = ORB_T / ORB_TY;   // pixel orbits per thread
constexpr int ORB_SL = 4;        // base-view slices unless tuned
constexpr int ORB_SL_MAX = 8;
constexpr int ORB_VC = 8;        // base views staged per chunk
constexpr int ORB_RW = 36;       // values per window: pairs (k, k+1), k <= ORB_RW - 2
constexpr int ORB_MAXS = 1024;   // base views per slice (V <= 8192)

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 4 : 0;   // 0: fill with zeros, read nothing
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sdst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src, bool valid)
{
    const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sdst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// Body of block (bx, by, bz) (c.nth() = ORB_TH threads, as ORB_T x ORB_TY);
// osm holds orbit_smem() bytes.  CL: instead of storing its sums, the
// block leaves them in osm, entry (k ORB_PX + j) ORB_TH + tid for rotation
// k of the thread's pixel orbit j, for a cluster reduction over slices.
template <bool AL, class Ctx, bool CL = false>
__device__ __forceinline__ void orbit_body(const Ctx &cb, int bx, int by, int bz, unsigned char *osm, const float *y,
                                           float *partial, const float4 *trig, int N, int V, int B, int nsl,
                                           int fin, float *out, const float *xin, const double *scal)
{
    // raw[buffer][view][row (v, v+V/2)][window (e, mirror e, e90, mirror e90)][value]
    float *raw = reinterpret_cast<float *>(osm);                               // 2 x ORB_VC x 8 x ORB_RW
    float4 *tt = reinterpret_cast<float4 *>(raw + 2 * ORB_VC * 8 * ORB_RW);    // 2 x ORB_VC
    int *wbs = reinterpret_cast<int *>(tt + 2 * ORB_VC);                       // ORB_MAXS x 2
    const int tid = cb.tid();   // tid / ORB_T < ORB_TY
    const int tx = tid % ORB_T, ty = tid / ORB_T;
    const int half = N / 2, V2 = V / 2;
    const int slice = bz % nsl, img = bz / nsl;
    const int r0 = by * ORB_T, c0 = half + bx * ORB_T;   // quadrant r < N/2, c >= N/2
    const int r = r0 + ty, c = c0 + tx;                  // pixels (r + j ORB_TY, c)
    const bool inside = r < half && c < N;
    const float h = 0.5f * (float)(N - 1), hb = 0.5f * (float)(B - 1), hb_lo = hb - 0.5f;
    const float xq = (float)c - h, yq = (float)r - h;               // P = (x, y); R90 P = (-y, x)
    const float *ys = y + (size_t)img * V * B;
    const int vb0 = (int)((long long)V2 * slice / nsl), vb1 = (int)((long long)V2 * (slice + 1) / nsl);
    const int nvs = vb1 - vb0;
    float acc[ORB_PX][4];   // per pixel orbit: P, R90 P, R180 P, R270 P
#pragma unroll
    for (int j = 0; j < ORB_PX; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;

    // window bases (multiples of 4) of the tile for every base view of this
    // slice: floor(e) - wb lies in [1, 29] for every pixel of the tile, as
    // e spans at most 15 (|cos| + |sin|) < 21.3 over it
    for (int vi = tid; vi < nvs; vi += ORB_TH) {
        const float4 T = trig[vb0 + vi];
        float emin = 3.0e38f, e9min = 3.0e38f;
#pragma unroll
        for (int cr = 0; cr < 4; ++cr) {
            const float xx = (float)(c0 + (cr & 1) * (ORB_T - 1)) - h;
            const float yy = (float)(r0 + (cr >> 1) * (ORB_T - 1)) - h;
            emin = fminf(emin, xx * T.x + yy * T.y);
            e9min = fminf(e9min, -yy * T.x + xx * T.y);
        }
        emin = fminf(fmaxf(emin + hb, -1.0e6f), 1.0e6f);
        e9min = fminf(fmaxf(e9min + hb, -1.0e6f), 1.0e6f);
        wbs[2 * vi] = ((int)floorf(emin) - 2) & ~3;
        wbs[2 * vi + 1] = ((int)floorf(e9min) - 2) & ~3;
    }
    cb.sync();

    // raw window values y[start + w], w < ORB_RW, start = wb (windows e, e90)
    // or B - ORB_RW - wb (their mirrors, holding pair B-2-f at ORB_RW-2 - (f - wb));
    // per view (cos, sin, |a|^2, |a| (1 - |a|/2)): the hat weights times |a|
    auto issue = [&](int v0, int nv, int buf) {
        float *dst0 = raw + (size_t)buf * ORB_VC * 8 * ORB_RW;
        if (tid < nv) {
            const float4 T = trig[v0 + tid];
            tt[buf * ORB_VC + tid] = make_float4(T.x, T.y, T.z * T.z, T.z * T.w);
        }
        constexpr int CH = AL ? ORB_RW / 4 : ORB_RW;   // copies per window
        for (int k = tid; k < nv * 8 * CH; k += ORB_TH) {
            const int q = k / CH, j = k - q * CH;
            const int win = q & 3, row = (q >> 2) & 1, vi = q >> 3;
            const int base = wbs[2 * (v0 - vb0 + vi) + (win >> 1)];
            const int d = ((win & 1) ? B - ORB_RW - base : base) + (AL ? 4 * j : j);
            const bool ok = d >= 0 && d < B;
            const float *src = ys + (size_t)(v0 + vi + row * V2) * B + (ok ? d : 0);
            if (AL) cp_async16(dst0 + (size_t)q * ORB_RW + 4 * j, src, ok);
            else cp_async4(dst0 + (size_t)q * ORB_RW + j, src, ok);
        }
        cp_async_commit();
    };
    const int nch = (nvs + ORB_VC - 1) / ORB_VC;
    if (nch > 0) issue(vb0, min(ORB_VC, nvs), 0);
    for (int ch = 0; ch < nch; ++ch) {
        const int v0 = vb0 + ch * ORB_VC, nv = min(ORB_VC, vb1 - v0);
        if (ch + 1 < nch) {
            issue(v0 + ORB_VC, min(ORB_VC, vb1 - v0 - ORB_VC), (ch + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        cb.sync();
        const float *tb = raw + (size_t)(ch & 1) * ORB_VC * 8 * ORB_RW;
        const float4 *tv = tt + (ch & 1) * ORB_VC;
        if (inside) {
            for (int vi = 0; vi < nv; ++vi) {
                const float4 T = tv[vi];
                const int2 wb = *reinterpret_cast<const int2 *>(wbs + 2 * (v0 - vb0 + vi));
                const float *t8 = tb + (size_t)vi * 8 * ORB_RW;   // [row][win][value]
                const float *e_v = t8, *m_v = t8 + ORB_RW, *e9_v = t8 + 2 * ORB_RW, *m9_v = t8 + 3 * ORB_RW;
                const float *e_w = t8 + 4 * ORB_RW, *m_w = t8 + 5 * ORB_RW, *e9_w = t8 + 6 * ORB_RW,
                            *m9_w = t8 + 7 * ORB_RW;
                // the orbit of the pixel at (x, y) = (xq, yy): e - 1/2 of P and of R90 P
                auto orbit = [&](float yy, float &cP, float &c90, float &c180, float &c270) {
                    const float e = fmaf(xq, T.x, fmaf(yy, T.y, hb_lo));
                    const float e9 = fmaf(xq, T.y, fmaf(-yy, T.x, hb_lo));
                    const float t = __fadd_rn(e, JOSEPH_BIAS), t9 = __fadd_rn(e9, JOSEPH_BIAS);
                    const unsigned k = min((unsigned)(__float_as_int(t) - (JOSEPH_BIAS_BITS + wb.x)),
                                           (unsigned)(ORB_RW - 2));
                    const unsigned k9 = min((unsigned)(__float_as_int(t9) - (JOSEPH_BIAS_BITS + wb.y)),
                                            (unsigned)(ORB_RW - 2));
                    const float g = __fsub_rn(e, __fsub_rn(t, JOSEPH_BIAS));
                    const float g9 = __fsub_rn(e9, __fsub_rn(t9, JOSEPH_BIAS));
                    const float w0 = fmaxf(0.0f, fmaf(-g, T.z, T.w)), w1 = fmaxf(0.0f, fmaf(g, T.z, T.w));
                    const float w09 = fmaxf(0.0f, fmaf(-g9, T.z, T.w)), w19 = fmaxf(0.0f, fmaf(g9, T.z, T.w));
                    const unsigned km = ORB_RW - 2 - k, km9 = ORB_RW - 2 - k9;
                    cP = fmaf(w0, e_v[k], fmaf(w1, e_v[k + 1], cP));             // P at v
                    c180 = fmaf(w1, m_v[km], fmaf(w0, m_v[km + 1], c180));       // R180 P at v
                    c90 = fmaf(w0, e_w[k], fmaf(w1, e_w[k + 1], c90));           // R90 P at v + V/2
                    c270 = fmaf(w1, m_w[km], fmaf(w0, m_w[km + 1], c270));       // R270 P at v + V/2
                    c90 = fmaf(w09, e9_v[k9], fmaf(w19, e9_v[k9 + 1], c90));     // R90 P at v
                    c270 = fmaf(w19, m9_v[km9], fmaf(w09, m9_v[km9 + 1], c270)); // R270 P at v
                    c180 = fmaf(w09, e9_w[k9], fmaf(w19, e9_w[k9 + 1], c180));   // R180 P at v + V/2
                    cP = fmaf(w19, m9_w[km9], fmaf(w09, m9_w[km9 + 1], cP));     // P at v + V/2
                };
#pragma unroll
                for (int j = 0; j < ORB_PX; ++j)
                    if (j == 0 || r + j * ORB_TY < half)
                        orbit(yq + (float)(j * ORB_TY), acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
            }
        }
        cb.sync();   // the buffer is refilled two chunks later
    }
    if constexpr (CL) {
        float *red = reinterpret_cast<float *>(osm);   // the staging buffers are free again
#pragma unroll
        for (int j = 0; j < ORB_PX; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[(k * ORB_PX + j) * ORB_TH + tid] = acc[j][k];
        return;
    }
    // fin 0: the slice's partial image; with a single slice the sums are
    // complete and the block writes the result itself: fin 1 out = sum,
    // fin 2 out = xin - tau sum
    float *pp = (fin ? out : partial) + ((size_t)img * (fin ? 1 : nsl) + slice) * N * N;
    const float *xq0 = fin == 2 ? xin + (size_t)img * N * N : nullptr;
    const float tau = fin == 2 ? fscal(scal, F_TAU) : 0.0f;
#pragma unroll
    for (int j = 0; j < ORB_PX; ++j) {
        const int rj = r + j * ORB_TY;
        if (rj < half && c < N) {
            const size_t o[4] = {(size_t)rj * N + c,                    // P
                                 (size_t)c * N + (N - 1 - rj),          // R90 (r, c) = (c, N-1-r)
                                 (size_t)(N - 1 - rj) * N + (N - 1 - c), // R180 (r, c) = (N-1-r, N-1-c)
                                 (size_t)(N - 1 - c) * N + rj};         // R270 (r, c) = (N-1-c, r)
#pragma unroll
            for (int k = 0; k < 4; ++k) pp[o[k]] = fin == 2 ? __fmaf_rn(-tau, acc[j][k], xq0[o[k]]) : acc[j][k];
        }
    }
}

}  // namespace ctpd
