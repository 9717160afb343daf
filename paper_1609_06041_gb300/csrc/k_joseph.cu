// k_joseph.cu -- Joseph forward projector A (ray-driven) and its transpose
// A^T (pixel-driven gather), the A and A^T of Eqs. 18-20 / 29-31.  Both are
// deterministic (fixed summation orders, no atomics).
#include <algorithm>

#include "ctpd_internal.cuh"

namespace ctpd {

__device__ __forceinline__ float joseph_h(int n) { return 0.5f * (float)(n - 1); }
__device__ __forceinline__ float joseph_dp(int d, int B) { return __fsub_rn((float)d, 0.5f * (float)(B - 1)); }

// =====================================================================
// Forward projection.
// A block owns a band of PROJ_R consecutive steps (rows for row-stepping
// views, columns for column-stepping views) and a group of PG views of one
// class.  It stages the band in shared memory as interpolation pairs
//     P[i] = ((x[i] + x[i+1]) / 2, x[i+1] - x[i]),  i = -2 .. N (zero padded),
// so one sample is fma(g, P.y, P.x) = (1/2 - g) x[i0] + (1/2 + g) x[i0+1].
// Each thread walks whole rays across the band and writes the band's
// partial ray sum; launch_band_reduce adds the bands in a fixed order.
// Images wider than one staged row (PROJ_CW pairs) are staged in several
// column passes; a sample is taken in the pass that holds its pair and the
// pass sums are added to the partial in pass order.
// =====================================================================
constexpr int PG = 16;         // views per block
constexpr int PT = 1024;       // threads per block
constexpr int PROJ_CW = 640;   // pairs per staged band row

static int proj_cw(int n) { return (n + 3) < PROJ_CW ? (n + 3) : PROJ_CW; }
static int proj_stride(int n) { return proj_cw(n) | 1; }   // odd: spreads smem banks
static size_t proj_smem(int n) { return sizeof(float2) * (size_t)PROJ_R * proj_stride(n) + sizeof(ViewP) * PG + 64; }

__device__ __forceinline__ int d_proj_cw(int n) { return (n + 3) < PROJ_CW ? (n + 3) : PROJ_CW; }

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
    float sa = (ulo - q) * inv_m + h, sb = (uhi - q) * inv_m + h;
    float smin = fminf(sa, sb), smax = fmaxf(sa, sb);
    // clamp before converting: far-off rays give huge (or infinite) s
    smin = fminf(fmaxf(smin, (float)s_lo - 2.0f), (float)s_hi + 2.0f);
    smax = fminf(fmaxf(smax, (float)s_lo - 2.0f), (float)s_hi + 2.0f);
    lo = max(s_lo, (int)floorf(smin) - 1);
    hi = min(s_hi, (int)ceilf(smax) + 1);
}

template <bool MULTI>
__global__ void __launch_bounds__(PT)
k_project_bands(const float *__restrict__ x, const ViewP *__restrict__ views,
                const int *__restrict__ row_list, int n_row, const int *__restrict__ col_list, int n_col,
                int N, int V, int B, float *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int CW = d_proj_cw(N), SP = CW | 1;
    float2 *P = reinterpret_cast<float2 *>(smraw);
    ViewP *sv = reinterpret_cast<ViewP *>(P + (size_t)PROJ_R * SP);
    int *svi = reinterpret_cast<int *>(sv + PG);

    const int band = blockIdx.x, nb = gridDim.x;
    const int row_groups = (n_row + PG - 1) / PG;
    const bool rows = (int)blockIdx.y < row_groups;
    const int grp = rows ? blockIdx.y : blockIdx.y - row_groups;
    const int *list = rows ? row_list : col_list;
    const int nl = rows ? n_row : n_col;
    const int nv = min(PG, nl - grp * PG);
    const float *img = x + (size_t)blockIdx.z * N * N;
    float *out = partial + ((size_t)blockIdx.z * nb + band) * V * B;
    const int s0 = band * PROJ_R, ns = min(PROJ_R, N - s0);
    const float h = joseph_h(N), hq = joseph_hq(N);
    const int tid = threadIdx.x;

    if (tid < nv) {
        svi[tid] = list[grp * PG + tid];
        sv[tid] = views[svi[tid]];
    }
    for (int I0 = -2; I0 <= N; I0 += CW) {
        const int I1 = min(I0 + CW, N + 1);   // this pass holds pairs I0 .. I1-1
        const int w = I1 - I0;
        __syncthreads();
        if (rows) {
            for (int k = tid; k < ns * w; k += PT) {
                const int si = k / w, i = I0 + (k - si * w);
                const float *rowp = img + (size_t)(s0 + si) * N;
                const float a = (i >= 0 && i < N) ? rowp[i] : 0.0f;
                const float b = (i + 1 >= 0 && i + 1 < N) ? rowp[i + 1] : 0.0f;
                P[si * SP + (i - I0)] = make_float2(0.5f * (a + b), b - a);
            }
        } else {
            // column band: pair i of step (column) c = s0 + si is (x[i][c], x[i+1][c]);
            // neighbouring threads take neighbouring columns (coalesced rows)
            for (int k = tid; k < ns * w; k += PT) {
                const int ii = k / ns, si = k - ii * ns, i = I0 + ii, c = s0 + si;
                const float a = (i >= 0 && i < N) ? img[(size_t)i * N + c] : 0.0f;
                const float b = (i + 1 >= 0 && i + 1 < N) ? img[(size_t)(i + 1) * N + c] : 0.0f;
                P[si * SP + ii] = make_float2(0.5f * (a + b), b - a);
            }
        }
        __syncthreads();
        // samples with non-zero weight have u' in (-1.5, N - 0.5); this pass
        // takes those with round(u') in [I0, I1)
        const float ulo = (float)max(I0, -1) - 1.5f, uhi = (float)min(I1, N) + 0.5f;
        for (int slot = tid; slot < nv * B; slot += PT) {
            const int vi = slot / B, d = slot - vi * B;
            const float a = sv[vi].a, m = sv[vi].m, inv_m = sv[vi].inv_m;
            const float q = joseph_q(joseph_dp(d, B), a, hq);
            int lo, hi;
            step_range(q, m, inv_m, h, ulo, uhi, s0, s0 + ns - 1, lo, hi);
            const float sp = (float)lo - h;
            int ridx = (lo - s0) * SP;                 // pair array offset of step lo
            float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
            if (!MULTI) {
                // steps lo, lo+1, ... as u'(s) = sp_k m + q with sp_k = (s - h) exact;
                // the pair index i0 + 2 is clamped to [0, N + 2] (both ends are zero pairs)
                const unsigned top = (unsigned)(N + 2);
                // q_u = q + u m: u'(s + u) = (s - h) m + q_u
                const float qu1 = __fadd_rn(q, m), qu2 = __fmaf_rn(2.0f, m, q), qu3 = __fmaf_rn(3.0f, m, q);
                float spk = sp;
                int s = lo;
                for (; s + 3 <= hi; s += 4) {
                    float2 pr[4];
                    float gg[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float qq = u == 0 ? q : (u == 1 ? qu1 : (u == 2 ? qu2 : qu3));
                        const float up = joseph_u(spk, m, qq);
                        const float t = __fadd_rn(up, JOSEPH_BIAS);
                        const unsigned ip = min((unsigned)(__float_as_int(t) - (JOSEPH_BIAS_BITS - 2)), top);
                        gg[u] = __fsub_rn(up, __fsub_rn(t, JOSEPH_BIAS));
                        pr[u] = P[ridx + u * SP + (int)ip];
                    }
                    acc0 += __fmaf_rn(gg[0], pr[0].y, pr[0].x);
                    acc1 += __fmaf_rn(gg[1], pr[1].y, pr[1].x);
                    acc2 += __fmaf_rn(gg[2], pr[2].y, pr[2].x);
                    acc3 += __fmaf_rn(gg[3], pr[3].y, pr[3].x);
                    spk = __fadd_rn(spk, 4.0f);
                    ridx += 4 * SP;
                }
                for (; s <= hi; ++s) {
                    const float up = joseph_u(spk, m, q);
                    const float t = __fadd_rn(up, JOSEPH_BIAS);
                    const unsigned ip = min((unsigned)(__float_as_int(t) - (JOSEPH_BIAS_BITS - 2)), top);
                    const float g = __fsub_rn(up, __fsub_rn(t, JOSEPH_BIAS));
                    const float2 p = P[ridx + (int)ip];
                    acc0 += __fmaf_rn(g, p.y, p.x);
                    spk = __fadd_rn(spk, 1.0f);
                    ridx += SP;
                }
            } else {
                float spk = sp;
                for (int s = lo; s <= hi; ++s) {
                    int i0;
                    float g;
                    joseph_round(joseph_u(spk, m, q), i0, g);
                    i0 = min(max(i0, -2), N);
                    if (i0 >= I0 && i0 < I1) {
                        const float2 p = P[ridx + (i0 - I0)];
                        acc0 += __fmaf_rn(g, p.y, p.x);
                    }
                    spk = __fadd_rn(spk, 1.0f);
                    ridx += SP;
                }
            }
            const float sum = (acc0 + acc1) + (acc2 + acc3);
            float *o = out + (size_t)svi[vi] * B + d;
            if (!MULTI || I0 == -2) *o = sum;
            else *o += sum;                       // this thread wrote it in the previous pass
        }
    }
}

// ---------------------------------------------------------------------
// Forward projection with the detector mirror (N a multiple of 32, one
// staged pass).  Ray B-1-d meets step N-1-s at the mirrored coordinate
// N-1-u of ray d at step s, so a block staging band A (steps s0 .. s0+15)
// and band B (steps N-1-s0-15 .. N-1-s0) turned by 180 degrees (step and
// pair order reversed) reads, for one evaluation of (u', g) at (d, s), the
// sample of ray d in band A and of ray B-1-d in band B at the same shared
// offset.  A thread takes the ray pair (d, B-1-d) and walks both rays; each
// ray's partial covers both bands.  Partial slots: N/32 per image, like the
// plain kernel's 32-step bands.
// ---------------------------------------------------------------------
constexpr int MR = 16;           // steps per band (two bands per block)
static_assert(PG * 64 == PT, "one view of the group per 64 threads");
static_assert(2 * MR == 32, "staging maps 32 lines (two bands) to 32 thread rows");

__global__ void __launch_bounds__(PT)
k_project_mirror(const float *__restrict__ x, const ViewP *__restrict__ views,
                 const int *__restrict__ row_list, int n_row, const int *__restrict__ col_list, int n_col,
                 int N, int V, int B, float *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int CW = N + 3, SP = CW | 1;
    float2 *PA = reinterpret_cast<float2 *>(smraw);
    float2 *PB = PA + (size_t)MR * SP;
    ViewP *sv = reinterpret_cast<ViewP *>(PB + (size_t)MR * SP);
    int *svi = reinterpret_cast<int *>(sv + PG);

    const int bp = blockIdx.x, nbp = gridDim.x;
    const int row_groups = (n_row + PG - 1) / PG;
    const bool rows = (int)blockIdx.y < row_groups;
    const int grp = rows ? blockIdx.y : blockIdx.y - row_groups;
    const int *list = rows ? row_list : col_list;
    const int nl = rows ? n_row : n_col;
    const int nv = min(PG, nl - grp * PG);
    const float *img = x + (size_t)blockIdx.z * N * N;
    float *out = partial + ((size_t)blockIdx.z * nbp + bp) * V * B;
    const int s0 = bp * MR;
    const float h = joseph_h(N), hq = joseph_hq(N);
    const int tid = threadIdx.x;

    if (tid < nv) {
        svi[tid] = list[grp * PG + tid];
        sv[tid] = views[svi[tid]];
    }
    // pair i (stored at i + 2) of step t: band A the image line s0 + t, band B
    // the line N-1-s0-t read backwards (image value at N-1-i).  Threads as
    // 32 x 32: rows class -> lanes along the line; column class -> lanes
    // across the 32 lines of both bands (coalesced image rows).
    {
        const int lx = tid & 31, ly = tid >> 5;
        if (rows) {
            const int band = ly >= MR, t = ly - band * MR;
            const int line = band == 0 ? s0 + t : N - 1 - s0 - t;
            const float *rowp = img + (size_t)line * N;
            float2 *dst = (band == 0 ? PA : PB) + t * SP;
            for (int ii = lx; ii < CW; ii += 32) {
                const int i = ii - 2;
                const int ia = band == 0 ? i : N - 1 - i, ib = band == 0 ? i + 1 : N - 2 - i;
                const float a = (ia >= 0 && ia < N) ? rowp[ia] : 0.0f;
                const float b = (ib >= 0 && ib < N) ? rowp[ib] : 0.0f;
                dst[ii] = make_float2(0.5f * (a + b), b - a);
            }
        } else {
            const int band = lx >= MR, t = lx - band * MR;
            const int line = band == 0 ? s0 + t : N - 1 - s0 - t;
            float2 *dst = (band == 0 ? PA : PB) + t * SP;
            for (int ii = ly; ii < CW; ii += 32) {
                const int i = ii - 2;
                const int ia = band == 0 ? i : N - 1 - i, ib = band == 0 ? i + 1 : N - 2 - i;
                const float a = (ia >= 0 && ia < N) ? img[(size_t)ia * N + line] : 0.0f;
                const float b = (ib >= 0 && ib < N) ? img[(size_t)ib * N + line] : 0.0f;
                dst[ii] = make_float2(0.5f * (a + b), b - a);
            }
        }
    }
    __syncthreads();
    const int npair = (B + 1) / 2;
    const unsigned top = (unsigned)(N + 2);
    // thread -> view tid / 64 of the group, ray pairs (tid % 64) + 64 j
    const int vi = tid >> 6;
    if (vi >= nv) return;
    for (int d = tid & 63; d < npair; d += 64) {
        const int dm = B - 1 - d;
        const float a = sv[vi].a, m = sv[vi].m, inv_m = sv[vi].inv_m;
        float accA[2] = {0.0f, 0.0f}, accB[2] = {0.0f, 0.0f};   // [0]: ray d, [1]: ray dm
#pragma unroll
        for (int which = 0; which < 2; ++which) {
            if (which == 1 && dm == d) break;
            const int dd = which == 0 ? d : dm;
            const float q = joseph_q(joseph_dp(dd, B), a, hq);
            int lo, hi;
            step_range(q, m, inv_m, h, -2.5f, (float)N + 0.5f, s0, s0 + MR - 1, lo, hi);
            const float qu1 = __fadd_rn(q, m);
            float spk = (float)lo - h;
            int ridx = (lo - s0) * SP;
            float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
            int s = lo;
            for (; s + 1 <= hi; s += 2) {
                const float up0 = joseph_u(spk, m, q), up1 = joseph_u(spk, m, qu1);
                const float t0 = __fadd_rn(up0, JOSEPH_BIAS), t1 = __fadd_rn(up1, JOSEPH_BIAS);
                const unsigned i0 = min((unsigned)(__float_as_int(t0) - (JOSEPH_BIAS_BITS - 2)), top);
                const unsigned i1 = min((unsigned)(__float_as_int(t1) - (JOSEPH_BIAS_BITS - 2)), top);
                const float g0 = __fsub_rn(up0, __fsub_rn(t0, JOSEPH_BIAS));
                const float g1 = __fsub_rn(up1, __fsub_rn(t1, JOSEPH_BIAS));
                const float2 pa0 = PA[ridx + (int)i0], pb0 = PB[ridx + (int)i0];
                const float2 pa1 = PA[ridx + SP + (int)i1], pb1 = PB[ridx + SP + (int)i1];
                a0 += __fmaf_rn(g0, pa0.y, pa0.x);
                b0 += __fmaf_rn(g0, pb0.y, pb0.x);
                a1 += __fmaf_rn(g1, pa1.y, pa1.x);
                b1 += __fmaf_rn(g1, pb1.y, pb1.x);
                spk = __fadd_rn(spk, 2.0f);
                ridx += 2 * SP;
            }
            if (s <= hi) {
                const float up0 = joseph_u(spk, m, q);
                const float t0 = __fadd_rn(up0, JOSEPH_BIAS);
                const unsigned i0 = min((unsigned)(__float_as_int(t0) - (JOSEPH_BIAS_BITS - 2)), top);
                const float g0 = __fsub_rn(up0, __fsub_rn(t0, JOSEPH_BIAS));
                const float2 pa0 = PA[ridx + (int)i0], pb0 = PB[ridx + (int)i0];
                a0 += __fmaf_rn(g0, pa0.y, pa0.x);
                b0 += __fmaf_rn(g0, pb0.y, pb0.x);
            }
            // band A sample of ray dd; band B sample of its mirror ray
            accA[which] = a0 + a1;
            accB[1 - which] = b0 + b1;
        }
        float *o = out + (size_t)svi[vi] * B;
        if (dm == d) {
            o[d] = accA[0] + accB[1];
        } else {
            o[d] = accA[0] + accB[0];
            o[dm] = accA[1] + accB[1];
        }
    }
}

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
template <bool PAIR, int ROWS>
__device__ __forceinline__ float4 quad_walk(const float4 *__restrict__ Q, int SP, float q, float m, int lo, int hi,
                                            int s0, float h, unsigned top)
{
    static_assert(ROWS % 2 == 0, "steps are evaluated in pairs");
    float2 qk[ROWS / 2];   // q + k m for the steps k, k + 1 of a pass
#pragma unroll
    for (int k = 0; k < ROWS / 2; ++k) qk[k] = pk(__fmaf_rn((float)(2 * k), m, q), __fmaf_rn((float)(2 * k + 1), m, q));
    const float2 mm = pk(m, m), bias = pk(JOSEPH_BIAS, JOSEPH_BIAS);
    float spk = (float)lo - h;
    int ridx = (lo - s0) * SP;
    float2 ab[ROWS], ce[ROWS];   // (band A, band B) sums at i0 and at the reflected pair
#pragma unroll
    for (int k = 0; k < ROWS; ++k) ab[k] = ce[k] = pk(0.0f, 0.0f);
    int s = lo;
    for (; s + ROWS - 1 <= hi; s += ROWS) {
#pragma unroll
        for (int k = 0; k < ROWS / 2; ++k) {
            const float2 up = pfma(pk(spk, spk), mm, qk[k]);
            const float2 t = padd(up, bias);
            const float2 tb = psub(t, bias);
            const float2 g = psub(up, tb), gn = psub(tb, up);
            const unsigned i0 = min((unsigned)(__float_as_int(t.x) - (JOSEPH_BIAS_BITS - 2)), top);
            const unsigned i1 = min((unsigned)(__float_as_int(t.y) - (JOSEPH_BIAS_BITS - 2)), top);
            const float4 p0 = Q[ridx + (2 * k) * SP + (int)i0];
            const float4 p1 = Q[ridx + (2 * k + 1) * SP + (int)i1];
            ab[2 * k] = pfma(pk(g.x, g.x), pk(p0.z, p0.w), padd(ab[2 * k], pk(p0.x, p0.y)));
            ab[2 * k + 1] = pfma(pk(g.y, g.y), pk(p1.z, p1.w), padd(ab[2 * k + 1], pk(p1.x, p1.y)));
            if (PAIR) {
                const float4 r0 = Q[ridx + (2 * k) * SP + (int)(top - i0)];
                const float4 r1 = Q[ridx + (2 * k + 1) * SP + (int)(top - i1)];
                ce[2 * k] = pfma(pk(gn.x, gn.x), pk(r0.z, r0.w), padd(ce[2 * k], pk(r0.x, r0.y)));
                ce[2 * k + 1] = pfma(pk(gn.y, gn.y), pk(r1.z, r1.w), padd(ce[2 * k + 1], pk(r1.x, r1.y)));
            }
        }
        spk = __fadd_rn(spk, (float)ROWS);
        ridx += ROWS * SP;
    }
    for (; s <= hi; ++s) {
        const float up = joseph_u(spk, m, qk[0].x);
        const float t = __fadd_rn(up, JOSEPH_BIAS);
        const unsigned i = min((unsigned)(__float_as_int(t) - (JOSEPH_BIAS_BITS - 2)), top);
        const float g = __fsub_rn(up, __fsub_rn(t, JOSEPH_BIAS));
        const float4 pv = Q[ridx + (int)i];
        ab[0] = pfma(pk(g, g), pk(pv.z, pv.w), padd(ab[0], pk(pv.x, pv.y)));
        if (PAIR) {
            const float4 rv = Q[ridx + (int)(top - i)];
            ce[0] = pfma(pk(-g, -g), pk(rv.z, rv.w), padd(ce[0], pk(rv.x, rv.y)));
        }
        spk = __fadd_rn(spk, 1.0f);
        ridx += SP;
    }
#pragma unroll
    for (int k = 1; k < ROWS; ++k) {
        ab[0] = padd(ab[0], ab[k]);
        ce[0] = padd(ce[0], ce[k]);
    }
    return make_float4(ab[0].x, ab[0].y, ce[0].x, ce[0].y);
}

// ROWS = 2: up to 16 items (1024 threads, 64 registers); ROWS = 4: more
// loads in flight per thread, up to 12 items (768 threads, 85 registers).
// DEEP: the staging issues the loads of four pairs per thread before it
// stores them, for grids of few blocks whose threads each stage many pairs
// (few views); otherwise one pair at a time (fewer registers).
template <int ROWS, bool DEEP>
__global__ void __launch_bounds__(ROWS == 2 ? 1024 : 768)
k_project_quad(const float *__restrict__ x, const ViewP *__restrict__ views,
               const int2 *__restrict__ row_items, int n_row, const int2 *__restrict__ col_items, int n_col,
               int N, int V, int B, int pg, float *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int CW = N + 3, SP = CW | 1;
    float4 *Q = reinterpret_cast<float4 *>(smraw);   // [step][pair]: band A pair, band B pair
    ViewP *sv = reinterpret_cast<ViewP *>(Q + (size_t)MR * SP);
    int2 *sit = reinterpret_cast<int2 *>(sv + PG);

    const int bp = blockIdx.x, nbp = gridDim.x;
    const int row_groups = (n_row + pg - 1) / pg;
    const bool rows = (int)blockIdx.y < row_groups;
    const int grp = rows ? blockIdx.y : blockIdx.y - row_groups;
    const int2 *list = rows ? row_items : col_items;
    const int nl = rows ? n_row : n_col;
    const int nv = min(pg, nl - grp * pg);
    const float *img = x + (size_t)blockIdx.z * N * N;
    float *out = partial + ((size_t)blockIdx.z * nbp + bp) * V * B;
    const int s0 = bp * MR;
    const float h = joseph_h(N), hq = joseph_hq(N);
    const int tid = threadIdx.x, nth = blockDim.x;

    if (tid < nv) {
        sit[tid] = list[grp * pg + tid];
        sv[tid] = views[sit[tid].x];
    }
    // pair i (stored at i + 2) of step t: band A the image line s0 + t, band B
    // the line N-1-s0-t read backwards (image value at N-1-i); one thread
    // forms both bands' pairs of (t, i) and stores them as one float4
    if constexpr (DEEP) {
        // the same pairs, each thread issuing the loads of SU of them before
        // it stores any, so that SU L2 round trips overlap
        {
            constexpr int SU = 4;
            const int lx = tid & 31, nw = nth >> 5;
            float a0[SU], a1[SU], b0[SU], b1[SU];
            if (rows) {
                const int nch = (CW + 31) >> 5, nc = MR * nch;
                for (int c0 = tid >> 5; c0 < nc; c0 += SU * nw) {
    #pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const int c = c0 + u * nw;
                        const int t = c / nch, ii = ((c - t * nch) << 5) + lx;
                        const bool ok = c < nc && ii < CW;
                        const int i = ii - 2;
                        const float *ra = img + (size_t)(s0 + t) * N, *rb = img + (size_t)(N - 1 - s0 - t) * N;
                        a0[u] = (ok && i >= 0 && i < N) ? ra[i] : 0.0f;
                        a1[u] = (ok && i + 1 >= 0 && i + 1 < N) ? ra[i + 1] : 0.0f;
                        b0[u] = (ok && N - 1 - i >= 0 && N - 1 - i < N) ? rb[N - 1 - i] : 0.0f;
                        b1[u] = (ok && N - 2 - i >= 0 && N - 2 - i < N) ? rb[N - 2 - i] : 0.0f;
                    }
    #pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const int c = c0 + u * nw;
                        const int t = c / nch, ii = ((c - t * nch) << 5) + lx;
                        if (c < nc && ii < CW)
                            Q[t * SP + ii] = make_float4(0.5f * (a0[u] + a1[u]), 0.5f * (b0[u] + b1[u]),
                                                         a1[u] - a0[u], b1[u] - b0[u]);
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
                            Q[t * SP + ii] = make_float4(0.5f * (a0[u] + a1[u]), 0.5f * (b0[u] + b1[u]),
                                                         a1[u] - a0[u], b1[u] - b0[u]);
                    }
                }
            }
        }
    } else {
        {
            const int lx = tid & 31, nw = nth >> 5;
            if (rows) {
                // warps take 32-pair chunks of the 16 steps, lanes neighbouring pairs
                const int nch = (CW + 31) >> 5;
                for (int c = tid >> 5; c < MR * nch; c += nw) {
                    const int t = c / nch, ii = ((c - t * nch) << 5) + lx;
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
                for (int c = tid >> 5; 2 * c < CW; c += nw) {
                    const int ii = 2 * c + (lx >> 4);
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
    }
    __syncthreads();
    const int npair = (B + 1) / 2;
    const unsigned top = (unsigned)(N + 2);
    const int vi = tid >> 6;
    if (vi >= nv) return;
    const int v = sit[vi].x, vp = sit[vi].y;
    const float a = sv[vi].a, m = sv[vi].m, inv_m = sv[vi].inv_m;
    for (int d = tid & 63; d < npair; d += 64) {
        const int dm = B - 1 - d;
        float ov[2] = {0.0f, 0.0f}, op[2] = {0.0f, 0.0f};   // view v / V-v: [0] ray d, [1] ray dm
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
}

// items per block of k_project_quad: the fewest waves of blocks (one block
// per SM, shared memory) times the per-block work, staging counted as two items
static int quad_pg(const Geometry *g, int batch, int max_pg)
{
    const long bands = g->n / (2 * MR);
    int best = max_pg;
    long best_cost = -1;
    for (int pg = 4; pg <= max_pg; ++pg) {
        const long groups = (g->n_row_items + pg - 1) / pg + (g->n_col_items + pg - 1) / pg;
        const long blocks = bands * groups * batch;
        const long cost = ((blocks + g->n_sm - 1) / g->n_sm) * (pg + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = pg;
        }
    }
    return best;
}

void launch_project_bands(const Geometry *g, const float *x, float *partial, int batch, cudaStream_t st)
{
    const int N = g->n;
    dim3 grd(proj_bands(N), (g->n_row + PG - 1) / PG + (g->n_col + PG - 1) / PG, batch);
    const size_t smem = proj_smem(N);
    counted();
    if (g->vpair && N % (2 * MR) == 0 && N + 3 <= PROJ_CW) {
        // view pairs and two mirrored 16-step bands per block: N/32 partial slots
        const int rows4 = g->tune_qrows == 4;
        const int max_pg = rows4 ? 12 : PG;
        const int pg = g->tune_pg > 0 ? std::min(g->tune_pg, max_pg) : quad_pg(g, batch, max_pg);
        const int groups = (g->n_row_items + pg - 1) / pg + (g->n_col_items + pg - 1) / pg;
        const size_t smem2 = sizeof(float2) * (size_t)2 * MR * ((N + 3) | 1) + sizeof(ViewP) * PG + sizeof(int2) * PG;
        const dim3 grd2(N / (2 * MR), groups, batch);
        // few blocks (few views): each thread stages many pairs, so issue their loads four at a time
        const bool deep = (long)grd2.x * grd2.y * grd2.z < 2L * g->n_sm;
        auto kern = rows4 ? (deep ? k_project_quad<4, true> : k_project_quad<4, false>)
                          : (deep ? k_project_quad<2, true> : k_project_quad<2, false>);
        kern<<<grd2, pg * 64, smem2, st>>>(x, g->d_views, g->d_row_items, g->n_row_items, g->d_col_items,
                                           g->n_col_items, N, g->n_views, g->n_bins, pg, partial);
    } else if (N % (2 * MR) == 0 && N + 3 <= PROJ_CW) {
        // two mirrored 16-step bands per block: N/32 partial slots, as below
        dim3 grd2(N / (2 * MR), grd.y, batch);
        const size_t smem2 = sizeof(float2) * (size_t)2 * MR * ((N + 3) | 1) + sizeof(ViewP) * PG + 64;
        k_project_mirror<<<grd2, PT, smem2, st>>>(x, g->d_views, g->d_row_list, g->n_row, g->d_col_list, g->n_col,
                                                 N, g->n_views, g->n_bins, partial);
    } else if (N + 3 <= PROJ_CW)
        k_project_bands<false><<<grd, PT, smem, st>>>(x, g->d_views, g->d_row_list, g->n_row, g->d_col_list,
                                                      g->n_col, N, g->n_views, g->n_bins, partial);
    else
        k_project_bands<true><<<grd, PT, smem, st>>>(x, g->d_views, g->d_row_list, g->n_row, g->d_col_list,
                                                     g->n_col, N, g->n_views, g->n_bins, partial);
}

// out[v][d] = scale_v * sum_b partial[b][v][d]  (+ residual epilogue)
template <int MODE>
__global__ void k_band_reduce(const float *__restrict__ partial, float *__restrict__ out,
                              const ViewP *__restrict__ views, int nb, int V, int B,
                              const float *__restrict__ b, const float *__restrict__ winv,
                              const float *__restrict__ mu)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y;
    if (d >= B) return;
    const size_t VB = (size_t)V * B;
    const float *p = partial + (size_t)blockIdx.z * nb * VB + (size_t)v * B + d;
    float acc = 0.0f;
    for (int k = 0; k < nb; ++k) acc += p[k * VB];
    const size_t o = (size_t)blockIdx.z * VB + (size_t)v * B + d;
    float val = acc * views[v].scale;
    if (MODE == 1) val = val - b[o] - winv[o] * mu[o];
    else if (MODE == 2) val = val - b[o];
    else if (MODE == 3) val *= (float)(*reinterpret_cast<const double *>(b));
    out[o] = val;
}

void launch_band_reduce(const Geometry *g, const float *partial, float *out, int mode,
                        const float *b, const float *winv, const float *mu, int batch, cudaStream_t st)
{
    dim3 grd((g->n_bins + 255) / 256, g->n_views, batch);
    const int nb = proj_bands(g->n);
    counted();
    if (mode == 0)
        k_band_reduce<0><<<grd, 256, 0, st>>>(partial, out, g->d_views, nb, g->n_views, g->n_bins, b, winv, mu);
    else if (mode == 1)
        k_band_reduce<1><<<grd, 256, 0, st>>>(partial, out, g->d_views, nb, g->n_views, g->n_bins, b, winv, mu);
    else
        k_band_reduce<2><<<grd, 256, 0, st>>>(partial, out, g->d_views, nb, g->n_views, g->n_bins, b, winv, mu);
}

// out = fac * A x from the band partials (fac: one device double)
void launch_band_reduce_scaled(const Geometry *g, const float *partial, float *out, const double *fac, int batch,
                               cudaStream_t st)
{
    dim3 grd((g->n_bins + 255) / 256, g->n_views, batch);
    counted();
    k_band_reduce<3><<<grd, 256, 0, st>>>(partial, out, g->d_views, proj_bands(g->n), g->n_views, g->n_bins,
                                          reinterpret_cast<const float *>(fac), nullptr, nullptr);
}

// =====================================================================
// Backprojection: a pixel-driven gather.  Pixel (r, c) sits at detector
// coordinate e = (c - h) cos t + (r - h) sin t + hb of view t, and ray d
// reaches it with Joseph's weight 1 - |u(d) - j| = 1 - |d - e| |a| (u the
// coordinate along the stepping direction, j the pixel's index along it,
// |a| = 1/max(|cos t|, |sin t|)), non-zero only for d = floor(e) and
// floor(e) + 1.  In exact arithmetic this is the weight the projector
// uses, so A^T is the transpose of A up to the float rounding of the
// weight (a few ulp); every pixel sums its rays in a fixed order, so the
// result is deterministic and needs no atomics.
//
// One block per BT x BT tile.  Views are staged in chunks: per view
// (cos, sin, |a|, 1 - |a|/2) and a window of ray pairs
// (y[d], y[d+1]) * |a| covering the rays that reach the tile.  The block's
// 256 threads form BSL view slices of 64 threads; a thread owns four
// pixels of one row and sums the views of its slice; the slices are added
// in a fixed order at the end.
// =====================================================================
constexpr int BT = 16;          // tile side
constexpr int BSL = 4;          // view slices per block
constexpr int BTH = 64 * BSL;   // threads per block
constexpr int BVC = 64;         // views staged per chunk
constexpr int BWW = 32;         // staged ray pairs per view (>= 15 (|cos|+|sin|) + 3)

template <int MODE>
__global__ void __launch_bounds__(BTH)
k_backproject_tiles(const float *__restrict__ y, float *__restrict__ out,
                    const float4 *__restrict__ trig, int N, int V, int B,
                    const float *__restrict__ xin, const double *__restrict__ scal)
{
    __shared__ float2 tab[BVC][BWW];
    __shared__ float4 sv[BVC];
    __shared__ int wbase[BVC];
    __shared__ float red[BSL][BT * BT];

    const int tid = threadIdx.x;
    const int slice = tid >> 6, l = tid & 63;
    const int R0 = blockIdx.y * BT, C0 = blockIdx.x * BT;
    const int r = R0 + (l >> 2), c0 = C0 + (l & 3) * 4;
    const float *ys = y + (size_t)blockIdx.z * V * B;
    const float h = 0.5f * (float)(N - 1);
    const float hb_lo = 0.5f * (float)(B - 1) - 0.5f;   // e - 1/2 is rounded to find floor(e)
    const float yr = (float)r - h;
    float xc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) xc[k] = (float)(c0 + k) - h;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};

    for (int v0 = 0; v0 < V; v0 += BVC) {
        const int nv = min(BVC, V - v0);
        __syncthreads();
        if (tid < nv) {
            const float4 T = trig[v0 + tid];   // cos, sin, |a|, 1 - |a|/2
            sv[tid] = T;
            // lowest detector coordinate over the tile corners
            float emin = 3.0e38f;
#pragma unroll
            for (int cr = 0; cr < 4; ++cr) {
                const float xx = (float)(C0 + (cr & 1) * (BT - 1)) - h;
                const float yy = (float)(R0 + (cr >> 1) * (BT - 1)) - h;
                emin = fminf(emin, xx * T.x + yy * T.y);
            }
            emin = fminf(fmaxf(emin + 0.5f * (float)(B - 1), -1.0e6f), 1.0e6f);
            wbase[tid] = (int)floorf(emin) - 2;
        }
        __syncthreads();
        for (int k = tid; k < nv * BWW; k += BTH) {
            const int vi = k / BWW, w = k - vi * BWW;
            const int d = wbase[vi] + w;
            const float *yv = ys + (size_t)(v0 + vi) * B;
            const float sc = sv[vi].z;
            const float y0 = (d >= 0 && d < B) ? yv[d] : 0.0f;
            const float y1 = (d + 1 >= 0 && d + 1 < B) ? yv[d + 1] : 0.0f;
            tab[vi][w] = make_float2(y0 * sc, y1 * sc);
        }
        __syncthreads();
        if (r < N) {
            for (int vi = slice; vi < nv; vi += BSL) {
                const float4 T = sv[vi];
                const int fb = JOSEPH_BIAS_BITS + wbase[vi];
                const float eb = fmaf(yr, T.y, hb_lo);
                const float2 *tv = tab[vi];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float e = fmaf(xc[k], T.x, eb);               // e - 1/2
                    const float t = __fadd_rn(e, JOSEPH_BIAS);
                    // floor(e) - wbase, kept inside the staged window
                    const unsigned f = min((unsigned)(__float_as_int(t) - fb), (unsigned)(BWW - 1));
                    const float g = __fsub_rn(e, __fsub_rn(t, JOSEPH_BIAS));   // frac(e) - 1/2
                    const float w0 = fmaxf(0.0f, fmaf(-g, T.z, T.w));   // 1 - frac |a|
                    const float w1 = fmaxf(0.0f, fmaf(g, T.z, T.w));    // 1 - (1 - frac) |a|
                    const float2 yy = tv[f];
                    acc[k] = fmaf(w0, yy.x, fmaf(w1, yy.y, acc[k]));
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[slice][(l >> 2) * BT + (l & 3) * 4 + k] = acc[k];
    __syncthreads();
    if (tid < BT * BT) {
        const int rr = R0 + tid / BT, cc = C0 + tid % BT;
        if (rr < N && cc < N) {
            float tot = red[0][tid];
#pragma unroll
            for (int k = 1; k < BSL; ++k) tot += red[k][tid];
            const size_t o = (size_t)blockIdx.z * N * N + (size_t)rr * N + cc;
            if (MODE == 0) out[o] = tot;
            else out[o] = xin[o] - fscal(scal, F_TAU) * tot;
        }
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
// nsl slices (grid.z; 4 unless tuned, at most ORB_SL_MAX); each slice
// writes its own partial image and k_orbit_reduce adds the slices in a
// fixed order.  The weights are the
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

// AL: B % 4 == 0 and y 16-byte aligned, so every window (its base a
// multiple of 4) is copied in aligned 16-byte pieces, each wholly on or
// wholly off the detector.
template <bool AL>
__global__ void __launch_bounds__(ORB_TH, 8)
k_backproject_orbit(const float *__restrict__ y, float *__restrict__ partial, const float4 *__restrict__ trig,
                    int N, int V, int B, int nsl, int fin, float *out, const float *xin,
                    const double *__restrict__ scal)
{
    // raw[buffer][view][row (v, v+V/2)][window (e, mirror e, e90, mirror e90)][value]
    extern __shared__ __align__(16) unsigned char osm[];
    float *raw = reinterpret_cast<float *>(osm);                               // 2 x ORB_VC x 8 x ORB_RW
    float4 *tt = reinterpret_cast<float4 *>(raw + 2 * ORB_VC * 8 * ORB_RW);    // 2 x ORB_VC
    int *wbs = reinterpret_cast<int *>(tt + 2 * ORB_VC);                       // ORB_MAXS x 2
    const int tid = threadIdx.y * ORB_T + threadIdx.x;   // threadIdx.y < ORB_TY
    const int half = N / 2, V2 = V / 2;
    const int slice = blockIdx.z % nsl, img = blockIdx.z / nsl;
    const int r0 = blockIdx.y * ORB_T, c0 = half + blockIdx.x * ORB_T;   // quadrant r < N/2, c >= N/2
    const int r = r0 + threadIdx.y, c = c0 + threadIdx.x;            // pixels (r + j ORB_TY, c)
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
    __syncthreads();

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
        __syncthreads();
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
        __syncthreads();   // the buffer is refilled two chunks later
    }
    // fin 0: the slice's partial image; with a single slice the sums are
    // complete and the block writes k_orbit_reduce's result itself: fin 1
    // out = sum, fin 2 out = xin - tau sum
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
            for (int k = 0; k < 4; ++k) pp[o[k]] = fin == 2 ? xq0[o[k]] - tau * acc[j][k] : acc[j][k];
        }
    }
}

static size_t orbit_smem()
{
    return sizeof(float) * 2 * ORB_VC * 8 * ORB_RW + sizeof(float4) * 2 * ORB_VC + sizeof(int) * 2 * ORB_MAXS;
}

// out = sum of the slice images (mode 0), or xin - tau * sum (mode 1)
template <int MODE>
__global__ void k_orbit_reduce(const float *__restrict__ partial, float *__restrict__ out, const float *xin,
                               const double *__restrict__ scal, size_t NN, int nsl)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= NN) return;
    const float *pp = partial + (size_t)blockIdx.y * nsl * NN + i;
    float t = pp[0];
    for (int s = 1; s < nsl; ++s) t += pp[s * NN];
    const size_t o = (size_t)blockIdx.y * NN + i;
    if (MODE == 0) out[o] = t;
    else out[o] = xin[o] - fscal(scal, F_TAU) * t;
}

bool orbit_ok(const Geometry *g) { return g->orbit; }
size_t orbit_partial_floats(const Geometry *g, int batch) { return (size_t)ORB_SL_MAX * g->n * g->n * batch; }

// base-view slices of the orbit kernel: a slice holds at most ORB_MAXS base views
bool orbit_slices_ok(const Geometry *g, int nsl)
{
    return nsl >= 1 && nsl <= ORB_SL_MAX && (g->n_views / 2 + nsl - 1) / nsl <= ORB_MAXS;
}
static int orbit_slices(const Geometry *g) { return g->tune_orb > 0 ? g->tune_orb : ORB_SL; }

void launch_backproject_orbit(const Geometry *g, const float *y, float *out, int mode, const float *xin,
                              const double *scal, int batch, float *partial, cudaStream_t st)
{
    const int q = g->n / 2;
    const int nsl = orbit_slices(g);
    dim3 grd((q + ORB_T - 1) / ORB_T, (q + ORB_T - 1) / ORB_T, nsl * batch);
    // one slice: the orbit kernel writes the result (the same arithmetic as
    // k_orbit_reduce with one slice), and no reduction pass runs
    const int fin = nsl == 1 ? 1 + (mode != 0) : 0;
    counted(fin ? 1 : 2);
    if (g->n_bins % 4 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0)
        k_backproject_orbit<true><<<grd, dim3(ORB_T, ORB_TY), orbit_smem(), st>>>(
            y, partial, g->d_trig, g->n, g->n_views, g->n_bins, nsl, fin, out, xin, scal);
    else
        k_backproject_orbit<false><<<grd, dim3(ORB_T, ORB_TY), orbit_smem(), st>>>(
            y, partial, g->d_trig, g->n, g->n_views, g->n_bins, nsl, fin, out, xin, scal);
    if (fin) return;
    const size_t NN = (size_t)g->n * g->n;
    dim3 g2((unsigned)((NN + 255) / 256), batch);
    if (mode == 0) k_orbit_reduce<0><<<g2, 256, 0, st>>>(partial, out, xin, scal, NN, nsl);
    else k_orbit_reduce<1><<<g2, 256, 0, st>>>(partial, out, xin, scal, NN, nsl);
}

void launch_backproject(const Geometry *g, const float *y, float *out, int mode,
                        const float *xin, const double *scal, int batch, cudaStream_t st)
{
    dim3 grd((g->n + BT - 1) / BT, (g->n + BT - 1) / BT, batch);
    counted();
    if (mode == 0)
        k_backproject_tiles<0><<<grd, BTH, 0, st>>>(y, out, g->d_trig, g->n, g->n_views, g->n_bins, xin, scal);
    else
        k_backproject_tiles<1><<<grd, BTH, 0, st>>>(y, out, g->d_trig, g->n, g->n_views, g->n_bins, xin, scal);
}

void kernel_attrs_joseph()
{
    cudaFuncSetAttribute(k_backproject_orbit<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)orbit_smem());
    cudaFuncSetAttribute(k_backproject_orbit<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)orbit_smem());
    cudaFuncSetAttribute(k_project_mirror, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_bands<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_bands<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
}

}  // namespace ctpd
