// k_joseph.cu -- Joseph forward projector A (ray-driven) and its transpose
// A^T (pixel-driven gather), the A and A^T of Eqs. 18-20 / 29-31.  Both are
// deterministic (fixed summation orders, no atomics).
#include <algorithm>
#include <cmath>
#include <vector>

#include <cooperative_groups.h>

#include "body_joseph.cuh"

namespace ctpd {


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
constexpr int PT = 1024;       // threads per block
constexpr int PROJ_CW = 640;   // pairs per staged band row

static int proj_cw(int n) { return (n + 3) < PROJ_CW ? (n + 3) : PROJ_CW; }
static int proj_stride(int n) { return proj_cw(n) | 1; }   // odd: spreads smem banks
static size_t proj_smem(int n) { return sizeof(float2) * (size_t)PROJ_R * proj_stride(n) + sizeof(ViewP) * PG + 64; }

__device__ __forceinline__ int d_proj_cw(int n) { return (n + 3) < PROJ_CW ? (n + 3) : PROJ_CW; }

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

// ROWS = 2: up to 16 items (1024 threads, 64 registers); ROWS = 4: more
// loads in flight per thread, up to 12 items (768 threads, 85 registers).
// DEEP: the staging issues the loads of four pairs per thread before it
// stores them, for grids of few blocks whose threads each stage many pairs
// (few views); otherwise one pair at a time (fewer registers).
template <int ROWS, bool DEEP>
__global__ void __launch_bounds__(ROWS == 2 ? 1024 : 768)
k_project_quad(const float *__restrict__ x, const ViewP *__restrict__ views,
               const int2 *__restrict__ row_items, int n_row, const int2 *__restrict__ col_items, int n_col,
               int N, int V, int B, int pg, int gpb, float *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    pdl_wait();
    quad_body<ROWS, DEEP>(whole_block(), blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, smraw, x, views, row_items,
                          n_row, col_items, n_col, N, V, B, pg, gpb, partial);
}

// The work-balanced form: block b takes units [total b / nb, total (b+1) / nb)
// (see quad_balanced_body); its unit counter sits after the staged pairs.
__device__ __forceinline__ unsigned long long global_time()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounds (optional): block b takes units [bounds[b], bounds[b+1]), a table
// of the geometry's written before any launch that reads it (so it is read
// before the wait for the previous kernel); else equal unit counts.
// times (optional): block b writes its start and end times (ns) to
// times[2b], times[2b+1].
template <int ROWS, bool DEEP>
__global__ void __launch_bounds__(ROWS == 2 ? 1024 : 768)
k_project_qbal(const float *__restrict__ x, const ViewP *__restrict__ views, const int2 *__restrict__ row_items,
               const int2 *__restrict__ col_items, int N, int V, int B, QuadUnits U, long long total,
               const long long *__restrict__ bounds, unsigned long long *__restrict__ times,
               float *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const long long nb = gridDim.x;
    long long u0, u1;
    if (bounds) {   // clamped: a table is never read outside [0, total)
        u0 = min(max(bounds[blockIdx.x], 0LL), total);
        u1 = min(max(bounds[blockIdx.x + 1], u0), total);
    } else {
        u0 = total * blockIdx.x / nb;
        u1 = total * (blockIdx.x + 1) / nb;
    }
    pdl_wait();
    const unsigned long long t0 = times ? global_time() : 0ull;
    quad_balanced_body<ROWS, DEEP>(whole_block(), u0, u1, U, smraw, reinterpret_cast<int *>(smraw + quad_smem(N)),
                                   x, views, row_items, col_items, N, V, B, partial);
    if (times) {
        __syncthreads();
        if (threadIdx.x == 0) {
            times[2 * blockIdx.x] = t0;
            times[2 * blockIdx.x + 1] = global_time();
        }
    }
}

// Launch shape of k_project_quad: items per group (pg, 64 threads each) and
// groups per block (gpb, walked one after the other on one staged band
// pair), by the fewest waves of blocks (one block per SM, shared memory)
// times the per-block work, staging counted as three items.  pg_fixed > 0
// fixes pg (the tuner's choice) and picks gpb for it.
static void quad_shape(const Geometry *g, int batch, int max_pg, int pg_fixed, int *pg_out, int *gpb_out)
{
    const long bands = g->n / (2 * MR);
    long best_cost = -1;
    for (int pg = pg_fixed > 0 ? pg_fixed : 4; pg <= (pg_fixed > 0 ? pg_fixed : max_pg); ++pg) {
        const long rg = (g->n_row_items + pg - 1) / pg, cg = (g->n_col_items + pg - 1) / pg;
        for (int gpb = 1; gpb <= 8; ++gpb) {
            const long blocks = bands * ((rg + gpb - 1) / gpb + (cg + gpb - 1) / gpb) * batch;
            const long cost = ((blocks + g->n_sm - 1) / g->n_sm) * ((long)gpb * pg + 3);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                *pg_out = pg;
                *gpb_out = gpb;
            }
        }
    }
}

// Launch shape of the work-balanced form: as many blocks as fit on the
// device at once (fewer when the work would leave a warp under two units).
struct QbalShape {
    QuadUnits U;
    long long total;
    int rows4, pgb, threads, blocks, key;
    size_t smem;
};
static QbalShape qbal_shape(const Geometry *g, int batch)
{
    QbalShape q;
    const int N = g->n;
    q.rows4 = g->tune_qrows == 4;
    const int max_pg = q.rows4 ? 12 : PG;
    q.pgb = g->tune_pg > 0 ? std::min(g->tune_pg, max_pg) : max_pg;
    q.threads = q.pgb * 64;
    q.key = 64 * q.rows4 + q.pgb;
    const int npair = (g->n_bins + 1) / 2, nch = (npair + 63) / 64;
    q.U.nch = nch;
    q.U.u_rows = g->n_row_items * nch;
    q.U.u_cols = g->n_col_items * nch;
    q.U.u_z = (long long)(N / (2 * MR)) * (q.U.u_rows + q.U.u_cols);
    q.total = q.U.u_z * batch;
    q.smem = quad_smem(N) + 16;
    auto kern = q.rows4 ? k_project_qbal<4, true> : k_project_qbal<2, true>;
    // blocks per SM, queried once per (steps per pass, items) for the geometry
    int &occ_slot = const_cast<Geometry *>(g)->qbal_occ[q.rows4][q.pgb];
    int occ = occ_slot;
    if (occ < 1) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, q.threads, q.smem) != cudaSuccess || occ < 1)
            occ = 1;
        occ_slot = occ;
    }
    const long long by_work = (q.total + 4 * q.pgb - 1) / (4 * q.pgb);   // two units per warp
    q.blocks = (int)std::max(1LL, std::min((long long)g->n_sm * occ, by_work));
    return q;
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
        int pg = 0, gpb = 1;
        quad_shape(g, batch, max_pg, g->tune_pg > 0 ? std::min(g->tune_pg, max_pg) : 0, &pg, &gpb);
        const int rg = (g->n_row_items + pg - 1) / pg, cg = (g->n_col_items + pg - 1) / pg;
        const int blocks_y = (rg + gpb - 1) / gpb + (cg + gpb - 1) / gpb;
        const dim3 grd2(N / (2 * MR), blocks_y, batch);
        const long static_blocks = (long)grd2.x * grd2.y * grd2.z;
        // the built-in rule takes the work-balanced form when one band pair
        // per block would need two waves of blocks or more
        if (g->tune_qbal == 2 || (g->tune_qbal == 0 && static_blocks >= 2L * g->n_sm)) {
            const QbalShape q = qbal_shape(g, batch);
            auto kern = q.rows4 ? k_project_qbal<4, true> : k_project_qbal<2, true>;
            // the tuner's measured-balance ranges, for the launch they were made for
            const long long *bounds =
                batch == 1 && g->d_qbounds && g->qbounds_nb > 0 && g->qbounds_nb == q.blocks && g->qbounds_key == q.key
                    ? g->d_qbounds
                    : nullptr;
            launch_kernel(kern, dim3(q.blocks), dim3(q.threads), q.smem, st, x, g->d_views, g->d_row_items,
                          g->d_col_items, N, g->n_views, g->n_bins, q.U, q.total, bounds, g->d_qtimes, partial);
            return;
        }
        const size_t smem2 = quad_smem(N);
        // few blocks (few views): each thread stages many pairs, so issue their loads four at a time
        const bool deep = static_blocks < 2L * g->n_sm;
        auto kern = rows4 ? (deep ? k_project_quad<4, true> : k_project_quad<4, false>)
                          : (deep ? k_project_quad<2, true> : k_project_quad<2, false>);
        launch_kernel(kern, grd2, dim3(pg * 64), smem2, st, x, g->d_views, g->d_row_items, g->n_row_items,
                      g->d_col_items, g->n_col_items, N, g->n_views, g->n_bins, pg, gpb, partial);
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

// AL: B % 4 == 0 and y 16-byte aligned, so every window (its base a
// multiple of 4) is copied in aligned 16-byte pieces, each wholly on or
// wholly off the detector.
template <bool AL>
__global__ void __launch_bounds__(ORB_TH, 8)
k_backproject_orbit(const float *__restrict__ y, float *__restrict__ partial, const float4 *__restrict__ trig,
                    int N, int V, int B, int nsl, int fin, float *out, const float *xin,
                    const double *__restrict__ scal)
{
    extern __shared__ __align__(16) unsigned char osm[];
    pdl_wait();
    orbit_body<AL>(Block2D{}, blockIdx.x, blockIdx.y, blockIdx.z, osm, y, partial, trig, N, V, B, nsl, fin, out, xin,
                   scal);
}

// The orbit backprojector with its base-view slices added in a thread-block
// cluster: the nsl blocks of one tile (grid.z = images x slices, cluster
// (1, 1, nsl)) each leave their partial sums in shared memory; block s then
// adds, for its share of the tile's 4 ORB_PX ORB_TH sums, the nsl partials
// in slice order through distributed shared memory and writes the sum
// (mode 0) or xin - tau sum (mode 1).  No slice images are written, and no
// reduction pass runs.
template <bool AL>
__global__ void __launch_bounds__(ORB_TH, 8)
k_backproject_orbit_cl(const float *__restrict__ y, const float4 *__restrict__ trig, int N, int V, int B, int nsl,
                       int mode, float *out, const float *xin, const double *__restrict__ scal)
{
    extern __shared__ __align__(16) unsigned char osm[];
    pdl_wait();
    orbit_body<AL, Block2D, true>(Block2D{}, blockIdx.x, blockIdx.y, blockIdx.z, osm, y, nullptr, trig, N, V, B, nsl, 0,
                                  nullptr, nullptr, scal);
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();   // every slice's partial sums are in its shared memory
    const int slice = blockIdx.z % nsl, img = blockIdx.z / nsl;   // the block's rank in its cluster
    float *red = reinterpret_cast<float *>(osm);
    constexpr int E = 4 * ORB_PX * ORB_TH;
    const int e0 = E * slice / nsl, e1 = E * (slice + 1) / nsl;
    const int half = N / 2;
    const float tau = mode ? fscal(scal, F_TAU) : 0.0f;
    float *o_img = out + (size_t)img * N * N;
    const float *x_img = mode ? xin + (size_t)img * N * N : nullptr;
    for (int e = e0 + (int)(threadIdx.y * blockDim.x + threadIdx.x); e < e1; e += ORB_TH) {
        float t = *cl.map_shared_rank(red + e, 0);
        for (int s = 1; s < nsl; ++s) t += *cl.map_shared_rank(red + e, s);
        const int k = e / (ORB_PX * ORB_TH), rem = e - k * (ORB_PX * ORB_TH);
        const int j = rem / ORB_TH, th = rem - j * ORB_TH;
        const int rj = blockIdx.y * ORB_T + th / ORB_T + j * ORB_TY, c = half + blockIdx.x * ORB_T + th % ORB_T;
        if (rj < half && c < N) {
            const size_t o = k == 0   ? (size_t)rj * N + c
                             : k == 1 ? (size_t)c * N + (N - 1 - rj)
                             : k == 2 ? (size_t)(N - 1 - rj) * N + (N - 1 - c)
                                      : (size_t)(N - 1 - c) * N + rj;
            o_img[o] = mode ? __fmaf_rn(-tau, t, x_img[o]) : t;
        }
    }
    cl.sync();   // no block leaves while its partial sums may still be read
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
    pdl_wait();
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= NN) return;
    const float *pp = partial + (size_t)blockIdx.y * nsl * NN + i;
    float t = pp[0];
    for (int s = 1; s < nsl; ++s) t += pp[s * NN];
    const size_t o = (size_t)blockIdx.y * NN + i;
    if (MODE == 0) out[o] = t;
    else out[o] = __fmaf_rn(-fscal(scal, F_TAU), t, xin[o]);   // one rounding, as every form of z
}

bool orbit_ok(const Geometry *g) { return g->orbit; }
size_t orbit_partial_floats(const Geometry *g, int batch) { return (size_t)ORB_SL_MAX * g->n * g->n * batch; }

// base-view slices of the orbit kernel: a slice holds at most ORB_MAXS base views
bool orbit_slices_ok(const Geometry *g, int nsl)
{
    return nsl >= 1 && nsl <= ORB_SL_MAX && (g->n_views / 2 + nsl - 1) / nsl <= ORB_MAXS;
}
int orbit_slices(const Geometry *g, bool cluster)
{
    const int t = cluster ? g->tune_orb : g->tune_orb_si;
    return t > 0 ? t : ORB_SL;
}
size_t orbit_smem_bytes() { return orbit_smem(); }
bool quad_ok(const Geometry *g) { return g->vpair && g->n % (2 * MR) == 0 && g->n + 3 <= PROJ_CW; }

// Measured balance of the work-balanced projector for one image.  Equal
// unit counts per block leave the blocks' times about 20 % apart at
// 512^2 / 720 views (views whose rays cross fewer staged steps, bank
// conflicts that differ by view, the two line classes), and the launch
// lasts as long as its slowest block.  The tuner keeps a cost per unit,
// uniform at first.  Each round times every block of a few launches
// (%globaltimer at its start and end), scales the costs of each block's
// units by (measured / modelled time)^0.7, and cuts the units again at
// equal shares of the modelled cost; as the ranges move between rounds the
// model resolves finer than one block.  The ranges of the round whose
// launch time (CUDA events) is least are kept, if they beat equal counts.
// A range only decides which block forms which units' sums, so results do
// not change.  The geometry's table (QB_CAP entries) is allocated once and
// kept until the geometry is destroyed, so that a graph captured before a
// later tuning never reads freed memory (and the kernel clamps what it
// reads); the rounds run on a scratch table.
constexpr int QB_CAP = 4096;
ct_status qbal_balance(Geometry *g, const float *x, float *band, cudaStream_t st)
{
    g->qbounds_nb = 0;   // no table until a better one is written
    if (!quad_ok(g) || g->tune_qbal != 2) return CT_OK;
    const QbalShape q = qbal_shape(g, 1);
    const int nb = q.blocks;
    if (nb < 2 || nb + 1 > QB_CAP) return CT_OK;
    const long long uz = q.U.u_z;
    unsigned long long *times = nullptr;
    long long *bounds = nullptr, *keep = g->d_qbounds;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    if (!keep) {
        e = cudaMalloc(&keep, sizeof(long long) * QB_CAP);
        if (e == cudaSuccess) g->d_qbounds = keep;
    }
    if (e == cudaSuccess) e = cudaMalloc(&times, sizeof(unsigned long long) * 2 * nb);
    if (e == cudaSuccess) e = cudaMalloc(&bounds, sizeof(long long) * (nb + 1));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    std::vector<long long> b(nb + 1), best;
    for (int i = 0; i <= nb; ++i) b[i] = uz * i / nb;
    std::vector<unsigned long long> h(2 * nb);
    std::vector<double> dur(nb), cost((size_t)uz, 1.0), cum((size_t)uz + 1);
    float best_ms = -1.0f;
    // the mean time of 8 launches with the current table (none: equal counts)
    auto time_it = [&](float &ms) {
        launch_project_bands(g, x, band, 1, st);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 8; ++r) launch_project_bands(g, x, band, 1, st);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms /= 8.0f;
    };
    if (e == cudaSuccess) time_it(best_ms);
    g->qbounds_key = q.key;
    for (int round = 0; round < 12 && e == cudaSuccess; ++round) {
        // block times of four launches with the current ranges
        e = cudaMemcpy(bounds, b.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice);
        g->d_qbounds = bounds;   // the scratch table for the rounds' launches
        g->qbounds_nb = nb;
        g->d_qtimes = times;
        std::fill(dur.begin(), dur.end(), 0.0);
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
            launch_project_bands(g, x, band, 1, st);
            e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) e = cudaMemcpy(h.data(), times, sizeof(unsigned long long) * 2 * nb,
                                                 cudaMemcpyDeviceToHost);
            for (int i = 0; i < nb && e == cudaSuccess; ++i) dur[i] += (double)(h[2 * i + 1] - h[2 * i]);
        }
        g->d_qtimes = nullptr;
        if (e != cudaSuccess) break;
        // scale each block's unit costs towards its measured time, then cut
        // the units at equal shares of the modelled cost
        for (int i = 0; i < nb; ++i) {
            double model = 0.0;
            for (long long u = b[i]; u < b[i + 1]; ++u) model += cost[(size_t)u];
            if (model <= 0.0 || b[i + 1] == b[i]) continue;
            const double f = std::pow(std::max(dur[i], 1.0) / model, 0.7);
            for (long long u = b[i]; u < b[i + 1]; ++u) cost[(size_t)u] *= f;
        }
        cum[0] = 0.0;
        for (long long u = 0; u < uz; ++u) cum[(size_t)u + 1] = cum[(size_t)u] + cost[(size_t)u];
        b[0] = 0;
        b[nb] = uz;
        for (int k = 1; k < nb; ++k) {
            const double t = cum[(size_t)uz] * k / nb;
            const long long u = (long long)(std::lower_bound(cum.begin(), cum.end(), t) - cum.begin());
            b[k] = std::min(uz, std::max(b[k - 1], u));
        }
        e = cudaMemcpy(bounds, b.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice);
        float ms = -1.0f;
        if (e == cudaSuccess) time_it(ms);
        if (e == cudaSuccess && ms > 0.0f && ms < best_ms) {
            best_ms = ms;
            best = b;
        }
    }
    g->d_qtimes = nullptr;
    g->d_qbounds = keep;
    g->qbounds_nb = 0;
    if (e == cudaSuccess && !best.empty() && keep) {
        e = cudaMemcpy(keep, best.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) g->qbounds_nb = nb;
    }
    if (bounds) cudaFree(bounds);
    if (times) cudaFree(times);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("ct_geometry_autotune: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA;
    }
    return CT_OK;
}

void launch_backproject_orbit(const Geometry *g, const float *y, float *out, int mode, const float *xin,
                              const double *scal, int batch, float *partial, cudaStream_t st, bool cluster)
{
    const int q = g->n / 2;
    const bool cl = cluster || !partial;
    const int nsl = orbit_slices(g, cl);
    dim3 grd((q + ORB_T - 1) / ORB_T, (q + ORB_T - 1) / ORB_T, nsl * batch);
    const bool al = g->n_bins % 4 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0;
    if (nsl > 1 && cl) {
        // several slices: their sums are added in a cluster of the slices' blocks
        counted();
        launch_kernel_cluster(al ? k_backproject_orbit_cl<true> : k_backproject_orbit_cl<false>, grd,
                              dim3(ORB_T, ORB_TY), orbit_smem(), st, dim3(1, 1, nsl), y, (const float4 *)g->d_trig,
                              g->n, g->n_views, g->n_bins, nsl, mode != 0 ? 1 : 0, out, xin, scal);
        return;
    }
    // one slice: the block's sums are complete and it writes the result;
    // several slices without a cluster: slice images, then k_orbit_reduce
    const int fin = nsl == 1 ? 1 + (mode != 0) : 0;
    counted(fin ? 1 : 2);
    launch_kernel(al ? k_backproject_orbit<true> : k_backproject_orbit<false>, grd, dim3(ORB_T, ORB_TY), orbit_smem(),
                  st, y, partial, g->d_trig, g->n, g->n_views, g->n_bins, nsl, fin, out, xin, scal);
    if (fin) return;
    const size_t NN = (size_t)g->n * g->n;
    launch_kernel(mode == 0 ? k_orbit_reduce<0> : k_orbit_reduce<1>, dim3((unsigned)((NN + 255) / 256), batch),
                  dim3(256), 0, st, (const float *)partial, out, xin, scal, NN, nsl);
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
    cudaFuncSetAttribute(k_backproject_orbit_cl<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)orbit_smem());
    cudaFuncSetAttribute(k_backproject_orbit_cl<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)orbit_smem());
    cudaFuncSetAttribute(k_project_mirror, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_quad<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_qbal<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_qbal<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_bands<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
    cudaFuncSetAttribute(k_project_bands<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem(8192));
}

}  // namespace ctpd
