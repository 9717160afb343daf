// persist.cu -- the iterations of a batched solve in one persistent launch.
//
// Each slice's iteration (Steps 1-3 of Algorithm 1 / Algorithm 2, Secs. 2.3
// and 3) is a chain of phases: A^T with the primal step (orbit tiles, plus
// the slice reduction when the base views are split), the TV prox (tiles),
// A (ranges of band pair x view pair x ray units) and the dual update with the next
// Step 1 (view pairs).  A phase of one slice may start only when the
// slice's previous phase is complete; different slices are independent.
//
// One block per SM takes work items from a single queue in the order
// (iteration, phase, slice, item), so every item depends only on items of
// its slice with smaller queue numbers.  Those were taken earlier by blocks
// that are running, so the items complete in queue order without any
// block waiting on one that has not started, whatever the residency.
// Before it runs an item, one thread of the block waits until the slice's
// completed-item counter reaches the count of the slice's earlier phases:
// a bounded spin on the global timer.  When the limit runs out (or another
// block reported that), the block sets the batch's error word, marks every
// slice's check flags with CHK_TIMEOUT and leaves; every block leaves at
// its next item once the error word is set, so the launch always ends.
// After an item the block's threads meet at a barrier and one thread
// publishes the completion with a fence and an atomic increment (release);
// the waiting thread's fence after the spin (acquire) and the block barrier
// make the slice's finished writes visible to the block's loads.
//
// The item bodies are those of the single-slice kernels (body_*.cuh), run
// by the whole 1024-thread block (the work-balanced projector's unit ranges) or
// by groups with their own named barriers (eight 128-thread orbit tiles,
// four 256-thread view pairs of the dual update, two 512-thread TV tiles),
// so A, A^T and the dual update keep the 32 warps per SM of their own
// kernels; the block's 64 registers per thread are fewer than the TV
// prox's own kernel uses, so the prox here holds regions of 48 rows.  All counters live in the slices' scalar blocks,
// which each slice's setup clears.
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>

#include "body_fft.cuh"
#include "body_joseph.cuh"
#include "body_tv.cuh"

namespace ctpd {

namespace {

constexpr int PS_THREADS = 1024;
constexpr int PS_MAX = 96;                         // slices per launch (kernel parameter space)
enum { PH_ORBIT = 0, PH_OREDUCE, PH_TV, PH_QUAD, PH_DUAL, PH_N };
constexpr int ORB_GROUPS = PS_THREADS / ORB_TH;    // orbit tiles per item
constexpr int DUAL_GROUPS = PS_THREADS / FFT_T;    // view pairs per item
constexpr int RED_PIX = PS_THREADS * 8;            // pixels per slice-reduction item
constexpr int QUAD_PG = PS_THREADS / 64;           // projector view-pair items per block
constexpr int TV_GROUPS = PS_THREADS / TV_THREADS; // TV tiles per item
// rows per warp of the prox's region here: three (48 rows) rather than the
// prox kernel's five, so that its cells fit the 64 registers a thread of a
// 1024-thread block has (with five they spill), at more halo work
constexpr int PS_TV_J = 3;
constexpr int PS_TV_PUB = (TV_WARPS * PS_TV_J + 2) * 32;   // float2 per published field
static_assert(TV_GROUPS * TV_THREADS == PS_THREADS && QUAD_PG == PG, "whole groups");
static_assert(1 + ORB_GROUPS + DUAL_GROUPS + TV_GROUPS <= 16, "named barriers 1..15");
static_assert(ORB_GROUPS * ORB_TH == PS_THREADS && DUAL_GROUPS * FFT_T == PS_THREADS, "whole groups");

struct PSlice {
    int N, V, B, P, nb, lowdose, al;
    int n_row_items, n_col_items, qseg;   // qseg: one projector item per staged band pair (segment)
    int nsl, q16, orb_smem, dual_smem;
    int tv_tc, tv_tr, tv_ncb, tv_nrb, ntv, fgp;
    int n_items[PH_N], pre[PH_N], per_iter;
    const ViewP *views;
    const int2 *row_items, *col_items;
    const float4 *trig;
    const float2 *tw, *hhat;
    const float *b, *winv;
    float *mu, *mubar, *x, *z, *p[2], *band, *orb;
    double *scal;
};

struct PParams {
    int n, K, R, total;
    unsigned long long wait_ns;
    int phase_off[PH_N + 1];
    int slice_off[PH_N][PS_MAX + 1];
    PSlice sl[PS_MAX];
};
static_assert(sizeof(PParams) <= 32000, "the launch's parameters must fit the kernel parameter space");

__device__ __forceinline__ unsigned *pslot(double *scal, int k) { return reinterpret_cast<unsigned *>(scal + k); }

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One work item of slice S: phase p of iteration k, item i of the phase.
__device__ __forceinline__ void run_item(const PSlice &S, int p, int k, int i, unsigned char *psm)
{
    const int tid = threadIdx.x;
    if (p == PH_ORBIT) {
        // z = x - tau A^T mu_bar (one slice), or the slices' partial images
        const int g = tid / ORB_TH, j = i * ORB_GROUPS + g, per = S.q16 * S.q16;
        if (j < per * S.nsl) {
            const int bz = j / per, rem = j - bz * per, by = rem / S.q16, bx = rem - by * S.q16;
            const GroupCtx c{tid % ORB_TH, ORB_TH, 1 + g};
            unsigned char *sm = psm + (size_t)g * S.orb_smem;
            const int fin = S.nsl == 1 ? 2 : 0;
            if (S.al)
                orbit_body<true>(c, bx, by, bz, sm, S.mubar, S.orb, S.trig, S.N, S.V, S.B, S.nsl, fin, S.z, S.x,
                                 S.scal);
            else
                orbit_body<false>(c, bx, by, bz, sm, S.mubar, S.orb, S.trig, S.N, S.V, S.B, S.nsl, fin, S.z, S.x,
                                  S.scal);
        }
    } else if (p == PH_OREDUCE) {
        // z = x - tau * (the slices' partial images added in slice order)
        const size_t NN = (size_t)S.N * S.N;
        const float tau = fscal(S.scal, F_TAU);
        for (size_t q = (size_t)i * RED_PIX + tid; q < NN && q < (size_t)(i + 1) * RED_PIX; q += PS_THREADS) {
            const float *pp = S.orb + q;
            float t = pp[0];
            for (int s = 1; s < S.nsl; ++s) t += pp[s * NN];
            S.z[q] = __fmaf_rn(-tau, t, S.x[q]);
        }
    } else if (p == PH_TV) {
        // x^{k+1} = prox(z): one tile per group, the dual field read from
        // p[k & 1] and written to p[(k + 1) & 1]
        const int g = tid / TV_THREADS, j = i * TV_GROUPS + g;
        if (j < S.tv_ncb * S.tv_nrb) {
            float2 *pub_x = reinterpret_cast<float2 *>(psm) + (size_t)g * 2 * PS_TV_PUB;
            float2 *pub_y = pub_x + PS_TV_PUB;
            const int bx = j % S.tv_ncb, by = j / S.tv_ncb;
            const GroupCtx c{tid % TV_THREADS, TV_THREADS, 1 + ORB_GROUPS + DUAL_GROUPS + g};
            if (S.fgp)
                tv_body<true, false, GroupCtx, PS_TV_J>(c, bx, by, 0, 1, pub_x, pub_y, S.z, S.p[k & 1],
                                                        S.p[(k + 1) & 1], S.x, S.N, S.ntv, 1, S.tv_tc, S.tv_tr,
                                                        S.scal, nullptr);
            else
                tv_body<false, false, GroupCtx, PS_TV_J>(c, bx, by, 0, 1, pub_x, pub_y, S.z, S.p[k & 1],
                                                         S.p[(k + 1) & 1], S.x, S.N, S.ntv, 1, S.tv_tc, S.tv_tr,
                                                         S.scal, nullptr);
        }
    } else if (p == PH_QUAD) {
        // band partial sums of A x^{k+1}: item i takes the i-th of the
        // phase's equal ranges of (band pair, view pair, 64-ray) units, as a
        // block of the work-balanced projector does
        const int npair = (S.B + 1) / 2;
        QuadUnits U;
        U.nch = (npair + 63) / 64;
        U.u_rows = S.n_row_items * U.nch;
        U.u_cols = S.n_col_items * U.nch;
        U.u_z = (long long)(S.N / (2 * MR)) * (U.u_rows + U.u_cols);
        const long long nq = S.n_items[PH_QUAD];
        long long u0 = U.u_z * i / nq, u1 = U.u_z * (i + 1) / nq;
        if (S.qseg) {
            // small slices: item i is segment i (row-class band pairs, then column-class)
            const int nbp = S.N / (2 * MR);
            const bool rows = i < nbp;
            const int bp = rows ? i : i - nbp;
            u0 = rows ? (long long)bp * U.u_rows : (long long)nbp * U.u_rows + (long long)bp * U.u_cols;
            u1 = u0 + (rows ? U.u_rows : U.u_cols);
        }
        quad_balanced_body<2, true>(BlockCtx{}, u0, u1, U, psm,
                                    reinterpret_cast<int *>(psm + quad_smem(S.N)), S.x, S.views, S.row_items,
                                    S.col_items, S.N, S.V, S.B, S.band);
    } else if (p == PH_DUAL) {
        // residual, Step 3 and the next Step 1 for one view pair per group
        const int g = tid / FFT_T, vp = i * DUAL_GROUPS + g;
        if (2 * vp < S.V)
            dual_fft_body(GroupCtx{tid % FFT_T, FFT_T, 1 + ORB_GROUPS + g}, vp, 0,
                          reinterpret_cast<float2 *>(psm + (size_t)g * S.dual_smem), S.hhat, S.band, S.nb, S.b, S.mu,
                          S.mu, S.mubar, S.winv, S.lowdose, S.views, S.scal, S.V, S.B, S.P, S.tw);
    } else {
        // after the last iteration: the iteration count, and the result check
        unsigned f = 0;
        const size_t NN = (size_t)S.N * S.N, VB = (size_t)S.V * S.B;
        for (size_t q = tid; q < NN; q += PS_THREADS)
            if (!isfinite(S.x[q])) f = CHK_NONFINITE_RESULT;
        for (size_t q = tid; q < VB; q += PS_THREADS)
            if (!isfinite(S.mu[q])) f = CHK_NONFINITE_RESULT;
        f = __reduce_or_sync(0xffffffffu, f);
        if ((tid & 31) == 0 && f) atomicOr(flags_of(S.scal), f);
        if (tid == 0) S.scal[S_K] = (double)k;
    }
}

__global__ void __launch_bounds__(PS_THREADS, 1) k_persistent(const __grid_constant__ PParams prm)
{
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int cur[4];   // slice (< 0: leave), phase, iteration, item
    unsigned *queue = pslot(prm.sl[0].scal, S_PQUEUE), *err = pslot(prm.sl[0].scal, S_PERR);
    for (;;) {
        if (threadIdx.x == 0) {
            int s = -1, p = 0, k = 0, i = 0;
            const unsigned t = atomicAdd(queue, 1u);
            if (t < (unsigned)prm.total && ld_relaxed(err) == 0) {
                unsigned need;
                if (t >= (unsigned)(prm.K * prm.R)) {   // a slice's closing item
                    s = (int)(t - (unsigned)(prm.K * prm.R));
                    p = PH_N;
                    k = prm.K;
                    need = (unsigned)(prm.K * prm.sl[s].per_iter);
                } else {
                    k = (int)(t / (unsigned)prm.R);
                    const int r = (int)(t - (unsigned)(k * prm.R));
                    while (p + 1 < PH_N && prm.phase_off[p + 1] <= r) ++p;
                    const int rr = r - prm.phase_off[p];
                    int lo = 0, hi = prm.n - 1;   // the last slice whose range starts at or before rr
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (prm.slice_off[p][mid] <= rr) lo = mid;
                        else hi = mid - 1;
                    }
                    s = lo;
                    i = rr - prm.slice_off[p][s];
                    need = (unsigned)(k * prm.sl[s].per_iter + prm.sl[s].pre[p]);
                }
                const unsigned *done = pslot(prm.sl[s].scal, S_PDONE);
                if (ld_relaxed(done) < need) {
                    const unsigned long long t0 = global_ns();
                    while (ld_relaxed(done) < need) {
                        if (ld_relaxed(err) != 0) {
                            s = -1;
                            break;
                        }
                        if (global_ns() - t0 >= prm.wait_ns) {
                            if (atomicExch(err, 1u) == 0u)
                                for (int q = 0; q < prm.n; ++q) atomicOr(flags_of(prm.sl[q].scal), CHK_TIMEOUT);
                            s = -1;
                            break;
                        }
                        __nanosleep(128);
                    }
                }
                __threadfence();
            }
            cur[0] = s;
            cur[1] = p;
            cur[2] = k;
            cur[3] = i;
        }
        __syncthreads();
        const int s = cur[0];
        if (s < 0) break;
        run_item(prm.sl[s], cur[1], cur[2], cur[3], psm);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(pslot(prm.sl[s].scal, S_PDONE), 1u);
        }
    }
}

std::atomic<long long> g_wait_ns{5000000000LL};
std::atomic<int> g_form{0};
std::mutex g_attr_mu;
size_t g_attr_smem = 0;

size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace

int batched_form() { return g_form.load(); }

// Whether slice i can run in the persistent launch (see persistent_ok in the header).
bool persistent_slice_ok(const Geometry *g, const ct_pdtv_params *p, int iters0)
{
    const int ntv = p->tv_iters > 0 ? p->tv_iters : 10;
    return g->orbit && quad_ok(g) && fft_supported(g) && orbit_slices_ok(g, orbit_slices(g, false)) &&
           (p->precond == 0 || p->precond == 1 || p->precond == 3) && !(p->eps > 0.0) && ntv <= TV_MAX_STEPS &&
           p->iters == iters0 && p->iters > 0 && !p->resume;
}

ct_status launch_persistent(int n, const ct_geometry *const *geoms, const float *const *b,
                            const ct_pdtv_params *params, float *const *x_out, void *const *workspaces,
                            cudaStream_t st)
{
    std::unique_ptr<PParams> P(new (std::nothrow) PParams);
    if (!P) return CT_ERR_OOM;
    for (int c0 = 0; c0 < n; c0 += PS_MAX) {
        const int m = std::min(PS_MAX, n - c0);
        PParams &pp = *P;
        memset(&pp, 0, sizeof(pp));
        pp.n = m;
        pp.K = params[c0].iters;
        pp.wait_ns = (unsigned long long)std::max(0LL, g_wait_ns.load());
        size_t smem = 0;
        int n_sm = 0;
        for (int j = 0; j < m; ++j) {
            const Geometry *g = geoms[c0 + j];
            const ct_pdtv_params &prm = params[c0 + j];
            const SolveBuffers sb = solve_buffers(g, &prm, workspaces[c0 + j]);
            PSlice &S = pp.sl[j];
            S.N = g->n;
            S.V = g->n_views;
            S.B = g->n_bins;
            S.P = g->n_fft;
            S.nb = proj_bands(g->n);
            S.lowdose = prm.mode == CT_LOWDOSE;
            S.al = g->n_bins % 4 == 0;   // workspace buffers are 256-byte aligned
            S.n_row_items = g->n_row_items;
            S.n_col_items = g->n_col_items;
            S.nsl = orbit_slices(g, false);
            S.q16 = (g->n / 2 + ORB_T - 1) / ORB_T;
            S.orb_smem = (int)a16(orbit_smem_bytes());
            S.dual_smem = (int)a16(dual_fft_smem(g));
            S.ntv = prm.tv_iters > 0 ? prm.tv_iters : 10;
            S.fgp = prm.tv_accel == 1;
            // TV tiles: the batch's tiles together fill the GPU about twice
            // (tiling does not change the prox's values)
            tv_tile_shape(g->n, S.ntv, std::max(1, 2 * g->n_sm / m), g->tune_tv, &S.tv_tc, &S.tv_tr, &S.tv_ncb,
                          &S.tv_nrb, TV_WARPS * PS_TV_J);
            S.n_items[PH_ORBIT] = (S.q16 * S.q16 * S.nsl + ORB_GROUPS - 1) / ORB_GROUPS;
            S.n_items[PH_OREDUCE] = S.nsl > 1 ? (int)(((size_t)g->n * g->n + RED_PIX - 1) / RED_PIX) : 0;
            S.n_items[PH_TV] = (S.tv_ncb * S.tv_nrb + TV_GROUPS - 1) / TV_GROUPS;
            {
                // projector items: ranges of about 228 units (the share of one block of the
                // work-balanced projector at 512^2 / 720 views), at most one per SM; slices
                // with fewer such ranges than staged band pairs take one item per band pair
                const int nbp = g->n / (2 * MR);
                const long long nch = ((g->n_bins + 1) / 2 + 63) / 64;
                const long long u_z = (long long)nbp * (g->n_row_items + g->n_col_items) * nch;
                const long long nr = (u_z + 227) / 228;
                S.qseg = nr <= 2 * nbp;
                S.n_items[PH_QUAD] = S.qseg ? 2 * nbp : (int)std::min((long long)g->n_sm, nr);
            }
            S.n_items[PH_DUAL] = ((g->n_views + 1) / 2 + DUAL_GROUPS - 1) / DUAL_GROUPS;
            S.per_iter = 0;
            for (int q = 0; q < PH_N; ++q) {
                S.pre[q] = S.per_iter;
                S.per_iter += S.n_items[q];
            }
            S.views = g->d_views;
            S.row_items = g->d_row_items;
            S.col_items = g->d_col_items;
            S.trig = g->d_trig;
            S.tw = g->d_tw;
            S.hhat = sb.hhat;
            S.b = b[c0 + j];
            S.winv = sb.winv;
            S.mu = sb.mu;
            S.mubar = sb.mubar;
            S.x = x_out[c0 + j];
            S.z = sb.z;
            S.p[0] = sb.p0;
            S.p[1] = sb.p1;
            S.band = sb.band;
            S.orb = sb.orb;
            S.scal = sb.scal;
            const size_t tv_smem = sizeof(float2) * 2 * PS_TV_PUB * TV_GROUPS;
            smem = std::max({smem, (size_t)ORB_GROUPS * S.orb_smem, tv_smem, quad_smem(g->n) + 16,
                             (size_t)DUAL_GROUPS * S.dual_smem});
            n_sm = std::max(n_sm, g->n_sm);
        }
        // queue order: iteration, phase, slice, item
        pp.R = 0;
        for (int q = 0; q < PH_N; ++q) {
            pp.phase_off[q] = pp.R;
            int o = 0;
            for (int j = 0; j < m; ++j) {
                pp.slice_off[q][j] = o;
                o += pp.sl[j].n_items[q];
            }
            pp.slice_off[q][m] = o;
            pp.R += o;
        }
        pp.phase_off[PH_N] = pp.R;
        pp.total = pp.K * pp.R + m;
        {
            std::lock_guard<std::mutex> lock(g_attr_mu);
            if (smem > g_attr_smem) {
                if (cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                    cudaSuccess) {
                    cudaGetLastError();
                    set_error("ct_pdtv_solve_batched: %zu bytes of shared memory per block are not available", smem);
                    return CT_ERR_CUDA;
                }
                g_attr_smem = smem;
            }
        }
        counted();
        k_persistent<<<n_sm, PS_THREADS, smem, st>>>(pp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("ct_pdtv_solve_batched: persistent launch: %s", cudaGetErrorString(e));
            return CT_ERR_CUDA;
        }
    }
    return CT_OK;
}

}  // namespace ctpd

extern "C" ct_status ct_batched_options(int form, double wait_seconds)
{
    ctpd::set_error("%s", "");
    if ((form != CT_BATCH_AUTO && form != CT_BATCH_POOL) || wait_seconds != wait_seconds || wait_seconds > 3600.0) {
        ctpd::set_error("ct_batched_options: form must be CT_BATCH_AUTO or CT_BATCH_POOL, wait_seconds at most 3600");
        return CT_ERR_ARG;
    }
    ctpd::g_form.store(form);
    ctpd::g_wait_ns.store(wait_seconds < 0.0 ? 5000000000LL : (long long)(wait_seconds * 1e9));
    return CT_OK;
}
