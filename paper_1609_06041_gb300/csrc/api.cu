// api.cu -- host side of the C ABI declared in include/ctpd.h: argument
// checks, geometry tables, workspace layout and the solve loop of
// Algorithm 1 / 1' / 2 (arXiv 1609.06041, Secs. 2.3 and 3.1).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "ctpd_internal.cuh"

using namespace ctpd;

std::atomic<unsigned long long> ctpd::g_launches{0};
thread_local unsigned long long ctpd::t_launches = 0;
thread_local int ctpd::t_pdl = 0;

namespace {

thread_local char g_err[512] = "";

ct_status fail(ct_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

}  // namespace

void ctpd::set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ct_status ctpd::read_report(const void *workspace, ct_pdtv_report *report)
{
    // the scalar block sits at the start of the workspace
    double h[S_COUNT];
    cudaError_t e = cudaMemcpy(h, workspace, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_error("reading the solve report: %s", cudaGetErrorString(e));
        return CT_ERR_CUDA;
    }
    report->tau = h[S_TAU];
    report->sigma = h[S_SIGMA];
    report->kappa = h[S_KAPPA];
    report->lambda = h[S_LAMBDA];
    report->norm_ADA = h[S_NADA];
    report->norm_WDW = h[S_NWDW];
    report->k = (int)h[S_K];
    unsigned flags = 0;
    memcpy(&flags, &h[S_FLAGS], sizeof(flags));
    return status_from_flags(flags, "ct_pdtv_solve");
}

ct_status ctpd::status_from_flags(unsigned flags, const char *who)
{
    if (flags & CHK_TIMEOUT) {
        set_error("%s: a wait of the persistent batched solve ran out of its time limit; the slices are "
                  "incomplete", who);
        return CT_ERR_TIMEOUT;
    }
    if (flags & CHK_WEIGHT_NOT_POSITIVE) {
        set_error("%s: a weight w_i is zero or negative (W of Eq. 1 must be positive definite)", who);
        return CT_ERR_ARG;
    }
    if (flags & CHK_NONFINITE_INPUT) {
        set_error("%s: b or w holds NaN or infinity", who);
        return CT_ERR_NONFINITE;
    }
    if (flags & CHK_NONFINITE_RESULT) {
        set_error("%s: the image or the dual variable holds NaN or infinity (step sizes too large?)", who);
        return CT_ERR_NONFINITE;
    }
    return CT_OK;
}

namespace {
std::mutex g_fork_mu;
Fork g_forks[64];
}  // namespace

Fork *ctpd::fork_for(int dev)
{
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_fork_mu);
    Fork &f = g_forks[dev];
    if (!f.ready) {
        cudaError_t e = cudaStreamCreateWithFlags(&f.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        f.ready = true;
    }
    return &f;
}

namespace {

ct_status cuda_check(const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return CT_OK;
    snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA;
}

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout of one solve (offsets in bytes, 256-aligned).
struct Layout {
    size_t scal, partials, taps, hhat, taps2, hhat2, sv, winv, mu, mubar, r, z, u, w3, p0, p1, band, orb, aux, eps,
        stage, total;
};

Layout layout(const Geometry *g, const ct_pdtv_params *prm)
{
    Layout L;
    const size_t I = (size_t)g->n_views * g->n_bins, J = (size_t)g->n * g->n;
    size_t o = 0;
    L.scal = o;     o += align256(sizeof(double) * S_COUNT);
    L.partials = o; o += align256(sizeof(double) * 2 * dot_partials_doubles());   // two concurrent reductions
    L.taps = o;     o += align256(sizeof(float) * (2 * (size_t)g->n_bins - 1));
    L.hhat = o;     o += align256(sizeof(float2) * (size_t)g->n_fft);
    // the shift-variant D: its high band's taps and response, and s
    L.taps2 = o;    o += align256(sizeof(float) * (2 * (size_t)g->n_bins - 1));
    L.hhat2 = o;    o += align256(sizeof(float2) * (size_t)g->n_fft);
    L.sv = o;       o += align256(sizeof(float) * I);
    L.winv = o;     o += align256(sizeof(float) * I);
    L.mu = o;       o += align256(sizeof(float) * I);
    L.mubar = o;    o += align256(sizeof(float) * I);
    L.r = o;        o += align256(sizeof(float) * I);
    L.z = o;        o += align256(sizeof(float) * J);
    L.u = o;        o += align256(sizeof(float) * J);
    L.w3 = o;       o += align256(sizeof(float) * J);
    L.p0 = o;       o += align256(sizeof(float) * 2 * J);
    L.p1 = o;       o += align256(sizeof(float) * 2 * J);
    L.band = o;     o += align256(sizeof(float) * (size_t)proj_bands(g->n) * I);
    L.orb = o;      o += align256(sizeof(float) * (orbit_ok(g) ? orbit_partial_floats(g, 1) : 1));
    L.aux = o;      o += align256(sizeof(float) * 2 * I);   // the sinogram-side Lanczos, run beside the image side
    // device copies of page-locked host b, w and x (ct_pdtv_solve with host buffers)
    L.stage = o;    o += align256(sizeof(float) * (2 * I + J));
    // error-tolerant form: s, w2 and the split-K partial sums of its maps
    L.eps = o;
    if (prm && prm->eps > 0.0) o += align256(sizeof(float) * (2 * (size_t)g->n_bins + eps_partial_floats(g)));
    L.total = o;
    return L;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// Ray stride of the view-pair projector's quarter warps for a view with
// |a| = 1 / max(|cos t|, |sin t|) and npair ray pairs.  The eight lanes of
// a quarter warp read 16-byte entries at slots round(phi + a c j),
// j = 0..7; entries whose slots agree mod 8 share a bank group and
// serialise.  Rays are assigned in whole blocks of 8 c positions (the
// positions past the last whole block keep stride 1), so the expected
// wavefronts over the offsets phi are weighted by the share of positions
// in whole blocks; the stride c in 1..16 with the fewest wins (c = 1, the
// consecutive rays, unless another is better by more than 1 %).  Larger
// strides simulate better but measured slower (their partial-sum stores
// spread over more sectors).
int quad_lane_stride(double a, int npair)
{
    auto cost = [a](int c) {
        double tot = 0.0;
        for (int t = 0; t < 64; ++t) {
            const double phi = 8.0 * (t + 0.5) / 64.0;
            long slot[8];
            int group[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int j = 0; j < 8; ++j) slot[j] = (long)floor(phi + a * c * j + 0.5);
            for (int j = 0; j < 8; ++j) {
                bool dup = false;
                for (int i = 0; i < j; ++i) dup = dup || slot[i] == slot[j];
                if (!dup) ++group[slot[j] & 7];
            }
            int mx = 0;
            for (int k = 0; k < 8; ++k) mx = std::max(mx, group[k]);
            tot += mx;
        }
        return tot / 64.0;
    };
    const double c1 = cost(1);
    int best = 1;
    double bc = c1;
    for (int c = 2; c <= 16 && 8 * c <= npair; ++c) {
        const int full = npair / (8 * c) * (8 * c);
        const double k = ((double)full * cost(c) + (double)(npair - full) * c1) / npair;
        if (k < 0.99 * bc) {
            bc = k;
            best = c;
        }
    }
    return best;
}

// Largest eigenvalue of the symmetric positive semi-definite operator `op`
// (n-vectors) by k Lanczos steps from the all-ones vector, into scal[slot]:
//   w = op(q_j) - beta_{j-1} q_{j-1};  alpha_j = <w, q_j>;  w -= alpha_j q_j;
//   beta_j = |w|;  q_{j+1} = w / beta_j,
// then the largest eigenvalue of the tridiagonal (alpha, beta) (Sturm
// multisection).  The vectors are kept unnormalised (t_j = beta_{j-1} q_j,
// t_0 = ones with norm sqrt(n)), the scaling folded into the two fused
// update-and-reduce kernels of each step.  Coefficients go to scal[base ..
// base + 2k), the norm of t_0 to scal[n0slot].  t, tp, w are n-vector
// buffers; the whole recurrence stays on the device.
template <class Op>
void lanczos_norm(Op op, float *t, float *tp, float *w, size_t n, int k, double *scal, int base, int n0slot,
                  double *partials, unsigned *ticket, int slot, cudaStream_t st)
{
    // start vector: +-1 by a hash of the index (norm sqrt(n)); the all-ones
    // vector is invariant under the geometry's rotations and reflections and
    // has no component along a top eigenvector of another symmetry class
    launch_fill_sign(t, n, st);
    launch_scalars(scal, SC_SET, sqrt((double)n), 0, 0, n0slot, st);
    for (int j = 0; j < k; ++j) {
        op(t, w);
        launch_lanczos_step(w, tp, t, n, scal, base, n0slot, j, 0, partials, ticket, st);
        launch_lanczos_step(w, tp, t, n, scal, base, n0slot, j, 1, partials, ticket, st);
        float *x = tp;
        tp = t;
        t = w;
        w = x;
    }
    launch_lanczos_max(scal, base, k, slot, st);
}



// ---------------------------------------------------------------------
// Solve graphs.  A call of ct_pdtv_solve with a caller-owned workspace, no
// report, no resume and eps = 0 enqueues only device work, so the whole
// solve (setup and iterations) can be captured once as a CUDA graph and
// replayed by later calls with the same geometry, pointers, stream and
// parameters: one graph launch instead of some 280 kernel launches.  The
// graph reads the buffers when it runs, so new data in the same buffers is
// solved as usual.  Per geometry the most recent GRAPH_CACHE_MAX graphs are
// kept (until ct_geometry_destroy).  The capture uses a fork stream of its
// own for the setup's second branch.  Environment CTPD_SOLVE_GRAPHS=0 turns
// this off (every call then launches its kernels).
// ---------------------------------------------------------------------
constexpr size_t GRAPH_CACHE_MAX = 16;

struct SolveKey {
    const void *b, *w, *x, *ws;
    cudaStream_t st;
    int dev;
    ct_pdtv_params p;
};

bool same_params(const ct_pdtv_params &a, const ct_pdtv_params &b)
{
    return a.mode == b.mode && a.iters == b.iters && a.tv_iters == b.tv_iters && a.precond == b.precond &&
           a.norm_iters == b.norm_iters && a.resume == b.resume && a.beta == b.beta && a.tau == b.tau &&
           a.sigma == b.sigma && a.rho == b.rho && a.tv_accel == b.tv_accel && a.eps == b.eps;
}

bool same_key(const SolveKey &a, const SolveKey &b)
{
    return a.b == b.b && a.w == b.w && a.x == b.x && a.ws == b.ws && a.st == b.st && a.dev == b.dev &&
           same_params(a.p, b.p);
}

struct SolveGraph {
    SolveKey key;
    cudaGraphExec_t exec;
    unsigned long long launches;   // kernels in the graph
};

struct GraphCache {
    std::mutex mu;
    std::vector<SolveGraph> entries;   // least recently used first
    cudaStream_t cap = nullptr;        // captures run here (the caller's stream may be the
                                       // legacy default stream, which cannot be captured)
    Fork fork;                         // the captures' own fork stream
};

bool solve_graphs_enabled()
{
    static const bool on = [] {
        const char *e = getenv("CTPD_SOLVE_GRAPHS");
        return !(e && e[0] == '0');
    }();
    return on;
}

ct_status solve_graph(const ct_geometry *g, const float *b, const float *w, const ct_pdtv_params *prm,
                      float *x_out, void *workspace, void *stream)
{
    cudaStream_t st = S(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    int dev = -1;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone ||
        cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();   // inside a caller's capture (or unknown): enqueue the kernels
        return ctpd::pdtv_solve(g, b, w, prm, x_out, workspace, nullptr, stream, true);
    }
    Geometry *gm = const_cast<ct_geometry *>(g);
    {
        static std::mutex create_mu;
        std::lock_guard<std::mutex> lock(create_mu);
        if (!gm->graph_cache) gm->graph_cache = new GraphCache();
    }
    GraphCache *c = static_cast<GraphCache *>(gm->graph_cache);
    std::lock_guard<std::mutex> lock(c->mu);
    const SolveKey key{b, w, x_out, workspace, st, dev, *prm};
    for (size_t i = 0; i < c->entries.size(); ++i)
        if (same_key(c->entries[i].key, key)) {
            SolveGraph e = c->entries[i];
            c->entries.erase(c->entries.begin() + i);
            c->entries.push_back(e);
            g_err[0] = 0;
            if (cudaGraphLaunch(e.exec, st) != cudaSuccess) return cuda_check("ct_pdtv_solve (graph)");
            counted((unsigned)e.launches);
            return CT_OK;
        }
    if (!c->fork.ready) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->fork.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork.join, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ctpd::pdtv_solve(g, b, w, prm, x_out, workspace, nullptr, stream, true);
        }
        c->fork.ready = true;
    }
    // capture this call on the cache's stream (nothing runs), instantiate,
    // then launch the graph on the caller's stream
    const unsigned long long t0 = t_launches;
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return ctpd::pdtv_solve(g, b, w, prm, x_out, workspace, nullptr, stream, true);
    }
    const ct_status r = ctpd::pdtv_solve(g, b, w, prm, x_out, workspace, nullptr, c->cap, true, &c->fork);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->cap, &graph);
    const unsigned long long n = t_launches - t0;
    g_launches.fetch_sub(n, std::memory_order_relaxed);   // captured, not run
    t_launches -= n;
    if (r != CT_OK) {   // an argument error: nothing was enqueued
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return r;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = ec;
    if (ei == cudaSuccess) ei = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {   // not capturable after all: run the call directly
        cudaGetLastError();
        return ctpd::pdtv_solve(g, b, w, prm, x_out, workspace, nullptr, stream, true);
    }
    if (cudaGraphLaunch(exec, st) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return cuda_check("ct_pdtv_solve (graph)");
    }
    counted((unsigned)n);
    if (c->entries.size() >= GRAPH_CACHE_MAX) {
        cudaGraphExecDestroy(c->entries.front().exec);
        c->entries.erase(c->entries.begin());
    }
    c->entries.push_back(SolveGraph{key, exec, n});
    g_err[0] = 0;
    return CT_OK;
}

}  // namespace

ctpd::SolveBuffers ctpd::solve_buffers(const Geometry *g, const ct_pdtv_params *prm, void *workspace)
{
    const Layout L = layout(g, prm);
    char *ws = static_cast<char *>(workspace);
    SolveBuffers sb;
    sb.scal = (double *)(ws + L.scal);
    sb.winv = (float *)(ws + L.winv);
    sb.mu = (float *)(ws + L.mu);
    sb.mubar = (float *)(ws + L.mubar);
    sb.z = (float *)(ws + L.z);
    sb.p0 = (float *)(ws + L.p0);
    sb.p1 = (float *)(ws + L.p1);
    sb.band = (float *)(ws + L.band);
    sb.orb = (float *)(ws + L.orb);
    sb.hhat = (float2 *)(ws + L.hhat);
    return sb;
}

// drop the cached graphs (their launch shapes are out of date); the streams stay
void ctpd::graph_cache_clear(Geometry *g)
{
    GraphCache *c = static_cast<GraphCache *>(g->graph_cache);
    if (!c) return;
    std::lock_guard<std::mutex> lock(c->mu);
    for (const SolveGraph &e : c->entries) cudaGraphExecDestroy(e.exec);
    c->entries.clear();
}

namespace {

void graph_cache_free(Geometry *g)
{
    GraphCache *c = static_cast<GraphCache *>(g->graph_cache);
    if (!c) return;
    for (const SolveGraph &e : c->entries) cudaGraphExecDestroy(e.exec);
    if (c->fork.ready) {
        cudaStreamDestroy(c->cap);
        cudaStreamDestroy(c->fork.s);
        cudaEventDestroy(c->fork.fork);
        cudaEventDestroy(c->fork.join);
    }
    delete c;
    g->graph_cache = nullptr;
}
}  // namespace

extern "C" {

const char *ct_version(void) { return "ctpd 0.1 sm_103a"; }

const char *ct_last_error(void) { return g_err; }

unsigned long long ct_kernel_launches(void) { return g_launches.load(); }

ct_status ct_geometry_create(int n, int n_views, int n_bins, const double *angles,
                             ct_geometry **out)
{
    g_err[0] = 0;
    if (!out) return fail(CT_ERR_ARG, "ct_geometry_create: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 8192 || n_views < 1 || n_views > 8192 || n_bins < 1 || n_bins > 8192)
        return fail(CT_ERR_ARG, "ct_geometry_create: sizes must be in [1, 8192]");
    ct_geometry *g = new (std::nothrow) ct_geometry();
    if (!g) return fail(CT_ERR_OOM, "ct_geometry_create: out of host memory");
    g->n = n;
    g->n_views = n_views;
    g->n_bins = n_bins;
    g->n_fft = 1;
    while (g->n_fft < 2 * n_bins) g->n_fft <<= 1;
    g->orbit = !angles && (n_views % 2 == 0) && (n % 2 == 0);   // V <= 8192, so a slice has <= 1024 base views
    cudaGetDevice(&g->device);
    g->n_sm = 0;
    if (cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess || g->n_sm < 1) {
        cudaGetLastError();
        g->n_sm = 1;
    }
    g->h_angles = new double[n_views];
    // candidate-window margin of the backprojector (bins): a generous bound
    // on the float rounding of the Joseph coordinates at this size
    g->win_eps = (float)(16.0 * (n + n_bins) * ldexp(1.0, -24) + ldexp(1.0, -13));
    ViewP *hv = new ViewP[n_views];
    float4 *ht = new float4[n_views];
    std::map<float, int> stride_of;
    int *rl = new int[n_views], *cl = new int[n_views];
    g->n_row = g->n_col = 0;
    for (int v = 0; v < n_views; ++v) {
        double t = angles ? angles[v] : (double)v * M_PI / (double)n_views;
        if (!isfinite(t)) {
            delete[] hv;
            delete[] ht;
            delete[] rl;
            delete[] cl;
            ct_geometry_destroy(g);
            return fail(CT_ERR_ARG, "ct_geometry_create: angle %d is not finite", v);
        }
        double c = cos(t), s = sin(t);
        g->h_angles[v] = t;
        int rows = angles ? (fabs(c) >= fabs(s)) : ((4 * v <= n_views) || (4 * v >= 3 * n_views));
        ViewP &P = hv[v];
        memset(&P, 0, sizeof(P));
        P.rows = rows;
        double a = rows ? 1.0 / c : 1.0 / s, m = rows ? -s / c : -c / s;
        P.a = (float)a;
        P.m = (float)m;
        P.scale = (float)fabs(a);
        P.inv_a = (float)(rows ? c : s);
        P.inv_m = P.m != 0.0f ? 1.0f / P.m : 0.0f;
        P.three = fabs((double)P.inv_a) >= 1.0 - 1.5 * (double)g->win_eps;
        {
            // views v, V - v, V/2 +- v share |a|: one search per value
            const float key = P.scale;
            auto it = stride_of.find(key);
            if (it == stride_of.end()) it = stride_of.emplace(key, quad_lane_stride(key, (n_bins + 1) / 2)).first;
            P.stride = it->second;
        }
        if (rows) rl[g->n_row++] = v;
        else cl[g->n_col++] = v;
        const double sc = 1.0 / fmax(fabs(c), fabs(s));
        ht[v] = make_float4((float)c, (float)s, (float)sc, (float)(1.0 - 0.5 * sc));
    }
    // view-pair work items of the projector (default angles only)
    g->vpair = !angles;
    int2 *hri = new int2[n_views + 1], *hci = new int2[n_views + 1];
    g->n_row_items = g->n_col_items = 0;
    if (g->vpair) {
        hri[g->n_row_items++] = make_int2(0, -1);
        for (int v = 1; v < n_views; ++v) {
            if (4 * v <= n_views) hri[g->n_row_items++] = make_int2(v, n_views - v);
            else if (4 * v < 3 * n_views && 2 * v < n_views) hci[g->n_col_items++] = make_int2(v, n_views - v);
            else if (2 * v == n_views) hci[g->n_col_items++] = make_int2(v, -1);
        }
    }
    float2 *htw = new float2[g->n_fft];
    for (int k = 0; k < g->n_fft; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)g->n_fft;
        htw[k] = make_float2((float)cos(ang), (float)sin(ang));
    }
    cudaError_t e = cudaMalloc(&g->d_views, sizeof(ViewP) * n_views);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_tw, sizeof(float2) * g->n_fft);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tw, htw, sizeof(float2) * g->n_fft, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_row_list, sizeof(int) * (n_views + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_col_list, sizeof(int) * (n_views + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_trig, sizeof(float4) * n_views);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_trig, ht, sizeof(float4) * n_views, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_views, hv, sizeof(ViewP) * n_views, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_row_list, rl, sizeof(int) * n_views, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_col_list, cl, sizeof(int) * n_views, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_row_items, sizeof(int2) * (n_views + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_col_items, sizeof(int2) * (n_views + 1));
    if (e == cudaSuccess && g->n_row_items)
        e = cudaMemcpy(g->d_row_items, hri, sizeof(int2) * g->n_row_items, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && g->n_col_items)
        e = cudaMemcpy(g->d_col_items, hci, sizeof(int2) * g->n_col_items, cudaMemcpyHostToDevice);
    delete[] hri;
    delete[] hci;
    delete[] hv;
    delete[] ht;
    delete[] htw;
    delete[] rl;
    delete[] cl;
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof(g_err), "ct_geometry_create: %s", cudaGetErrorString(e));
        ct_geometry_destroy(g);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA;
    }
    kernel_attrs_filter();
    kernel_attrs_tv();
    kernel_attrs_joseph();
    kernel_attrs_fft();
    kernel_attrs_grad();
    ct_status st = cuda_check("ct_geometry_create");
    if (st != CT_OK) {
        ct_geometry_destroy(g);
        return st;
    }
    *out = g;
    return CT_OK;
}

void ct_geometry_destroy(ct_geometry *g)
{
    if (!g) return;
    if (g->d_views) cudaFree(g->d_views);
    if (g->d_row_list) cudaFree(g->d_row_list);
    if (g->d_col_list) cudaFree(g->d_col_list);
    if (g->d_trig) cudaFree(g->d_trig);
    if (g->d_tw) cudaFree(g->d_tw);
    if (g->d_row_items) cudaFree(g->d_row_items);
    if (g->d_col_items) cudaFree(g->d_col_items);
    if (g->d_qbounds) cudaFree(g->d_qbounds);
    eps_cache_free(g);
    graph_cache_free(g);
    delete[] g->h_angles;
    delete g;
}

ct_status ct_project(const ct_geometry *g, const float *img, float *sino, int batch, void *stream)
{
    g_err[0] = 0;
    if (!g || batch < 0 || batch > 65535) return fail(CT_ERR_ARG, "ct_project: bad argument");
    if (batch == 0) return CT_OK;
    if (!img || !sino) return fail(CT_ERR_ARG, "ct_project: NULL pointer");
    if (!aligned16(img) || !aligned16(sino)) return fail(CT_ERR_ARG, "ct_project: pointers must be 16-byte aligned");
    // band partial sums: stream-ordered scratch, freed after the reduction
    const size_t bytes = sizeof(float) * (size_t)proj_bands(g->n) * g->n_views * g->n_bins * batch;
    float *partial = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&partial, bytes, S(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CT_ERR_OOM, "ct_project: scratch allocation failed (%zu bytes)", bytes);
    }
    launch_project_bands(g, img, partial, batch, S(stream));
    launch_band_reduce(g, partial, sino, 0, nullptr, nullptr, nullptr, batch, S(stream));
    cudaFreeAsync(partial, S(stream));
    return cuda_check("ct_project");
}

int ct_project_bands_count(const ct_geometry *g) { return g ? proj_bands(g->n) : 0; }

ct_status ct_project_bands(const ct_geometry *g, const float *img, float *partial, int batch, void *stream)
{
    g_err[0] = 0;
    if (!g || batch < 0 || batch > 65535) return fail(CT_ERR_ARG, "ct_project_bands: bad argument");
    if (batch == 0) return CT_OK;
    if (!img || !partial) return fail(CT_ERR_ARG, "ct_project_bands: NULL pointer");
    if (!aligned16(img) || !aligned16(partial))
        return fail(CT_ERR_ARG, "ct_project_bands: pointers must be 16-byte aligned");
    launch_project_bands(g, img, partial, batch, S(stream));
    return cuda_check("ct_project_bands");
}

ct_status ct_backproject(const ct_geometry *g, const float *sino, float *img, int batch, void *stream)
{
    g_err[0] = 0;
    if (!g || batch < 0 || batch > 65535) return fail(CT_ERR_ARG, "ct_backproject: bad argument");
    if (batch == 0) return CT_OK;
    if (!img || !sino) return fail(CT_ERR_ARG, "ct_backproject: NULL pointer");
    if (!aligned16(img) || !aligned16(sino)) return fail(CT_ERR_ARG, "ct_backproject: pointers must be 16-byte aligned");
    if (!orbit_ok(g)) launch_backproject(g, sino, img, 0, nullptr, nullptr, batch, S(stream));
    else launch_backproject_orbit(g, sino, img, 0, nullptr, nullptr, batch, nullptr, S(stream));
    return cuda_check("ct_backproject");
}

ct_status ct_ramp_taps(const ct_geometry *g, int mode, double tau, double kappa, float *taps, void *stream)
{
    g_err[0] = 0;
    if (!g || !taps || mode < CT_LOWDOSE || mode > CT_TAPS_HIGH_BAND || !(tau > 0.0) ||
        (mode != CT_FEWVIEW && !(kappa >= 0.0)))
        return fail(CT_ERR_ARG, "ct_ramp_taps: bad argument");
    launch_taps(g, mode, nullptr, tau, kappa, taps, S(stream));
    return cuda_check("ct_ramp_taps");
}

ct_status ct_ramp_filter_split(const ct_geometry *g, const float *taps_lo, const float *taps_hi, int half_len,
                               const float *sv, const float *in, float *out, int batch, void *stream)
{
    g_err[0] = 0;
    if (!g || half_len < 1 || half_len > g->n_bins || batch < 0 || batch > 65535)
        return fail(CT_ERR_ARG, "ct_ramp_filter_split: bad argument");
    if (!fft_supported(g)) return fail(CT_ERR_ARG, "ct_ramp_filter_split: needs n_bins <= 4096");
    if (batch == 0) return CT_OK;
    if (!taps_lo || !taps_hi || !sv || !in || !out || in == out)
        return fail(CT_ERR_ARG, "ct_ramp_filter_split: bad pointer");
    // the bands' frequency responses: stream-ordered scratch, freed after use
    float2 *hs = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&hs, sizeof(float2) * 2 * g->n_fft, S(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CT_ERR_OOM, "ct_ramp_filter_split: scratch allocation failed");
    }
    launch_sv_hhat(g, taps_lo, taps_hi, half_len, hs, hs + g->n_fft, S(stream));
    launch_filter_sv(g, hs, hs + g->n_fft, sv, in, out, nullptr, nullptr, 0, nullptr, batch, S(stream));
    cudaFreeAsync(hs, S(stream));
    return cuda_check("ct_ramp_filter_split");
}

ct_status ct_ramp_filter(const ct_geometry *g, const float *taps, int half_len, const float *in,
                         float *out, int batch, void *stream)
{
    g_err[0] = 0;
    if (!g || half_len < 1 || half_len > g->n_bins || batch < 0 || batch > 65535)
        return fail(CT_ERR_ARG, "ct_ramp_filter: bad argument");
    if (batch == 0) return CT_OK;
    if (!taps || !in || !out || in == out) return fail(CT_ERR_ARG, "ct_ramp_filter: bad pointer");
    if (!fft_supported(g)) {
        launch_filter(g, taps, half_len, in, out, nullptr, nullptr, 0, nullptr, batch, S(stream));
        return cuda_check("ct_ramp_filter");
    }
    // frequency response of the taps: stream-ordered scratch, freed after use
    float2 *hhat = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&hhat, sizeof(float2) * g->n_fft, S(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CT_ERR_OOM, "ct_ramp_filter: scratch allocation failed");
    }
    launch_hhat(g, taps, half_len, hhat, S(stream));
    launch_filter_fft(g, hhat, in, out, nullptr, nullptr, 0, nullptr, batch, S(stream));
    cudaFreeAsync(hhat, S(stream));
    return cuda_check("ct_ramp_filter");
}

ct_status ct_pdtv_status(const void *workspace, void *stream)
{
    g_err[0] = 0;
    if (!workspace) return fail(CT_ERR_ARG, "ct_pdtv_status: NULL workspace");
    cudaError_t e = cudaStreamSynchronize(S(stream));
    unsigned flags = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&flags, static_cast<const char *>(workspace) + sizeof(double) * S_FLAGS, sizeof(flags),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(CT_ERR_CUDA, "ct_pdtv_status: %s", cudaGetErrorString(e));
    return status_from_flags(flags, "ct_pdtv_status");
}

size_t ct_pdtv_workspace_bytes(const ct_geometry *g, const ct_pdtv_params *p)
{
    if (!g) return 0;
    return layout(g, p).total;
}

// Where a buffer lives: 0 device (or managed) memory, 1 page-locked host
// memory, -1 memory the device cannot copy from asynchronously (pageable).
static int buffer_kind(const void *p)
{
    if (!p) return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 0;
    return a.type == cudaMemoryTypeHost ? 1 : -1;
}

static ct_status solve_device(const ct_geometry *g, const float *b, const float *w, const ct_pdtv_params *prm,
                              float *x_out, void *workspace, ct_pdtv_report *report, void *stream)
{
    // a repeat of an earlier call replays that call's CUDA graph (the
    // error-tolerant form once D's eigenbasis is cached: its first solve
    // computes it on the host)
    if (g && prm && workspace && !report && !prm->resume && solve_graphs_enabled() &&
        (!(prm->eps > 0.0) || eps_basis_ready(g, prm->precond, prm->tau)))
        return solve_graph(g, b, w, prm, x_out, workspace, stream);
    return ctpd::pdtv_solve(g, b, w, prm, x_out, workspace, report, stream, true);
}

ct_status ct_pdtv_solve(const ct_geometry *g, const float *b, const float *w,
                        const ct_pdtv_params *prm, float *x_out, void *workspace,
                        ct_pdtv_report *report, void *stream)
{
    const int kb = buffer_kind(b), kw = buffer_kind(w), kx = buffer_kind(x_out);
    if (kb < 0 || kw < 0 || kx < 0)
        return fail(CT_ERR_ARG, "ct_pdtv_solve: host buffers must be page-locked (cudaHostAlloc, cudaHostRegister)");
    if (!(kb || kw || kx) || !g || !prm || !b || !x_out) return solve_device(g, b, w, prm, x_out, workspace, report, stream);
    // page-locked host buffers: stream-ordered copies to and from the
    // workspace's staging area around the device solve
    g_err[0] = 0;
    const Layout L = layout(g, prm);
    const size_t I = (size_t)g->n_views * g->n_bins, J = (size_t)g->n * g->n;
    cudaStream_t st = S(stream);
    char *ws = static_cast<char *>(workspace);
    bool owned = false;
    if (!ws) {
        if (prm->resume) return fail(CT_ERR_ARG, "ct_pdtv_solve: resume needs the workspace");
        if (cudaMallocAsync((void **)&ws, L.total, st) != cudaSuccess) {
            cudaGetLastError();
            return fail(CT_ERR_OOM, "ct_pdtv_solve: workspace allocation failed");
        }
        owned = true;
    }
    float *bd = (float *)(ws + L.stage), *wd = bd + I, *xd = wd + I;
    const float *b_use = b, *w_use = w;
    float *x_use = x_out;
    cudaError_t e = cudaSuccess;
    if (kb) {
        e = cudaMemcpyAsync(bd, b, sizeof(float) * I, cudaMemcpyHostToDevice, st);
        b_use = bd;
    }
    if (kw && e == cudaSuccess) {
        e = cudaMemcpyAsync(wd, w, sizeof(float) * I, cudaMemcpyHostToDevice, st);
        w_use = wd;
    }
    if (kx) {
        if (prm->resume && e == cudaSuccess) e = cudaMemcpyAsync(xd, x_out, sizeof(float) * J, cudaMemcpyHostToDevice, st);
        x_use = xd;
    }
    ct_status cs = e == cudaSuccess ? solve_device(g, b_use, w_use, prm, x_use, ws, report, stream)
                                    : fail(CT_ERR_CUDA, "ct_pdtv_solve: host copy: %s", cudaGetErrorString(e));
    if (kx && cs == CT_OK) {
        e = cudaMemcpyAsync(x_out, xd, sizeof(float) * J, cudaMemcpyDeviceToHost, st);
        // the report path synchronises: x_out is then ready when the call returns
        if (e == cudaSuccess && report) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) cs = fail(CT_ERR_CUDA, "ct_pdtv_solve: host copy: %s", cudaGetErrorString(e));
    }
    if (owned) cudaFreeAsync(ws, st);
    return cs;
}

}  // extern "C"

ct_status ctpd::pdtv_solve(const ct_geometry *g, const float *b, const float *w, const ct_pdtv_params *prm,
                           float *x_out, void *workspace, ct_pdtv_report *report, void *stream, bool allow_fork,
                           void *fork)
{
    g_err[0] = 0;
    if (!g || !b || !prm || !x_out) return fail(CT_ERR_ARG, "ct_pdtv_solve: NULL argument");
    const int mode = prm->mode;
    if (mode != CT_LOWDOSE && mode != CT_FEWVIEW) return fail(CT_ERR_ARG, "ct_pdtv_solve: unknown mode");
    if (mode == CT_LOWDOSE && !w) return fail(CT_ERR_ARG, "ct_pdtv_solve: low-dose needs weights w");
    if (prm->iters < 0 || prm->tv_iters < 0 || prm->norm_iters < 0)
        return fail(CT_ERR_ARG, "ct_pdtv_solve: negative iteration count");
    if (mode == CT_LOWDOSE && !(prm->beta >= 0.0)) return fail(CT_ERR_ARG, "ct_pdtv_solve: beta must be >= 0");
    if (prm->resume && !workspace) return fail(CT_ERR_ARG, "ct_pdtv_solve: resume needs the workspace");
    if (prm->precond < 0 || prm->precond > 3) return fail(CT_ERR_ARG, "ct_pdtv_solve: precond must be 0, 1, 2 or 3");
    if (prm->precond == 3 && mode != CT_FEWVIEW)
        return fail(CT_ERR_ARG, "ct_pdtv_solve: the few-view smoothed ramp (precond 3) needs CT_FEWVIEW");
    if (prm->tv_accel != 0 && (prm->tv_accel != 1 || prm->tv_iters > tv_max_steps()))
        return fail(CT_ERR_ARG, "ct_pdtv_solve: tv_accel must be 0 or 1 (1 needs tv_iters <= %d)", tv_max_steps());
    if (prm->precond == 2 && (mode != CT_LOWDOSE || !fft_supported(g)))
        return fail(CT_ERR_ARG, "ct_pdtv_solve: the shift-variant preconditioner needs CT_LOWDOSE and n_bins <= 4096");
    if (!(prm->eps >= 0.0) || !std::isfinite(prm->eps))
        return fail(CT_ERR_ARG, "ct_pdtv_solve: eps must be finite and >= 0");
    const bool epsf = prm->eps > 0.0;
    if (epsf && (mode != CT_FEWVIEW || prm->precond == 2 || !fft_supported(g)))
        return fail(CT_ERR_ARG, "ct_pdtv_solve: the error-tolerant form (eps > 0) needs CT_FEWVIEW, precond 0, 1 or 3 "
                                "and n_bins <= 4096");
    if (!aligned16(b) || !aligned16(x_out) || (w && !aligned16(w)) || (workspace && !aligned16(workspace)))
        return fail(CT_ERR_ARG, "ct_pdtv_solve: pointers must be 16-byte aligned");
    const double rho = prm->rho > 0.0 ? prm->rho : 0.95;
    if (!(rho < 1.0)) return fail(CT_ERR_ARG, "ct_pdtv_solve: rho must be in (0, 1)");
    const int ntv = prm->tv_iters > 0 ? prm->tv_iters : 10;
    const int nlz = std::min(prm->norm_iters > 0 ? prm->norm_iters : 12, (int)LANCZOS_MAX);
    cudaStream_t st = S(stream);
    const Layout L = layout(g, prm);
    const size_t I = (size_t)g->n_views * g->n_bins, J = (size_t)g->n * g->n;

    char *ws = static_cast<char *>(workspace);
    bool owned = false;
    if (!ws) {
        cudaError_t e = cudaMallocAsync((void **)&ws, L.total, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(CT_ERR_OOM, "ct_pdtv_solve: workspace allocation failed");
        }
        owned = true;
    }
    double *scal = (double *)(ws + L.scal);
    double *partials = (double *)(ws + L.partials);
    unsigned *ticket = (unsigned *)(partials + dot_partials_doubles() - 64);
    double *partials2 = partials + dot_partials_doubles();
    unsigned *ticket2 = (unsigned *)(partials2 + dot_partials_doubles() - 64);
    float *aux = (float *)(ws + L.aux);
    float *taps = (float *)(ws + L.taps);
    float2 *hhat = (float2 *)(ws + L.hhat);
    const bool use_fft = fft_supported(g);
    // precond 2: hhat / hhat2 hold (H_lo +- H_hi) / 2, sv = sqrt(kappa w)
    const bool sv_d = prm->precond == 2;
    float *taps2 = (float *)(ws + L.taps2), *sv = (float *)(ws + L.sv);
    float2 *hhat2 = (float2 *)(ws + L.hhat2);
    // out = post .* D(pre .* in) * (mode 1 ? -sigma : 1), and D applied to A x given as band sums
    auto filter = [&](const float *in, float *out, const float *pre, const float *post, int md, cudaStream_t s_) {
        if (sv_d) launch_filter_sv(g, hhat, hhat2, sv, in, out, pre, post, md, scal, 1, s_);
        else if (use_fft) launch_filter_fft(g, hhat, in, out, pre, post, md, scal, 1, s_);
        else launch_filter(g, taps, prm->precond ? g->n_bins : 1, in, out, pre, post, md, scal, 1, s_);
    };
    float *winv = (float *)(ws + L.winv);
    float *mu = (float *)(ws + L.mu), *mubar = (float *)(ws + L.mubar), *r = (float *)(ws + L.r);
    float *z = (float *)(ws + L.z), *uimg = (float *)(ws + L.u), *w3img = (float *)(ws + L.w3);
    float *band = (float *)(ws + L.band);
    float *orb = (float *)(ws + L.orb);
    // A^T, by rotation orbits when the geometry allows
    auto backproject = [&](const float *yy, float *out, int md, const float *xin) {
        if (orbit_ok(g)) launch_backproject_orbit(g, yy, out, md, xin, scal, 1, orb, st, allow_fork);
        else launch_backproject(g, yy, out, md, xin, scal, 1, st);
    };
    float *pbuf[2] = {(float *)(ws + L.p0), (float *)(ws + L.p1)};
    const int half = prm->precond ? g->n_bins : 1;
    const int lowdose = mode == CT_LOWDOSE;
    // per-iteration trace (report->trace, host): device values, copied at the report's sync
    double *trace_h = report ? report->trace : nullptr;
    double *trace_d = nullptr;
    if (trace_h && prm->iters > 0) {
        if (cudaMallocAsync((void **)&trace_d, sizeof(double) * (prm->iters + trace_scratch_doubles()), st) !=
            cudaSuccess) {
            cudaGetLastError();
            if (owned) cudaFreeAsync(ws, st);
            return fail(CT_ERR_OOM, "ct_pdtv_solve: trace buffer allocation failed");
        }
    }
    unsigned *flags = flags_of(scal);

    long long k0 = 0;
    if (prm->resume) {
        double kd = 0.0;
        cudaMemcpyAsync(&kd, scal + S_K, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        k0 = (long long)kd;
    } else {
        // ---- setup (Alg. 1 / Alg. 2 boxes): kappa, tau, D, sigma ----
        cudaMemsetAsync(scal, 0, sizeof(double) * S_COUNT, st);
    }
    // the input checks: w > 0 and finite (low-dose), b finite; bits in the flag word
    cudaMemsetAsync(flags, 0, sizeof(unsigned), st);
    launch_check_inputs(b, lowdose ? w : nullptr, I, flags, st);
    if (!prm->resume) {
        cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
        cudaMemsetAsync(ticket2, 0, sizeof(unsigned), st);
        if (lowdose) {
            launch_recip(w, winv, I, st);
            launch_dot(winv, nullptr, I, scal, S_RED0, partials, st);
            launch_scalars(scal, SC_KAPPA_FROM_SUM, (double)I, 0, 0, 0, st);
        }
        launch_scalars(scal, SC_TAU, prm->tau, (double)g->n_views, 0, mode, st);
        if (sv_d) {
            launch_taps(g, CT_TAPS_LOW_BAND, scal, 0.0, 0.0, taps, st);
            launch_taps(g, CT_TAPS_HIGH_BAND, scal, 0.0, 0.0, taps2, st);
            launch_sv_hhat(g, taps, taps2, half, hhat, hhat2, st);
            launch_sv_scale(w, scal, sv, I, st);
        } else if (prm->precond == 3) {
            // few-view smoothed ramp: Eq. 24's form with kappa = tau l (l the mean
            // diagonal of A A^T, from the view constants), tau as SC_TAU sets it
            double sa = 0.0;
            for (int v = 0; v < g->n_views; ++v) {
                const double t = g->h_angles[v];
                sa += 1.0 / std::max(fabs(cos(t)), fabs(sin(t)));
            }
            const double ell = (2.0 / 3.0) * ((double)g->n * g->n / g->n_bins) * (sa / g->n_views);
            const double tau_h = prm->tau > 0.0 ? prm->tau : 0.01;
            launch_scalars(scal, SC_SET, tau_h * ell, 0, 0, S_KAPPA, st);
            launch_taps(g, CT_LOWDOSE, scal, 0.0, 0.0, taps, st);
            if (use_fft) launch_hhat(g, taps, half, hhat, st);
        } else {
            if (prm->precond) launch_taps(g, mode, scal, 0.0, 0.0, taps, st);
            else launch_fill(taps, 1.0f, 1, st);
            if (use_fft) launch_hhat(g, taps, half, hhat, st);
        }
        if (!(prm->sigma > 0.0)) {
            // ||W^-1/2 D W^-1/2|| by Lanczos on the sinogram side (low-dose),
            // on a second stream beside the image-side run when D is applied
            // by FFT (the two then share no buffers)
            Fork *fk = nullptr;
            if (allow_fork && lowdose && use_fft) {
                int dev = -1;
                if (fork) fk = static_cast<Fork *>(fork);
                else if (cudaGetDevice(&dev) == cudaSuccess) fk = fork_for(dev);
            }
            if (lowdose) {
                cudaStream_t s2 = st;
                if (fk) s2 = fork_begin(fk, st);
                float *sw = aux;
                launch_sqrt(winv, sw, I, s2);
                auto op_wdw = [&](const float *v, float *out) { filter(v, out, sw, sw, 0, s2); };
                lanczos_norm(op_wdw, mu, r, aux + I, I, nlz, scal, S_LZ2, S_LN0B, partials2, ticket2, S_NWDW, s2);
            }
            // ||A^T D A|| by Lanczos on the image side
            auto op_ada = [&](const float *v, float *out) {
                launch_project_bands(g, v, band, 1, st);
                if (sv_d) {
                    launch_filter_sv_bands(g, hhat, hhat2, sv, band, mubar, 1, st);
                } else if (use_fft) {
                    launch_filter_fft_bands(g, hhat, band, mubar, 1, st);
                } else {
                    launch_band_reduce(g, band, r, 0, nullptr, nullptr, nullptr, 1, st);
                    launch_filter(g, taps, half, r, mubar, nullptr, nullptr, 0, nullptr, 1, st);
                }
                backproject(mubar, out, 0, nullptr);
            };
            {
                // its projector and backprojector launches, like the loop's, may start as their
                // predecessors finish (each waits for it before any memory access)
                PdlScope pdl(true);
                lanczos_norm(op_ada, z, uimg, w3img, J, nlz, scal, S_LZ, S_LN0, partials, ticket, S_NADA, st);
            }
            if (fk) fork_end(fk, st);
        }
        launch_scalars(scal, SC_SIGMA, prm->sigma, rho, 0, mode, st);
        launch_scalars(scal, SC_LAMBDA, lowdose ? prm->beta : 0.0, 0, 0, mode, st);
        // ---- x^0 = mu^0 = 0, p = 0; Step 1 at k = 0: mu_bar = -sigma D b ----
        launch_fill(x_out, 0.0f, J, st);
        launch_fill(pbuf[0], 0.0f, 2 * J, st);
        launch_fill(pbuf[1], 0.0f, 2 * J, st);
        launch_fill(mu, 0.0f, I, st);
        filter(b, mubar, nullptr, nullptr, 1, st);
    }
    ct_status cs = cuda_check("ct_pdtv_solve setup");
    // error-tolerant form: D's eigenbasis (precond 1, 3; none for D = I),
    // and Step 1 at k = 0 through the same proximal map
    const float *eQ = nullptr, *eLam = nullptr;
    float *es = (float *)(ws + L.eps), *ew2 = es + g->n_bins, *epart = ew2 + g->n_bins;
    if (cs == CT_OK && epsf && prm->precond != 0) cs = eps_basis(g, prm->precond, prm->tau, taps, st, &eQ, &eLam);
    if (cs == CT_OK && epsf && !prm->resume)
        launch_eps_step(g, mubar, mubar, nullptr, nullptr, eQ, eLam, prm->eps, scal, aux, es, ew2, epart, st);
    if (cs != CT_OK) {
        if (trace_d) cudaFreeAsync(trace_d, st);
        if (owned) cudaFreeAsync(ws, st);
        return cs;
    }

    // ---- the iteration: Steps 2 and 3, with the next Step 1 fused ----
    const int chunk = tv_max_steps();
    const int chunks = ntv == 0 ? 1 : (ntv + chunk - 1) / chunk;
    int cur = (int)((k0 * chunks) & 1);
    // each kernel of the loop may be scheduled while its predecessor finishes
    // (programmatic dependent launch; it waits for it before any memory access)
    PdlScope pdl(true);
    for (int k = 0; k < prm->iters; ++k) {
        // Step 2: z = x^k - tau A^T mu_bar ; x^{k+1} = prox_{tau g}(z)
        backproject(mubar, z, 1, x_out);
        // equal chunks of at most tv_max_steps() steps
        int left = ntv;
        for (int c = chunks; c > 0; --c) {
            const int steps = (left + c - 1) / c;
            left -= steps;
            launch_tv(z, pbuf[cur], pbuf[cur ^ 1], x_out, g->n, g->n_sm, g->tune_tv, steps, c == 1, scal, st,
                      prm->tv_accel == 1);
            cur ^= 1;
        }
        // Step 3: A x^{k+1} (band partial sums); the dual update forms the
        // residual A x^{k+1} - b [- W^-1 mu^k] from them, applies D and also
        // performs Step 1 of the next iteration
        launch_project_bands(g, x_out, band, 1, st);
        if (trace_d)
            launch_trace(g, band, b, w, x_out, lowdose ? prm->beta : 0.0, lowdose, trace_d + prm->iters,
                         trace_d + k, st);
        if (epsf) cudaMemcpyAsync(r, mu, sizeof(float) * I, cudaMemcpyDeviceToDevice, st);   // mu^k
        if (sv_d) launch_dual_sv(g, hhat, hhat2, sv, band, b, mu, mubar, winv, scal, st);
        else if (use_fft) launch_dual_fft(g, hhat, band, b, mu, mubar, winv, lowdose, scal, st);
        else launch_dual_update(g, taps, half, band, b, mu, mubar, winv, lowdose, scal, st);
        // error-tolerant form: mu^{k+1} = the proximal map of Algorithm 2's
        // update, mu_bar = 2 mu^{k+1} - mu^k
        if (epsf)
            launch_eps_step(g, mu, mu, mubar, r, eQ, eLam, prm->eps, scal, aux, es, ew2, epart, st);
    }
    launch_scalars(scal, SC_SET, (double)(k0 + prm->iters), 0, 0, S_K, st);
    launch_check_finite(x_out, J, flags, CHK_NONFINITE_RESULT, st);
    launch_check_finite(mu, I, flags, CHK_NONFINITE_RESULT, st);   // x >= 0 clamps a diverged x, not mu
    cs = cuda_check("ct_pdtv_solve");
    if (report && cs == CT_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) cs = fail(CT_ERR_CUDA, "ct_pdtv_solve: %s", cudaGetErrorString(e));
        else {
            if (trace_d) {
                e = cudaMemcpy(trace_h, trace_d, sizeof(double) * prm->iters, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) cs = fail(CT_ERR_CUDA, "ct_pdtv_solve: trace: %s", cudaGetErrorString(e));
            }
            const ct_status rs = ctpd::read_report(ws, report);
            if (cs == CT_OK) cs = rs;
        }
    }
    if (trace_d) cudaFreeAsync(trace_d, st);
    if (owned) cudaFreeAsync(ws, st);
    return cs;
}
