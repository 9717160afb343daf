// ctpd_internal.cuh -- shared definitions of the CUDA path (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/ctpd.h"

namespace ctpd {

// Per-view constants of Joseph's projector, rounded once to float on the
// host from double-precision trig.  With h = (N-1)/2, hb = (B-1)/2, a view
// that steps along image rows crosses row r of ray d at the column
//     u(d, r) = h + (d - hb) * a + (r - h) * m,   a = 1/cos t, m = -sin t/cos t,
// and a column-stepping view crosses column c at the row
//     u(d, c) = h + (d - hb) * a + (c - h) * m,   a = 1/sin t, m = -cos t/sin t.
// Each step contributes the linear interpolation of the row (column) at u,
// and the ray sum is scaled by 1/|cos t| (1/|sin t|).
struct ViewP {
    float a;       // d coefficient
    float m;       // step coefficient
    float scale;   // path length per step, |a|
    float inv_a;   // 1/a (cos t or sin t), for the pixel->ray inverse map
    float inv_m;   // 1/m (0 when m = 0), for the ray->step range
    int rows;      // 1: steps along rows; 0: along columns
    int three;     // 1: a pixel's candidate-ray window can hold three rays
    int stride;    // view-pair projector: rays of one quarter warp are `stride` apart (bank spread)
};

struct Geometry {
    int n, n_views, n_bins, device;
    int n_fft;            // P = 2^ceil(log2(2B))
    int n_row, n_col;     // views stepping along rows / columns
    float win_eps;        // candidate-window margin (bins) of the backprojector
    ViewP *d_views;       // device, n_views entries
    int *d_row_list;      // device, the n_row row-stepping view indices
    int *d_col_list;      // device, the n_col column-stepping view indices
    float4 *d_trig;       // device, per view (cos t, sin t, |a|, 1 - |a|/2) for A^T
    float2 *d_tw;         // device, n_fft twiddles e^{-2 pi i k / P} (from double precision)
    int orbit;            // default angles with V and N even: A^T by rotation orbits
    int vpair;            // default angles: A by view pairs (v, V-v)
    int n_row_items, n_col_items;
    int2 *d_row_items;    // device, (v, V-v) for 1 <= v <= V/4, and (0, -1)
    int2 *d_col_items;    // device, (v, V-v) for V/4 < v < V/2, and (V/2, -1) for even V
    int n_sm;             // multiprocessors of the device
    // launch shapes chosen by ct_geometry_autotune (0: the built-in rule)
    int tune_pg;          // projector view items per block (4..16; 4..12 with 4 steps per pass)
    int tune_qrows;       // projector steps per pass of a ray walk (2 or 4)
    int tune_orb;         // A^T orbit base-view slices (1..8), slices added in a cluster
    int tune_orb_si;      // the same for the slice-image form (solves side by side, the persistent kernel)
    int tune_tv;          // fewest interior rows of a TV tile (4..64)
    int tune_qbal;        // projector form: 1 band pair per block, 2 work-balanced ranges (0: the rule)
    int qbal_occ[2][17];  // blocks per SM of the work-balanced projector by (4 steps per pass, items); 0: not queried
    long long *d_qbounds; // device, qbounds_nb + 1 entries: the work-balanced projector's unit ranges for one
                          // image, balanced by the tuner from measured block times (NULL: equal unit counts)
    int qbounds_nb;       // the launch they fit: blocks ...
    int qbounds_key;      // ... and 64 (4 steps per pass) + items per block
    unsigned long long *d_qtimes;   // device: the tuner's per-block start and end times while it measures
    double *h_angles;     // host copy
    void *eps_cache;      // eigenbases of D for the error-tolerant form (eps.cu)
    void *graph_cache;    // instantiated CUDA graphs of repeated solves (api.cu)
};

// Balances the work-balanced projector's unit ranges for one image by
// measuring its blocks (k_joseph.cu; the tuner calls it once it has chosen
// the launch shape): keeps g->d_qbounds when it makes the launch faster.
// x and band: an image and band partials of the geometry's size.
ct_status qbal_balance(Geometry *g, const float *x, float *band, cudaStream_t st);

// Records a printf-style message as the calling thread's last error.
void set_error(const char *fmt, ...);
// Copies the scalars of a finished solve out of its workspace (synchronous).
ct_status read_report(const void *workspace, ct_pdtv_report *report);

}  // namespace ctpd

// The opaque handle of the C ABI is the geometry itself.
struct ct_geometry : public ctpd::Geometry {};

namespace ctpd {
// Drops the geometry's cached solve graphs (api.cu); the tuning calls use it,
// as the graphs hold the old launch shapes.
void graph_cache_clear(Geometry *g);
// ct_pdtv_solve; allow_fork lets one solve run independent setup work on a
// second stream of the device (off for solves already run side by side).
// fork (optional): the Fork to put the setup's second branch on instead of
// the device's shared one.
ct_status pdtv_solve(const ct_geometry *g, const float *b, const float *w, const ct_pdtv_params *prm,
                     float *x_out, void *workspace, ct_pdtv_report *report, void *stream, bool allow_fork,
                     void *fork = nullptr);

// A side stream and two events for running independent work beside a
// caller's stream: fork_begin makes the side stream wait for the work
// enqueued so far on `st` and returns it; fork_end makes `st` wait for
// everything enqueued on the side stream.  Each record-and-wait pair runs
// under the Fork's lock, so calls from several host threads each wait on
// their own record.  Both are stream-ordered and can be captured.
struct Fork {
    bool ready = false;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    std::mutex mu;
};
inline cudaStream_t fork_begin(Fork *f, cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(f->mu);
    cudaEventRecord(f->fork, st);
    cudaStreamWaitEvent(f->s, f->fork, 0);
    return f->s;
}
inline void fork_end(Fork *f, cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(f->mu);
    cudaEventRecord(f->join, f->s);
    cudaStreamWaitEvent(st, f->join, 0);
}
// The device's shared Fork (created on first use, kept until exit; NULL if
// that fails or dev is outside [0, 64)).
Fork *fork_for(int dev);
}  // namespace ctpd

namespace ctpd {

// Joseph coordinate of the projector.  For ray d (dp = d - hb) the per-ray
// constant q = dp*a + (h - 1/2) is formed once, and at step s (sp = s - h)
// the coordinate u' = sp*m + q = u - 1/2.  Rounding u' to the nearest
// integer i0 gives floor(u) (ties pick either neighbour; the interpolated
// value is the same), and g = u' - i0 in [-1/2, 1/2] gives the weights
// 1/2 - g on pixel i0 and 1/2 + g on pixel i0 + 1 (the usual 1-f and f
// with f = g + 1/2).
__device__ __forceinline__ float joseph_hq(int n) { return __fsub_rn(0.5f * (float)(n - 1), 0.5f); }

__device__ __forceinline__ float joseph_q(float dp, float a, float hq) { return __fmaf_rn(dp, a, hq); }

__device__ __forceinline__ float joseph_u(float sp, float m, float q) { return __fmaf_rn(sp, m, q); }

// Round to nearest by the 1.5*2^23 bias (valid for |u'| < 2^22; callers
// keep u' inside a few image widths).  i0 = rounded value, g = u' - i0.
// The backprojector uses the same bias to find floor(e) of a pixel's
// detector coordinate.
constexpr float JOSEPH_BIAS = 12582912.0f;
constexpr int JOSEPH_BIAS_BITS = 0x4B400000;

__device__ __forceinline__ void joseph_round(float up, int &i0, float &g)
{
    const float t = __fadd_rn(up, JOSEPH_BIAS);
    i0 = __float_as_int(t) - JOSEPH_BIAS_BITS;
    g = __fsub_rn(up, __fsub_rn(t, JOSEPH_BIAS));
}

// The threads that run one kernel body: a whole one-dimensional thread
// block (a normal launch; sync = __syncthreads), or one fixed group of a
// persistent block (GroupCtx: its own named barrier `bar` (1..15) over nth
// threads).  Bodies are templates on the context type, so a normal launch
// pays nothing for the choice.
struct BlockCtx {
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
    __device__ __forceinline__ int nth() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct GroupCtx {
    int t, n, bar;
    __device__ __forceinline__ int tid() const { return t; }
    __device__ __forceinline__ int nth() const { return n; }
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(n) : "memory"); }
};
__device__ __forceinline__ BlockCtx whole_block() { return BlockCtx{}; }
// A whole two-dimensional block, threads numbered row by row.
struct Block2D {
    __device__ __forceinline__ int tid() const { return threadIdx.y * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int nth() const { return blockDim.x * blockDim.y; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Packed two-wide FP32 arithmetic of sm_100-family GPUs (fma / add / sub
// .rn.f32x2: two lanes per instruction, each rounded as its scalar form).
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    unsigned long long A, Bv, D;
    asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(Bv) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(Bv));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(D));
    return d;
}

// Device scalar block at the start of a solve workspace (doubles).
enum {
    S_KAPPA = 0, S_TAU, S_SIGMA, S_LAMBDA, S_INV8LAM, S_NADA, S_NWDW, S_K,
    S_RED0 = 16,   // reduction results
    S_LN0 = 24,    // norm of the first Lanczos vector (image side)
    S_LN0B = 25,   // and of the sinogram side
    S_EPSC = 26,   // u = 1 / c of the last proximal map of the error-tolerant form
    S_FLAGS = 27,  // input / result check bits (CHK_*), an unsigned in the slot's first 4 bytes
    S_PDONE = 28,  // persistent batched kernel: items of the slice's current task completed (unsigned)
    S_PQUEUE = 29, // persistent batched kernel, first slice only: slices finished (unsigned)
    S_PERR = 30,   // persistent batched kernel, first slice only: a wait ran out (unsigned)
    S_PSTATE = 31, // persistent batched kernel: current task << 32 | items handed out (64-bit)
    S_LZ = 32,     // Lanczos coefficients: alpha_j at S_LZ + 2j, beta_j at S_LZ + 2j + 1 (image side)
    S_LZ2 = 32 + 2 * 64,   // the same for the sinogram side
    S_COUNT = 32 + 4 * 64
};
constexpr int LANCZOS_MAX = 64;
// Bits of the S_FLAGS word (k_check.cu).
enum : unsigned {
    CHK_WEIGHT_NOT_POSITIVE = 1u,   // some w_i <= 0 (W of Eq. 1 must be positive definite)
    CHK_NONFINITE_INPUT = 2u,       // NaN or infinity in b or w
    CHK_NONFINITE_RESULT = 4u,      // NaN or infinity in the returned image or dual variable
    CHK_TIMEOUT = 8u                // a wait of the persistent batched kernel ran out
};
__host__ __device__ inline unsigned *flags_of(double *scal) { return reinterpret_cast<unsigned *>(scal + S_FLAGS); }
// Status of a finished solve from its flag word (CT_OK if none is set; the
// message names the first problem).
ct_status status_from_flags(unsigned flags, const char *who);
// Float copies of the scalars the per-iteration kernels read (doubles 20-21
// hold four floats; every scalar-program launch refreshes them), so those
// kernels convert nothing on the slow FP64 pipe.
constexpr int S_F32 = 20;
enum { F_TAU = 0, F_SIGMA, F_LAMBDA, F_INV8LAM };

// Neumaier-compensated FP32 sum: the running sum s and the rounding errors
// it dropped, c (value s + c).  The data-parallel reductions of the
// adjoint use it instead of FP64, which is slow on this GPU; with a fixed
// order of additions the result is deterministic.
struct FSum {
    float s, c;
};
__device__ __forceinline__ void fsum_add(FSum &a, float x)
{
    const float t = a.s + x;
    a.c += fabsf(a.s) >= fabsf(x) ? (a.s - t) + x : (x - t) + a.s;
    a.s = t;
}
__device__ __forceinline__ void fsum_merge(FSum &a, const FSum &b)
{
    fsum_add(a, b.s);
    a.c += b.c;
}
__device__ __forceinline__ float fscal(const double *scal, int k) { return reinterpret_cast<const float *>(scal + S_F32)[k]; }

// Number of kernels this library has enqueued (all threads), for callers
// that account for launches.
extern std::atomic<unsigned long long> g_launches;
extern thread_local unsigned long long t_launches;   // this thread's share of g_launches
inline void counted(unsigned n = 1)
{
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}

// Programmatic dependent launch.  A kernel launched with the
// programmatic-serialization attribute is launched as the blocks of its
// predecessor in the stream exit, before the predecessor's completion is
// signalled; pdl_wait() blocks until the predecessor has completed and its
// writes are visible, so it comes before the kernel's first global load or
// store.  Without the attribute it returns at once.  (The kernels do not
// signal their successors early: successor blocks scheduled while the last
// blocks of a kernel still run were measured slower in replayed graphs.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launches made through launch_kernel while a PdlScope is open on the
// calling thread carry the programmatic-serialization attribute (the solve
// loop, whose kernels each begin with pdl_wait()); otherwise launch_kernel
// is an ordinary launch.
extern thread_local int t_pdl;
struct PdlScope {
    int old;
    explicit PdlScope(bool on) : old(t_pdl) { t_pdl = on ? 1 : 0; }
    ~PdlScope() { t_pdl = old; }
};
template <class T>
struct same_type {
    using type = T;
};
template <typename... KArgs>
inline void launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          typename same_type<KArgs>::type... args)
{
    if (t_pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, kern, args...);
    } else {
        kern<<<grid, block, smem, st>>>(args...);
    }
}

// launch_kernel for a grid of thread-block clusters of `cluster` blocks
template <typename... KArgs>
inline void launch_kernel_cluster(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  dim3 cluster, typename same_type<KArgs>::type... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster.x;
    at[0].val.clusterDim.y = cluster.y;
    at[0].val.clusterDim.z = cluster.z;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = t_pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---- kernels (defined in the k_*.cu files) ----
// The persistent batched solve (persist.cu).  persistent_slice_ok: the slice
// qualifies (default angles with N, V even, N a multiple of 32 and at most
// 637, n_bins <= 4096, precond 0, 1 or 3, no eps, at most 16 prox steps,
// iters == iters0 > 0, no resume).  launch_persistent enqueues on st one
// persistent launch per 96 slices that runs all iterations of the slices,
// whose setup (and Step 1 at k = 0) must already be enqueued before it.
int batched_form();
bool persistent_slice_ok(const Geometry *g, const ct_pdtv_params *p, int iters0);
ct_status launch_persistent(int n, const ct_geometry *const *geoms, const float *const *b,
                            const ct_pdtv_params *params, float *const *x_out, void *const *workspaces,
                            cudaStream_t st);
// Launch shapes shared with the persistent batched kernel (persist.cu).
// base-view slices of the orbit backprojector: of its cluster form, or
// (cluster false) of its slice-image form
int orbit_slices(const Geometry *g, bool cluster = true);
size_t orbit_smem_bytes();                      // shared memory of one orbit block
bool quad_ok(const Geometry *g);                // the view-pair projector serves this geometry
// TV prox tiles of one image spread over n_sm blocks (k_tv.cu's rule)
void tv_tile_shape(int n, int steps, int n_sm, int min_rows, int *tc, int *tr, int *ncb, int *nrb, int rows = 0);
size_t dual_fft_smem(const Geometry *g);
// Device pointers into a solve workspace (api.cu's layout).
struct SolveBuffers {
    double *scal;
    float *winv, *mu, *mubar, *z, *p0, *p1, *band, *orb;
    float2 *hhat;
};
SolveBuffers solve_buffers(const Geometry *g, const ct_pdtv_params *prm, void *workspace);
// Input and result checks, and the per-iteration trace (k_check.cu).
void launch_check_inputs(const float *b, const float *w, size_t n, unsigned *flags, cudaStream_t st);
void launch_check_finite(const float *x, size_t n, unsigned *flags, unsigned bit, cudaStream_t st);
size_t trace_scratch_doubles();
// *out = beta psi(x) + 1/2 sum w (A x - b)^2 (lowdose) or ||A x - b|| (A x
// given as the projector's band partial sums of one slice); part holds
// trace_scratch_doubles() doubles
void launch_trace(const Geometry *g, const float *partial, const float *b, const float *w, const float *x,
                  double beta, int lowdose, double *part, double *out, cudaStream_t st);
// Forward projection in two parts: band partial sums (one image band of
// PROJ_R rows / columns per block, deterministic) and their reduction.
// partial holds n_bands(N) x V x B floats per image.
constexpr int PROJ_R = 32;
inline int proj_bands(int n) { return (n + PROJ_R - 1) / PROJ_R; }
void launch_project_bands(const Geometry *g, const float *x, float *partial, int batch, cudaStream_t st);
// out = scale_v * sum_b partial[b]   (mode 0), minus b and winv*mu (mode 1),
// minus b (mode 2).
void launch_band_reduce(const Geometry *g, const float *partial, float *out, int mode,
                        const float *b, const float *winv, const float *mu, int batch,
                        cudaStream_t st);
// Backprojection; mode 0: out = A^T y; mode 1: out = xin - tau*A^T y with
// tau = (float)scal[S_TAU].  The orbit form adds its base-view slices in a
// thread-block cluster (cluster, or partial NULL), or through slice images
// in `partial` (orbit_partial_floats() floats) and a reduction pass: the
// form for solves run side by side, whose clusters would wait for a GPC's
// SMs to free together.
bool orbit_ok(const Geometry *g);
size_t orbit_partial_floats(const Geometry *g, int batch);
bool orbit_slices_ok(const Geometry *g, int nsl);
void launch_backproject_orbit(const Geometry *g, const float *y, float *out, int mode, const float *xin,
                              const double *scal, int batch, float *partial, cudaStream_t st, bool cluster = true);
void launch_backproject(const Geometry *g, const float *y, float *out, int mode,
                        const float *xin, const double *scal, int batch, cudaStream_t st);

// Filter: out = post .* (D (pre .* in)) * (scal ? -sigma : 1); pre/post
// may be NULL.  mode 0 plain, 1 "-sigma D in" (start of the iteration).
void launch_filter(const Geometry *g, const float *taps, int half, const float *in,
                   float *out, const float *pre, const float *post, int mode,
                   const double *scal, int batch, cudaStream_t st);
// Fused Step 3 + next Step 1 for one iteration, per view:
//   mu' = mu + sigma D r;  mu_bar = 2 mu' - mu [- sigma D (winv .* (mu' - mu))].
// The residual r = A x - b [- winv mu] is formed from the projector's band
// partial sums while the view is loaded.
void launch_dual_update(const Geometry *g, const float *taps, int half, const float *partial,
                        const float *b, float *mu, float *mu_bar, const float *winv, int lowdose,
                        const double *scal, cudaStream_t st);
void launch_taps(const Geometry *g, int mode, const double *scal, double tau, double kappa,
                 float *taps, cudaStream_t st);

// Frequency-domain D (k_fft.cu), for n_fft <= FFT_MAX_P.
constexpr int FFT_MAX_P = 8192;
bool fft_supported(const Geometry *g);
// hhat (n_fft complex) = DFT of the taps placed circularly
void launch_hhat(const Geometry *g, const float *taps, int half, float2 *hhat, cudaStream_t st);
// out = post .* D(pre .* in) * (mode 1 ? -sigma : 1)
void launch_filter_fft(const Geometry *g, const float2 *hhat, const float *in, float *out,
                       const float *pre, const float *post, int mode, const double *scal, int batch,
                       cudaStream_t st);
// out = D (A x) with A x given as the projector's band partial sums
void launch_filter_fft_bands(const Geometry *g, const float2 *hhat, const float *partial, float *out, int batch,
                             cudaStream_t st);
// fused residual + Step 3 + next Step 1 (as launch_dual_update)
void launch_dual_fft(const Geometry *g, const float2 *hhat, const float *partial, const float *b, float *mu,
                     float *mu_bar, const float *winv, int lowdose, const double *scal, cudaStream_t st);
// The shift-variant preconditioner D = T_lo + S T_hi S (k_fft.cu; low-dose,
// FFT path).  hs, hd (n_fft complex each) = (H_lo +- H_hi) / 2 from the band
// taps; sv = s (V x B), s_i = sqrt(kappa w_i).
void launch_sv_hhat(const Geometry *g, const float *taps_lo, const float *taps_hi, int half, float2 *hs, float2 *hd,
                    cudaStream_t st);
void launch_filter_sv(const Geometry *g, const float2 *hs, const float2 *hd, const float *sv, const float *in,
                      float *out, const float *pre, const float *post, int mode, const double *scal, int batch,
                      cudaStream_t st);
void launch_filter_sv_bands(const Geometry *g, const float2 *hs, const float2 *hd, const float *sv,
                            const float *partial, float *out, int batch, cudaStream_t st);
void launch_dual_sv(const Geometry *g, const float2 *hs, const float2 *hd, const float *sv, const float *partial,
                    const float *b, float *mu, float *mu_bar, const float *winv, const double *scal,
                    cudaStream_t st);
// s = sqrt(kappa w), kappa = scal[S_KAPPA]
void launch_sv_scale(const float *w, const double *scal, float *s, size_t n, cudaStream_t st);
// out[i] = +-1 from an integer hash of i (the Lanczos start vector)
void launch_fill_sign(float *out, size_t n, cudaStream_t st);
void kernel_attrs_fft();
void launch_dual_fft_batched(const Geometry *g, const float2 *hhat, const float *partial, const float *b,
                             const float *mu_in, float *mu_out, float *mu_bar, const float *winv, int lowdose,
                             const double *scal, int batch, cudaStream_t st);
void launch_dual_bwd_fft(const Geometry *g, const float2 *hhat, const float *partial, const float *b,
                         const float *winv, const float *mu, const float *mu1, const float *gm, const float *gmb,
                         float *gmu, float *gr, float *gm1, float *r, float *v, int lowdose, const double *scal,
                         int batch, cudaStream_t st);

// Reductions of the adjoint (k_grad.cu).
// acc[half - 1 + k] += c0 <g0, T_k s0> + c1 <g1, T_k s1> over nviews rows of B
// bins (T_k: shift by k, |k| < half); g1 = NULL drops the second pair.  acc
// holds compensated sums (value x + y, see FSum).
size_t tapcorr_partial_bytes(int nviews, int B, int half);
void launch_tapcorr_acc(const float *g0, const float *s0, double c0, const float *g1, const float *s1, double c1,
                        int nviews, int B, int half, float *partial, float2 *acc, cudaStream_t st);
void kernel_attrs_grad();
void launch_grad_out(const float2 *acc, int nl, const double *scal, int slot, double fac, float *grad,
                     cudaStream_t st);
// out = fac[0] * scale_v * sum_b partial[b]
void launch_band_reduce_scaled(const Geometry *g, const float *partial, float *out, const double *fac, int batch,
                               cudaStream_t st);

// Whole-image TV steps and their adjoints (k_tv.cu), batched over images.
size_t tv_px_blocks(int n, int batch);
void launch_tv_step(const float *z, const float *p_in, float *p_out, int n, int batch, const double *scal,
                    cudaStream_t st);
void launch_tv_final(const float *z, const float *p, float *x, int n, int batch, const double *scal, cudaStream_t st);
// The adjoints write their block sums of the inv8 and lambda derivative
// terms as pairs into part[tv_px_blocks] (floats; the final step's inv8
// terms are 0); launch_pair_sums adds the pairs of many launches into two
// scalar slots, deterministically (scratch: pair_sums_scratch_floats()).
void launch_tv_final_bwd(const float *z, const float *p, const float *gx, const float *gp_next, float *gz,
                         float *gp, int n, int batch, const double *scal, float *part, cudaStream_t st);
void launch_tv_step_bwd(const float *z, const float *p, const float *gp_next, float *gz, float *gp, int n,
                        int batch, const double *scal, float *part, cudaStream_t st);
size_t pair_sums_scratch_floats();
void launch_pair_sums(const float *part, size_t npairs, float *scratch, double *scal, int slot_a, int slot_b,
                      cudaStream_t st);

// TV prox of Eq. 17 with x >= 0 (projected-gradient dual steps, warm-started
// dual field p = (px, py)), temporally blocked tiles held in registers.
// Runs `steps` <= tv_max_steps() dual steps reading p_in and writing p_out;
// when final != 0 also writes x = max(0, z + lam div p).  n_sm (the
// device's SM count) and min_rows (fewest interior rows per tile, 0: the
// default) size the tiles.
// batch > 1 runs that many images (z, x: n x n each; p: 2 n x n each);
// traj, when not NULL (plain projected-gradient steps), receives p after each of the first
// steps - 1 steps: step l + 1 at traj + (l * batch + image) * 2 n n.
void launch_tv(const float *z, const float *p_in, float *p_out, float *x,
               int n, int n_sm, int min_rows, int steps, int final, const double *scal, cudaStream_t st,
               bool fgp = false, int batch = 1, float *traj = nullptr);
int tv_max_steps();

// The error-tolerant few-view form (eps.cu).  toeplitz_eig: FP64 host
// eigendecomposition of T[i][j] = t[|i - j|].  eps_basis: D's eigenbasis
// (Q as B x B row-major floats, lambda) for a geometry, precond and tau,
// computed from the device taps (2B - 1 values) on first use and cached.
// launch_eps_step: out = the proximal map of q (see eps.cu), out2 (may be
// NULL) = 2 out - mu0; Q = NULL means D = I.  wbuf: V x B floats, s and w2:
// B floats each, part: eps_partial_floats(g) floats.
bool toeplitz_eig(const double *t, int n, double *q, double *lambda);
ct_status eps_basis(const Geometry *g, int precond, double tau_key, const float *taps, cudaStream_t st,
                    const float **q, const float **lambda);
void eps_cache_free(Geometry *g);
// whether eps_basis has the basis already (so a solve needs no host step)
bool eps_basis_ready(const Geometry *g, int precond, double tau_key);
size_t eps_partial_floats(const Geometry *g);
void launch_eps_step(const Geometry *g, const float *q, float *out, float *out2, const float *mu0, const float *Q,
                     const float *lambda, double eps, double *scal, float *wbuf, float *s, float *w2, float *part,
                     cudaStream_t st);

// Small helpers
void launch_fill(float *p, float v, size_t n, cudaStream_t st);
void launch_recip(const float *w, float *winv, size_t n, cudaStream_t st);
void launch_sqrt(const float *a, float *out, size_t n, cudaStream_t st);
void launch_scale_by(const float *in, const float *s, int sqrt_s, float *out, size_t n, cudaStream_t st);
// scal[slot] = sum(a .* b) (b may be NULL: sum(a)), deterministic two-pass.
void launch_dot(const float *a, const float *b, size_t n, double *scal, int slot,
                double *partials, cudaStream_t st);
// scalar program: set tau/sigma/lambda from norms and parameters
void launch_scalars(double *scal, int op, double a0, double a1, double a2, int i0,
                    cudaStream_t st);
enum { SC_KAPPA_FROM_SUM = 0, SC_TAU, SC_NORM_FROM_DOT, SC_SIGMA, SC_LAMBDA, SC_SET, SC_COPY,
       SC_NORM_SQRT, SC_AXPY_SLOT };
// scal[out] = largest eigenvalue of the Lanczos tridiagonal of k steps with
// coefficients at scal[base ..]
void launch_lanczos_max(double *scal, int base, int k, int out, cudaStream_t st);
// One half (phase 0 / 1) of a Lanczos step on unnormalised vectors: w holds
// op(t_j), tp = t_{j-1}, tc = t_j; coefficients at scal[base ..], the norm of
// t_0 at scal[n0slot].  partials: dot_partials_doubles(); ticket: a
// zero-initialised counter (left at zero).
void launch_lanczos_step(float *w, const float *tp, const float *tc, size_t n, double *scal, int base, int n0slot,
                         int j, int phase, double *partials, unsigned *ticket, cudaStream_t st);
// w -= scal[slot] * q
void launch_axpy_neg(float *w, const float *q, size_t n, const double *scal, int slot, cudaStream_t st);

size_t dot_partials_doubles();
void kernel_attrs_filter();
void kernel_attrs_tv();
void kernel_attrs_joseph();

}  // namespace ctpd
