/*
 * ctpd.h -- C ABI of libctpd.so: ramp-filter-preconditioned first-order
 * primal-dual TV reconstruction for 2-D parallel-beam CT on one GB300 GPU
 * (Kudo, Yamazaki, Nemoto, Takaki, arXiv 1609.06041).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Geometry (Sec. 2.1: "standard parallel-beam geometry", uniform samples of
 * p(r, theta)).  Unit pixels and unit detector bins.
 *   image     x[r*N + c], float32, row-major; pixel (r, c) has centre
 *             (c - (N-1)/2, r - (N-1)/2).
 *   sinogram  s[v*B + d], float32, view-major; bin d of view v is the line
 *             x cos(t_v) + y sin(t_v) = d - (B-1)/2.
 *   angles    t_v = v*pi/V by default (V views over 180 degrees, m = V in
 *             Eq. 24 and Eq. 32).
 *   batches   `batch` images / sinograms stored back to back; batch = 0 is
 *             a no-op, 0 <= batch <= 65535.
 * A (the system matrix of Eq. 1) is Joseph's ray-driven interpolation: a
 * view with |cos t| >= |sin t| (default angles: 4v <= V or 4v >= 3V) steps
 * along image rows, interpolating each row linearly at the ray's column and
 * weighting by 1/|cos t|; other views step along columns with 1/|sin t|.
 * ct_backproject applies the transpose: each weight 1 - |d - e| / max(|cos t|,
 * |sin t|) is evaluated from the pixel side (e = the pixel centre's detector
 * coordinate), equal to A's weight in exact arithmetic and to within the
 * float rounding of the coordinates (about 2^-24 times the image size) in
 * practice.
 *
 * Memory.  Every float pointer argument is a DEVICE pointer owned by the
 * caller (for example torch tensor storage), contiguous, 16-byte aligned;
 * the library never frees it.  Host pointers are marked "host".  A
 * geometry handle owns a few KB of device memory (per-view constants) on
 * the device that was current at creation; use it on that device only.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Calls enqueue work and return without synchronising,
 * except where stated.  Inputs must stay valid until the work completes.
 *
 * Errors.  Every entry point returns a ct_status and never aborts or
 * throws.  CT_ERR_ARG: a bad size, NULL pointer, or unsupported option (no
 * work enqueued).  CT_ERR_CUDA / CT_ERR_OOM: a CUDA call failed (the
 * stream may hold partial work).  ct_last_error() gives a message for the
 * calling thread.
 */
#ifndef CTPD_H
#define CTPD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CT_OK = 0,
    CT_ERR_ARG = 1,
    CT_ERR_CUDA = 2,
    CT_ERR_OOM = 3,
    CT_ERR_TIMEOUT = 4,
    CT_ERR_NONFINITE = 5
} ct_status;

enum { CT_LOWDOSE = 0, CT_FEWVIEW = 1 };
/* Band taps of the shift-variant preconditioner (ct_ramp_taps modes). */
enum { CT_TAPS_LOW_BAND = 2, CT_TAPS_HIGH_BAND = 3 };

typedef struct ct_geometry ct_geometry;

/* Library version, e.g. "ctpd 0.1 sm_103a". */
const char *ct_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *ct_last_error(void);

/* Kernels enqueued by this library so far (all threads), for launch
 * accounting; never decreases. */
unsigned long long ct_kernel_launches(void);

/*
 * Measured FP32 FMA throughput of the current device in TFLOP/s (*tflops,
 * host), the denominator of the roofline fraction of the FMA-carrying
 * operators.  No counterpart in the paper: a fixed kernel of independent
 * FMA chains (packed = 0: fma.rn.f32; 1: the packed fma.rn.f32x2, two FMAs
 * per instruction) over 8 blocks of 256 threads per SM, timed with CUDA
 * events on `stream` (best of three after one warm-up launch).
 * Synchronises the stream; allocates a small stream-ordered buffer.
 */
ct_status ct_probe_fp32_fma(int packed, double *tflops, void *stream);

/*
 * Create a 2-D parallel-beam geometry (Sec. 2.1): N x N image, V views,
 * B bins.  angles (host, V doubles, radians) may be NULL for t_v = v*pi/V.
 * 1 <= N, V, B <= 8192.  On success *out receives a handle; destroy it with
 * ct_geometry_destroy.  Allocates and fills a small device table on the
 * current device (synchronous).
 */
ct_status ct_geometry_create(int n, int n_views, int n_bins,
                             const double *angles, ct_geometry **out);
void ct_geometry_destroy(ct_geometry *geom);

/*
 * Launch-shape tuning (no counterpart in the paper: it picks how the work of
 * A, A^T and the TV prox of Eq. 17 is cut into thread blocks, never what is
 * computed).  Five shapes are held by the geometry:
 *   items_per_block  view pairs (v, V-v) sharing one staged band pair in the
 *                    projector, 64 threads each (4..16; 4..12 when
 *                    proj_rows is 4);
 *   proj_rows        steps a projector thread evaluates per pass of a ray
 *                    walk (2 or 4: more loads in flight, more registers;
 *                    the same sums either way);
 *   orbit_slices     base-view slices of the rotation-orbit backprojector
 *                    (1..8, at most 1024 base views per slice), added in a
 *                    thread-block cluster of the slices' blocks, or (solves
 *                    run side by side in the batched form) through one
 *                    partial image each; the tuner picks the count for each
 *                    of the two forms, this call sets both and the getter
 *                    returns the first;
 *   tv_rows          fewest interior rows of a TV prox tile (4..64);
 *   proj_form        how the projector's work is cut into blocks (1 or 2):
 *                    1, each block stages one band pair and walks a few
 *                    groups of items_per_block items on it, the grid sized
 *                    by a wave-count model; 2, the work is cut into units
 *                    (band pair, item, 64 rays) and each block, with
 *                    64 x items_per_block threads, takes an equal range of
 *                    them, as many blocks as fit on the device at once,
 *                    its warps taking the units of each staged band pair
 *                    from a shared counter.  Both give the same sums.
 * 0 selects the built-in rule (a wave-count model for items_per_block, 2
 * steps per pass, 4 slices, 16 rows; form 2 with 16 items' threads when
 * form 1 would need two waves of blocks or more, else form 1).  The
 * projector's shapes (items_per_block, proj_rows, proj_form) and tv_rows
 * leave every result bit unchanged; orbit_slices changes the order in
 * which the backprojector's slice sums are added, so results can differ in
 * the last float bits between slice counts; for one shape they are
 * deterministic.
 *
 * ct_geometry_autotune times every candidate of each shape on synthetic data
 * of the geometry's size (batch images for A and A^T) on `stream`, with
 * CUDA events, and stores the fastest; when it picks proj_form 2 it also
 * balances that form's unit ranges for single-image launches from measured
 * block times (a table the geometry keeps for that launch shape; it moves
 * work between blocks and leaves every result bit unchanged).  It allocates and frees device
 * memory and synchronises the stream: call it before capturing a graph and
 * not while other calls use the geometry.  On error the previous shapes
 * are kept.  Errors: CT_ERR_ARG (NULL geometry, batch outside [1, 64]),
 * CT_ERR_OOM, CT_ERR_CUDA.
 * ct_geometry_set_tuning validates and stores shapes (CT_ERR_ARG when one is
 * out of range); ct_geometry_get_tuning reads them (NULL outputs skipped).
 */
ct_status ct_geometry_autotune(ct_geometry *geom, int batch, void *stream);
ct_status ct_geometry_set_tuning(ct_geometry *geom, int items_per_block, int proj_rows, int orbit_slices,
                                 int tv_rows, int proj_form);
ct_status ct_geometry_get_tuning(const ct_geometry *geom, int *items_per_block, int *proj_rows,
                                 int *orbit_slices, int *tv_rows, int *proj_form);

/*
 * Forward projection sino = A img (A of Eq. 1; Joseph interpolation).
 * img: batch x N x N, sino: batch x V x B (overwritten).
 */
ct_status ct_project(const ct_geometry *geom, const float *img, float *sino,
                     int batch, void *stream);

/*
 * The forward projection's band partial sums, the form in which the solve
 * takes Step 3's A x^{k+1} (Eq. 20) before the dual step adds them: the
 * image lines (rows for views stepping along rows, columns otherwise) are
 * cut into ct_project_bands_count(geom) bands (32 lines each, paired by
 * the image's mirror symmetry), and partial[b][v][d] holds the Joseph
 * samples of ray (v, d) in band b, summed in step order, before the
 * per-view path length |a_v| = 1 / max(|cos t_v|, |sin t_v|) is applied:
 *     sino[v][d] = |a_v| sum_b partial[b][v][d]      (ct_project adds the
 * bands in b order).  img: batch x N x N; partial: batch x n_bands x V x B
 * floats (device, caller-owned, overwritten; 16-byte aligned).  The launch
 * is the projector kernel alone, with no scratch allocation.  Errors:
 * CT_ERR_ARG (NULL or unaligned pointer, batch outside [0, 65535]).
 */
int ct_project_bands_count(const ct_geometry *geom);
ct_status ct_project_bands(const ct_geometry *geom, const float *img, float *partial,
                           int batch, void *stream);

/*
 * Backprojection img = A^T sino (the A^T of Eq. 19), a pixel-driven gather
 * over the two rays around each pixel's detector coordinate; deterministic
 * and free of atomics.  sino: batch x V x B, img: batch x N x N (overwritten).
 */
ct_status ct_backproject(const ct_geometry *geom, const float *sino, float *img,
                         int batch, void *stream);

/*
 * Taps of the preconditioner D = F^-1 H F applied along the detector axis
 * of every view: mode CT_LOWDOSE the smoothed ramp H = |w|/(2 m tau +
 * kappa |w|) (Eq. 24), mode CT_FEWVIEW the ramp H = |w|/(2 m tau) (Eq. 32),
 * m = V.  The discrete filter is the linear convolution over the detector
 * with t[k] = (1/P) sum_j H(w_j) cos(2 pi j k / P), |k| <= B-1, on the
 * period P = 2^ceil(log2(2B)), w_j = 2 pi min(j, P-j)/P.  taps (device,
 * 2B-1 floats) receives t[-(B-1)] .. t[B-1] (centre at index B-1).
 * Modes CT_TAPS_LOW_BAND and CT_TAPS_HIGH_BAND give the two bands of the
 * shift-variant preconditioner (see ct_ramp_filter_split), which add up to
 * the CT_LOWDOSE taps:
 *     H_lo = 2 m tau |w| / (2 m tau + kappa |w|)^2,  H_hi = kappa w^2 / (2 m tau + kappa |w|)^2.
 * tau > 0, kappa >= 0 (kappa ignored for CT_FEWVIEW).
 */
ct_status ct_ramp_taps(const ct_geometry *geom, int mode, double tau, double kappa,
                       float *taps, void *stream);

/*
 * Per-view linear convolution out[v][d] = sum_e taps[half-1 + d - e] in[v][e]
 * (the D of Eqs. 18-20 and 29-31), zero beyond the detector edges.
 * taps: device, 2*half_len-1 floats centred at half_len-1, 1 <= half_len <= B.
 * in, out: batch x V x B; in == out is not allowed.
 */
ct_status ct_ramp_filter(const ct_geometry *geom, const float *taps, int half_len,
                         const float *in, float *out, int batch, void *stream);

/*
 * The shift-variant preconditioner: out = T_lo in + s .* T_hi (s .* in), per
 * view, with T_lo, T_hi the linear convolutions with taps_lo and taps_hi
 * (layout as ct_ramp_filter) and s elementwise.  Sec. 5 reports that a
 * shift-variant preconditioner approximating D = (tau A A^T + W^-1)^-1
 * (Eq. 23) better than Eq. 24 improves the low-dose iteration, without
 * giving its form; this is the project's form: with the band taps of
 * ct_ramp_taps and s_i = sqrt(kappa w_i) it tends to the pure ramp of Eq. 32
 * at low frequency and to W = diag(w) at high frequency, the two limits of
 * Eq. 23, and equals Eq. 24 when all w_i = 1/kappa.  It is symmetric
 * positive definite, so the iteration keeps its limit (Sec. 2.2).
 * s: device, V x B floats (one slice; the same s for every batch image).
 * in, out: batch x V x B, in == out not allowed.  Needs n_bins <= 4096 (an
 * FFT of at most 8192 points); CT_ERR_ARG otherwise.  Allocates two
 * frequency responses of n_fft complex values from the stream-ordered
 * allocator and frees them after use (CT_ERR_OOM if that fails).
 */
ct_status ct_ramp_filter_split(const ct_geometry *geom, const float *taps_lo, const float *taps_hi, int half_len,
                               const float *s, const float *in, float *out, int batch, void *stream);

/*
 * ct_ramp_filter without any device memory allocation.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory while they run: for example a caller that reserves all of
 * its memory at start-up and must not touch the allocator afterwards, or
 * one that calls from a context where an allocation (which can block or
 * fail under memory pressure) is not acceptable.
 *
 * Same arguments and result as ct_ramp_filter.  Instead of a scratch
 * buffer from the allocator it uses one fixed device array of 8192 complex
 * values (64 KiB) that every GPU which loads the library holds until the
 * process exits, so it supports n_bins <= 4096 (a transform of at most
 * 8192 points); larger geometries return CT_ERR_ARG with a message.
 * The first call on a device looks up that array's device address (a
 * synchronous runtime query); make that first call before any stream
 * capture.  All calls share the array and each call overwrites all of its
 * contents, so calls whose work may overlap on the GPU (other streams,
 * other threads) race with each other: serialise them.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  The geometry's device
 * must be the current device (CT_ERR_ARG otherwise).
 */
ct_status ct_ramp_filter_noalloc(const ct_geometry *geom, const float *taps, int half_len,
                                 const float *in, float *out, int batch, void *stream);

/*
 * Eigendecomposition of the n x n symmetric Toeplitz matrix T[i][j] =
 * t[|i - j|] (host memory, FP64, no GPU work): q (n x n, row-major) gets
 * the unit eigenvectors as columns, lambda[j] the eigenvalue of column j,
 * in no particular order.  The matrix of the per-view convolution D with
 * taps of half length h is t[k] = taps[h - 1 + k] for k < h, 0 beyond.
 * Used by the error-tolerant few-view form (ct_pdtv_params.eps); exported
 * for checking.  Householder tridiagonalisation and implicit QR steps on
 * the two half-size problems of T's symmetric and antisymmetric
 * eigenvectors.  CT_ERR_ARG for NULL pointers or n < 1; CT_ERR_NONFINITE
 * if the QR steps do not converge.
 */
ct_status ct_sym_toeplitz_eig(const double *t, int n, double *q, double *lambda);

/* Parameters of ct_pdtv_solve (zero-initialise, then set what you need). */
typedef struct {
    int mode;         /* CT_LOWDOSE: Algorithm 1 (beta > 0) / 1' (beta = 0);
                         CT_FEWVIEW: Algorithm 2 (beta ignored, Sec. 3)      */
    int iters;        /* outer iterations to run (>= 0)                       */
    int tv_iters;     /* inner projected-gradient steps of the TV prox (Eq. 17),
                         0 -> 10; warm-started across outer iterations       */
    int precond;      /* 1: ramp preconditioner D (Eq. 24 / Eq. 32);
                         0: D = I (the unpreconditioned iteration);
                         2: the shift-variant D of ct_ramp_filter_split with
                            s = sqrt(kappa w) (CT_LOWDOSE, n_bins <= 4096);
                         3: few-view smoothed ramp, the form of Eq. 24 with
                            kappa = tau l, l = (2/3)(N^2/B) mean_v |a_v| the
                            mean diagonal of A A^T (CT_FEWVIEW): Eq. 32 adds
                            the same-view part of A A^T that sparse views
                            leave out of 2m/|w|                              */
    int norm_iters;   /* Lanczos steps for the operator norms of the automatic
                         sigma (0 -> 12, at most 64); the estimate is the
                         Ritz value plus its residual norm, from a +-1 start */
    int resume;       /* 1: continue from the state held in `workspace`       */
    double beta;      /* TV weight of Eq. 1 (low-dose)                         */
    double tau;       /* primal step; <= 0: low-dose pi*kappa/(2m) with
                         kappa = mean(1/w) (Eq. 24), few-view 0.01            */
    double sigma;     /* dual step; <= 0: rho * the bound of the Alg. 1 / Alg. 2
                         box from Lanczos estimates of the operator norms     */
    double rho;       /* safety factor for the automatic sigma (0 -> 0.95)    */
    int tv_accel;     /* prox of Eq. 17: 0 projected gradient on the dual
                         field; 1 its fast form (Beck-Teboulle FGP: Nesterov
                         momentum, restarted every outer iteration;
                         tv_iters <= 16)                                      */
    double eps;       /* CT_FEWVIEW only: > 0 solves the error-tolerant form of
                         Sec. 5, min TV(x) s.t. ||Ax - b|| <= eps, x >= 0:
                         Step 3 (and Step 1 at k = 0) take the proximal map
                         nu = argmin sigma eps |nu| + 1/2 |nu - q|^2_{D^-1} of
                         Algorithm 2's update q, i.e. (I + c D) nu = q with
                         c = sigma eps / |nu|, or nu = 0 when
                         |D^-1 q| <= sigma eps.  precond 0, 1 or 3 and
                         n_bins <= 4096.  With precond 1 or 3 the map runs in
                         the eigenbasis of D's B x B Toeplitz matrix: the first
                         solve for a geometry, precond and tau copies the taps
                         to the host, synchronises the stream once, computes
                         the FP64 eigendecomposition (cached in the geometry;
                         that solve cannot be captured in a CUDA graph, later
                         ones with the same precond and tau can).  0: the
                         equality form (Eq. 25).                              */
} ct_pdtv_params;

/* Scalars of a solve, copied to the host at the end when requested.  The
 * caller sets `trace` before the call (zero-initialise the struct first);
 * the solve fills the other fields. */
typedef struct {
    double tau, sigma, kappa, lambda;  /* lambda = tau*beta (Alg. 1), tau (Alg. 2) */
    double norm_ADA;   /* ||A^T D A|| = ||D^1/2 A A^T D^T/2||                    */
    double norm_WDW;   /* ||W^-1/2 D W^-1/2|| = ||D^1/2 W^-1 D^T/2|| (low-dose)   */
    int k;             /* iterations done in total (including resumed ones)      */
    double *trace;     /* host, params->iters doubles, or NULL (no trace).  After
                          iteration i of this call: CT_LOWDOSE the cost of Eq. 1,
                          f(x) = beta TV(x) + 1/2 ||Ax - b||_W^2 (with its 1/2),
                          CT_FEWVIEW the residual ||Ax - b|| of the constraint of
                          Eq. 25, both at x = x^{k+1} (one device reduction per
                          iteration over the projector's partial sums; a stream-
                          ordered buffer of iters + 608 doubles is allocated for
                          the call)                                             */
} ct_pdtv_report;

/* Device workspace (bytes) a solve with these parameters needs. */
size_t ct_pdtv_workspace_bytes(const ct_geometry *geom, const ct_pdtv_params *params);

/*
 * Ramp-preconditioned primal-dual TV reconstruction: Algorithm 1 / 1'
 * (low-dose, min_{x>=0} beta TV(x) + 1/2 ||Ax - b||_W^2, Eq. 1) or
 * Algorithm 2 (few-view, min TV(x) s.t. Ax = b, x >= 0, Eq. 25), iteration
 * for iteration as boxed in the paper:
 *   Step 1  mu_bar = -sigma D b (k = 0), else 2 mu^k - mu^{k-1}
 *           [- sigma D W^-1 (mu^k - mu^{k-1}) for Algorithm 1]
 *   Step 2  x^{k+1} = prox_{tau g}(x^k - tau A^T mu_bar)
 *   Step 3  mu^{k+1} = mu^k + sigma D (A x^{k+1} - b [- W^-1 mu^k])
 * b: V x B line integrals.  w: V x B statistical weights W = diag(w), w > 0
 * (CT_LOWDOSE; NULL for CT_FEWVIEW).  x_out: N x N, receives x^K (with
 * params->resume it must hold the x of the resumed state).
 * b, w and x_out are device memory or page-locked host memory (pageable
 * host memory: CT_ERR_ARG).  Host buffers are copied stream-ordered
 * through a staging area of the workspace: b and w (and x_out with resume)
 * before the solve, x^K into a host x_out after it, which then holds it
 * once the stream has reached that copy (before the call returns when a
 * report is asked for).
 * Input checks: b and w live on the device, so a device pass checks them
 * (w > 0 and finite, b finite) and the result (x^K and mu^K finite) and records what
 * it finds in the workspace.  The result comes back at the next
 * synchronisation the caller asks for: with a report this call returns
 * CT_ERR_ARG (some w_i <= 0) or CT_ERR_NONFINITE (NaN or infinity in b, w,
 * x^K or mu^K) after filling the report; without one, ct_pdtv_status(workspace,
 * stream) returns the same codes.  The solve itself still runs (its image
 * is then not meaningful).
 * workspace: device memory of ct_pdtv_workspace_bytes(); it holds the whole
 * iteration state (mu, mu_bar, TV dual field, scalars), so a later call
 * with resume = 1 continues exactly.  workspace == NULL: the library
 * allocates it stream-ordered and frees it at the end (no resume).
 * report (host, may be NULL): filled after the stream has been synchronised
 * (the only synchronising path of this call).
 * The call enqueues only device work (no host round trip), so it can be
 * captured into a CUDA graph when workspace and report are non-NULL / NULL.
 * Such a call (workspace given, report NULL, resume 0; with eps > 0 once an
 * earlier solve has computed D's eigenbasis) is also captured by the
 * library itself: the first call with a geometry, b, w,
 * x_out, workspace, stream and parameters records the whole solve as a CUDA
 * graph and launches it; later identical calls launch that graph (one
 * launch instead of some 280).  The graph reads the buffers when it runs,
 * so new contents of the same buffers are solved as usual.  Per geometry
 * the 16 most recently used graphs are kept until ct_geometry_destroy.
 * Inside a caller's stream capture, and with the environment variable
 * CTPD_SOLVE_GRAPHS=0, the kernels are launched directly instead.
 */
ct_status ct_pdtv_solve(const ct_geometry *geom, const float *b, const float *w,
                        const ct_pdtv_params *params, float *x_out,
                        void *workspace, ct_pdtv_report *report, void *stream);

/*
 * Result of the input and result checks of the last solve that used this
 * workspace (caller-owned, device): synchronises `stream` and returns
 * CT_OK, CT_ERR_ARG (a weight w_i <= 0: W of Eq. 1 is not positive
 * definite), or CT_ERR_NONFINITE (NaN or infinity in b, w, the image or the dual variable),
 * with a message in ct_last_error().  CT_ERR_CUDA if the synchronisation
 * or the read fails.
 */
ct_status ct_pdtv_status(const void *workspace, void *stream);

/*
 * Many independent slices in one call (the batched form of the solve):
 * slice i is ct_pdtv_solve(geoms[i], b[i], w[i], &params[i], x_out[i],
 * workspaces[i]) with no report, for n slices of any mix of geometries
 * (image sizes, view counts, bins), modes and parameters.
 * geoms, b, w, params, x_out, workspaces (host arrays of n entries) hold
 * per-slice handles, device pointers and parameters; w may be NULL when no
 * slice is low-dose, and w[i] may be NULL for few-view slices.  Every
 * workspace must be ct_pdtv_workspace_bytes(geoms[i], &params[i]) bytes;
 * resume is not accepted here.
 *
 * Two forms, the same result up to the order of float additions:
 *   persistent  when every slice qualifies (default angles with N and V
 *               even, N a multiple of 32 and at most 637, n_bins <= 4096,
 *               precond 0, 1 or 3, eps = 0, tv_iters <= 16, the same
 *               iters > 0 for all slices, the geometries on the current
 *               device) and the form is CT_BATCH_AUTO (ct_batched_options):
 *               each slice's setup (kappa, tau, D, the Lanczos step sizes,
 *               Step 1 at k = 0) runs on the stream pool below, and then ONE
 *               kernel launch on `stream` (one per 96 slices) runs every
 *               iteration of every slice: one block per SM takes work items
 *               (slice, phase, tile) from a queue in iteration order, and
 *               waits for the slice's previous phase with a bounded spin
 *               (ct_batched_options' limit, 5 s by default).  A wait that
 *               runs out stops the launch and marks every slice's checks,
 *               so the reports (or ct_pdtv_status) give CT_ERR_TIMEOUT.
 *   stream pool otherwise: the slices' ordinary solves run concurrently.
 * The slices run on a pool of streams the library creates per device on
 * first use (keep that first call outside stream capture); the work is
 * forked from `stream` and joined back into it, so later work on `stream`
 * sees every x_out, and the whole call can be captured into a CUDA graph.
 * reports (host, n entries, may be NULL) are filled after synchronising
 * `stream` (their trace is not used); the call then returns the first
 * slice's check failure, if any (see ct_pdtv_solve), naming the slice.
 * Calls from several host threads at once share the pool: each call holds
 * the pool's lock while it enqueues, so its slices wait on its own fork and
 * its stream on its own joins, and the calls' slices run one call after the
 * other on the pool.  Do not capture two calls at the same time, and do not
 * run an uncaptured call while another thread captures one (the pool
 * streams would join the capture).
 */
ct_status ct_pdtv_solve_batched(int n, const ct_geometry *const *geoms, const float *const *b,
                                const float *const *w, const ct_pdtv_params *params,
                                float *const *x_out, void *const *workspaces,
                                ct_pdtv_report *reports, void *stream);

/*
 * Options of ct_pdtv_solve_batched for this process (no counterpart in the
 * paper; they choose how the slices are scheduled, never what is
 * computed).  form: CT_BATCH_AUTO (the default) uses the persistent launch
 * when every slice qualifies, CT_BATCH_POOL always the stream pool.
 * wait_seconds: time limit of one wait of the persistent launch for a
 * slice's previous phase (< 0: the default, 5 s; 0: a wait that is not
 * satisfied at once fails, which tests use to see the timeout path).
 * CT_ERR_ARG for an unknown form, NaN or more than 3600 s.
 */
enum { CT_BATCH_AUTO = 0, CT_BATCH_POOL = 1 };
ct_status ct_batched_options(int form, double wait_seconds);

/*
 * The differentiable form: `iters` iterations of Algorithm 1 (mode
 * CT_LOWDOSE, lambda = tau beta) or Algorithm 2 (CT_FEWVIEW, lambda = tau)
 * unrolled for `batch` slices of one geometry that share the taps of D (any
 * real taps, 2*half_len-1 values centred at half_len-1, for example
 * learned ones), tau, sigma and beta.  The steps are those of
 * ct_pdtv_solve (Eqs. 18-20 / 29-31), with the prox of Eq. 17 taken as
 * tv_iters whole-image projected-gradient steps warm-started from the
 * previous iteration's dual field.
 *
 * ct_unrolled_forward writes x_K (batch x N x N) and keeps one checkpoint
 * per iteration (x, mu, mubar, TV dual field, and z = x - tau A^T mubar,
 * the band partial sums of A x_{k+1} and the dual fields after each inner
 * prox step, which it computes anyway) in `workspace`
 * (ct_unrolled_workspace_bytes, device; about 1.6 GB for 16 slices of
 * 256^2, 180 views, 10 iterations, 10 prox steps).
 * ct_unrolled_backward, given grad_x = dL/dx_K (batch x N x N, device) and
 * the workspace of the forward call with the same arguments, applies the
 * adjoint of every step in reverse order (A^T for A, A for A^T, D^T for D,
 * the adjoints of the projected-gradient steps); it writes grad (device, 2*half_len floats): grad[0 .. 2*half_len-2]
 * = dL/dtaps, grad[2*half_len-1] = dL/dbeta (0 for CT_FEWVIEW).  tau and
 * sigma are constants of the unroll.  b, w: batch x V x B; w > 0, required
 * for CT_LOWDOSE.  Needs n_bins <= 4096.  Both calls only enqueue work.
 * ct_unrolled_backward runs the tap correlations on a side stream of the
 * device (created on first use, kept until exit; make the first call
 * outside stream capture), forked from `stream` and joined back into it
 * with events, so later work on `stream` sees grad and the call can be
 * captured into a CUDA graph; concurrent calls from several host threads
 * share that side stream.
 */
size_t ct_unrolled_workspace_bytes(const ct_geometry *geom, int batch, int half_len, int iters, int tv_iters);
ct_status ct_unrolled_forward(const ct_geometry *geom, const float *b, const float *w, int batch,
                              const float *taps, int half_len, double tau, double sigma, double beta,
                              int mode, int iters, int tv_iters, float *x_out, void *workspace, void *stream);
ct_status ct_unrolled_backward(const ct_geometry *geom, const float *b, const float *w, int batch,
                               const float *taps, int half_len, double tau, double sigma, double beta,
                               int mode, int iters, int tv_iters, const float *grad_x, float *grad,
                               void *workspace, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CTPD_H */
