// unrolled.cu -- the differentiable form: K iterations of Algorithm 1 / 2
// unrolled, with per-iteration checkpoints in the forward pass and the
// hand-written adjoint of every step in the backward pass.
//
// Forward, for a batch of slices sharing one geometry, taps t, tau, sigma
// and lambda (= tau beta for Algorithm 1, tau for Algorithm 2):
//   mubar_0 = -sigma D b
//   z_k      = x_k - tau A^T mubar_k
//   x_{k+1}  = prox(z_k), n_tv projected-gradient steps from p_k -> p_{k+1}
//   mu_{k+1}, mubar_{k+1} = dual step (Step 3 and the next Step 1)
// The checkpoint of iteration k is (x_k, mu_k, mubar_k, p_k), plus z_k, the
// band partial sums of A x_{k+1} and the prox's intermediate dual fields,
// which the forward computes anyway: the backward then needs no A^T for z_k,
// no A for the dual step's residual and no second run of the prox.
// Backward, from dL/dx_K, for k = K-1 .. 0: apply the adjoint of the dual
// step (k_dual_bwd_fft), of A (A^T), of the prox (k_tv_*_bwd) and of A^T
// (A), accumulating dL/dt (tap correlations) and dL/dlambda.  sigma and tau
// are constants of the unroll (not differentiated).
#include <algorithm>

#include "ctpd_internal.cuh"

using namespace ctpd;

namespace {

struct UL {
    size_t scal, scal2, hhat, winv, ck, zk, bk, band, gx, gz, gp, gp2, gm, gmb, gmu, gr, gm1, rr, vv, traj, pa,
        tcorr, tacc, orb, psum, total;
    size_t ck_stride;   // floats per checkpoint
};

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

UL layout(const Geometry *g, int S, int half, int iters, int ntv)
{
    UL L;
    const size_t J = (size_t)g->n * g->n, I = (size_t)g->n_views * g->n_bins, F = sizeof(float);
    L.ck_stride = (size_t)S * (4 * J + 2 * I);
    size_t o = 0;
    L.scal = o;  o += a256(sizeof(double) * S_COUNT);
    L.scal2 = o; o += a256(sizeof(double) * S_COUNT);
    L.hhat = o;  o += a256(sizeof(float2) * g->n_fft);
    L.winv = o;  o += a256(F * S * I);
    L.ck = o;    o += a256(F * L.ck_stride * (iters + 1));
    L.zk = o;    o += a256(F * S * J * (size_t)std::max(iters, 1));                       // z_k
    L.bk = o;    o += a256(F * S * I * proj_bands(g->n) * (size_t)std::max(iters, 1));    // A x_{k+1}
    L.band = o;  o += a256(F * S * I * proj_bands(g->n));
    L.gx = o;    o += a256(F * S * J);
    L.gz = o;    o += a256(F * S * J);
    L.gp = o;    o += a256(F * S * 2 * J);
    L.gp2 = o;   o += a256(F * S * 2 * J);
    L.gm = o;    o += a256(F * S * I);
    L.gmb = o;   o += a256(F * S * I);
    L.gmu = o;   o += a256(F * S * I);
    L.gr = o;    o += a256(F * S * I);
    L.gm1 = o;   o += a256(F * S * I);
    L.rr = o;    o += a256(F * S * I);
    L.vv = o;    o += a256(F * S * I);
    // the prox's dual fields after steps 1 .. n_tv - 1 of every iteration
    L.traj = o;  o += a256(F * (size_t)std::max(ntv - 1, 0) * iters * S * 2 * J);
    // block pairs of every prox adjoint launch of the backward pass
    L.pa = o;    o += a256(sizeof(float) * tv_px_blocks(g->n, S) * (size_t)iters * (ntv + 1));
    L.psum = o;  o += a256(sizeof(float) * pair_sums_scratch_floats());
    L.tcorr = o; o += a256(tapcorr_partial_bytes(S * g->n_views, g->n_bins, half));
    L.tacc = o;  o += a256(sizeof(float2) * (2 * (size_t)half - 1));
    L.orb = o;   o += a256(sizeof(float) * (orbit_ok(g) ? orbit_partial_floats(g, S) : 1));
    L.total = o;
    return L;
}

struct CK {
    float *x, *mu, *mubar, *p;
};

CK ck_at(char *ws, const UL &L, const Geometry *g, int S, int k)
{
    const size_t J = (size_t)g->n * g->n, I = (size_t)g->n_views * g->n_bins;
    float *base = (float *)(ws + L.ck) + (size_t)k * L.ck_stride;
    CK c;
    c.x = base;
    c.mu = c.x + S * J;
    c.mubar = c.mu + S * I;
    c.p = c.mubar + S * I;
    return c;
}

// the dual field of iteration k's prox after inner step l (1 <= l < n_tv)
float *traj_at(char *ws, const UL &L, const Geometry *g, int S, int ntv, int k, int l)
{
    const size_t f = (size_t)S * 2 * g->n * g->n;
    return (float *)(ws + L.traj) + ((size_t)k * (ntv - 1) + (l - 1)) * f;
}

enum { U_LAMACC = S_RED0 + 1, U_INV8ACC = S_RED0 + 2 };

ct_status check_args(const Geometry *g, const float *b, const float *w, int batch, const float *taps, int half,
                     double tau, double sigma, double beta, int mode, int iters, int ntv, void *ws)
{
    if (!g || !b || !taps || !ws || batch < 1 || batch > 65535 || half < 1 || half > g->n_bins || !(tau > 0.0) ||
        !(sigma > 0.0) || !(beta >= 0.0) || iters < 0 || ntv < 0 || (mode != CT_LOWDOSE && mode != CT_FEWVIEW) ||
        (mode == CT_LOWDOSE && !w)) {
        set_error("ct_unrolled: bad argument");
        return CT_ERR_ARG;
    }
    if (!fft_supported(g)) {
        set_error("ct_unrolled: n_bins %d is above the frequency-domain filter's limit", g->n_bins);
        return CT_ERR_ARG;
    }
    return CT_OK;
}

void set_scalars(double *scal, double *scal2, double tau, double sigma, double beta, int mode, cudaStream_t st)
{
    const double lam = mode == CT_LOWDOSE ? tau * beta : tau;
    launch_scalars(scal, SC_SET, tau, 0, 0, S_TAU, st);
    launch_scalars(scal, SC_SET, sigma, 0, 0, S_SIGMA, st);
    launch_scalars(scal, SC_SET, lam, 0, 0, S_LAMBDA, st);
    launch_scalars(scal, SC_SET, lam > 0.0 ? 1.0 / (8.0 * lam) : 0.0, 0, 0, S_INV8LAM, st);
    launch_scalars(scal, SC_SET, -tau, 0, 0, S_RED0, st);       // factor of mubar's adjoint
    launch_scalars(scal, SC_SET, 0.0, 0, 0, U_LAMACC, st);
    launch_scalars(scal, SC_SET, 0.0, 0, 0, U_INV8ACC, st);
    launch_scalars(scal2, SC_SET, -1.0, 0, 0, S_TAU, st);       // backprojection that adds
}

// The prox steps of one iteration run as one register-resident launch
// (launch_tv) when there are 1 .. tv_max_steps() of them and lambda > 0
// (otherwise as whole-image single steps); both give the same iterates.
constexpr int TV_UNROLL_ROWS = 48;   // interior rows per tile: the batch fills the GPU
bool tv_fused(double tau, double beta, int mode, int ntv)
{
    const double lam = mode == CT_LOWDOSE ? tau * beta : tau;
    return ntv >= 1 && ntv <= tv_max_steps() && lam > 0.0;
}

void backproject(const Geometry *g, const float *y, float *out, int mode, const float *xin, const double *scal,
                 int S, char *ws, const UL &L, cudaStream_t st)
{
    if (orbit_ok(g)) launch_backproject_orbit(g, y, out, mode, xin, scal, S, (float *)(ws + L.orb), st);
    else launch_backproject(g, y, out, mode, xin, scal, S, st);
}

}  // namespace

extern "C" size_t ct_unrolled_workspace_bytes(const ct_geometry *geom, int batch, int half_len, int iters,
                                              int tv_iters)
{
    if (!geom || batch < 1 || half_len < 1 || iters < 0 || tv_iters < 0) return 0;
    return layout(geom, batch, half_len, iters, tv_iters).total;
}

extern "C" ct_status ct_unrolled_forward(const ct_geometry *geom, const float *b, const float *w, int batch,
                                         const float *taps, int half_len, double tau, double sigma, double beta,
                                         int mode, int iters, int tv_iters, float *x_out, void *workspace,
                                         void *stream)
{
    const Geometry *g = geom;
    set_error("%s", "");
    ct_status cs = check_args(g, b, w, batch, taps, half_len, tau, sigma, beta, mode, iters, tv_iters, workspace);
    if (cs != CT_OK) return cs;
    if (!x_out) {
        set_error("ct_unrolled_forward: x_out is NULL");
        return CT_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int S = batch, N = g->n, lowdose = mode == CT_LOWDOSE;
    const size_t J = (size_t)N * N, I = (size_t)g->n_views * g->n_bins;
    const UL L = layout(g, S, half_len, iters, tv_iters);
    char *ws = static_cast<char *>(workspace);
    double *scal = (double *)(ws + L.scal), *scal2 = (double *)(ws + L.scal2);
    float2 *hhat = (float2 *)(ws + L.hhat);
    float *winv = (float *)(ws + L.winv), *zk = (float *)(ws + L.zk), *bk = (float *)(ws + L.bk);
    const size_t bstride = (size_t)S * I * proj_bands(N);

    cudaMemsetAsync(scal, 0, sizeof(double) * S_COUNT, st);
    cudaMemsetAsync(scal2, 0, sizeof(double) * S_COUNT, st);
    set_scalars(scal, scal2, tau, sigma, beta, mode, st);
    launch_hhat(g, taps, half_len, hhat, st);
    if (lowdose) launch_recip(w, winv, S * I, st);
    CK c0 = ck_at(ws, L, g, S, 0);
    cudaMemsetAsync(c0.x, 0, sizeof(float) * S * J, st);
    cudaMemsetAsync(c0.mu, 0, sizeof(float) * S * I, st);
    cudaMemsetAsync(c0.p, 0, sizeof(float) * S * 2 * J, st);
    launch_filter_fft(g, hhat, b, c0.mubar, nullptr, nullptr, 1, scal, S, st);      // mubar_0 = -sigma D b
    const bool fused = tv_fused(tau, beta, mode, tv_iters);
    for (int k = 0; k < iters; ++k) {
        CK c = ck_at(ws, L, g, S, k), n = ck_at(ws, L, g, S, k + 1);
        float *z = zk + (size_t)k * S * J, *band = bk + (size_t)k * bstride;
        backproject(g, c.mubar, z, 1, c.x, scal, S, ws, L, st);                       // z = x - tau A^T mubar
        if (fused) {
            // the prox, writing its intermediate dual fields for the backward pass
            launch_tv(z, c.p, n.p, n.x, N, g->n_sm, TV_UNROLL_ROWS, tv_iters, 1, scal, st, false, S,
                      tv_iters > 1 ? traj_at(ws, L, g, S, tv_iters, k, 1) : nullptr);
            launch_project_bands(g, n.x, band, S, st);
            launch_dual_fft_batched(g, hhat, band, b, c.mu, n.mu, n.mubar, winv, lowdose, scal, S, st);
            continue;
        }
        if (tv_iters == 0) {
            cudaMemcpyAsync(n.p, c.p, sizeof(float) * S * 2 * J, cudaMemcpyDeviceToDevice, st);
        } else {
            const float *src = c.p;
            for (int l = 0; l < tv_iters; ++l) {
                float *dst = (l == tv_iters - 1) ? n.p : traj_at(ws, L, g, S, tv_iters, k, l + 1);
                launch_tv_step(z, src, dst, N, S, scal, st);
                src = dst;
            }
        }
        launch_tv_final(z, n.p, n.x, N, S, scal, st);                               // x_{k+1}
        launch_project_bands(g, n.x, band, S, st);
        launch_dual_fft_batched(g, hhat, band, b, c.mu, n.mu, n.mubar, winv, lowdose, scal, S, st);
    }
    cudaMemcpyAsync(x_out, ck_at(ws, L, g, S, iters).x, sizeof(float) * S * J, cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("ct_unrolled_forward: %s", cudaGetErrorString(e));
        return CT_ERR_CUDA;
    }
    return CT_OK;
}

extern "C" ct_status ct_unrolled_backward(const ct_geometry *geom, const float *b, const float *w, int batch,
                                          const float *taps, int half_len, double tau, double sigma, double beta,
                                          int mode, int iters, int tv_iters, const float *grad_x, float *grad,
                                          void *workspace, void *stream)
{
    const Geometry *g = geom;
    set_error("%s", "");
    ct_status cs = check_args(g, b, w, batch, taps, half_len, tau, sigma, beta, mode, iters, tv_iters, workspace);
    if (cs != CT_OK) return cs;
    if (!grad_x || !grad) {
        set_error("ct_unrolled_backward: NULL gradient pointer");
        return CT_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int S = batch, N = g->n, V = g->n_views, lowdose = mode == CT_LOWDOSE;
    const size_t J = (size_t)N * N, I = (size_t)V * g->n_bins;
    const UL L = layout(g, S, half_len, iters, tv_iters);
    char *ws = static_cast<char *>(workspace);
    double *scal = (double *)(ws + L.scal), *scal2 = (double *)(ws + L.scal2);
    const float2 *hhat = (const float2 *)(ws + L.hhat);
    const float *winv = (const float *)(ws + L.winv);
    const float *zk = (const float *)(ws + L.zk), *bk = (const float *)(ws + L.bk);
    float *band = (float *)(ws + L.band);
    const size_t bstride = (size_t)S * I * proj_bands(N);
    float *gx = (float *)(ws + L.gx), *gz = (float *)(ws + L.gz);
    float *gp = (float *)(ws + L.gp), *gp2 = (float *)(ws + L.gp2);
    float *gm = (float *)(ws + L.gm), *gmb = (float *)(ws + L.gmb), *gmu = (float *)(ws + L.gmu);
    float *gr = (float *)(ws + L.gr), *gm1 = (float *)(ws + L.gm1), *rr = (float *)(ws + L.rr),
          *vv = (float *)(ws + L.vv);
    float *pa = (float *)(ws + L.pa), *psum = (float *)(ws + L.psum);
    const size_t npx = tv_px_blocks(N, S), ncall = (size_t)iters * (tv_iters + 1);
    float *tcorr = (float *)(ws + L.tcorr);
    float2 *tacc = (float2 *)(ws + L.tacc);
    const int nl = 2 * half_len - 1;
    const double lam = lowdose ? tau * beta : tau;

    // the scalars of the forward pass are still in the workspace; reset the accumulators
    set_scalars(scal, scal2, tau, sigma, beta, mode, st);
    cudaMemsetAsync(gm, 0, sizeof(float) * S * I, st);
    cudaMemsetAsync(gmb, 0, sizeof(float) * S * I, st);
    cudaMemsetAsync(gp, 0, sizeof(float) * S * 2 * J, st);
    cudaMemsetAsync(tacc, 0, sizeof(float2) * nl, st);
    cudaMemsetAsync(pa, 0, sizeof(float) * npx * ncall, st);
    float *part = pa;   // the next launch's block pairs
    // the tap correlations of a step read only its dual adjoints, so they
    // run on the device's side stream beside the adjoints of A^T and the prox
    int dev = -1;
    Fork *fk = cudaGetDevice(&dev) == cudaSuccess ? fork_for(dev) : nullptr;
    cudaMemcpyAsync(gx, grad_x, sizeof(float) * S * J, cudaMemcpyDeviceToDevice, st);
    for (int k = iters - 1; k >= 0; --k) {
        CK c = ck_at(ws, L, g, S, k), n = ck_at(ws, L, g, S, k + 1);
        const float *z = zk + (size_t)k * S * J;
        // the prox trajectory p_k = tp(0) .. tp(n_tv) = p_{k+1}, kept by the forward pass
        auto tp = [&](int l) -> const float * {
            return l == 0 ? c.p : (l == tv_iters ? n.p : traj_at(ws, L, g, S, tv_iters, k, l));
        };
        // adjoint of the dual step (A x_{k+1} from the checkpoint's band sums)
        launch_dual_bwd_fft(g, hhat, bk + (size_t)k * bstride, b, winv, c.mu, n.mu, gm, gmb, gmu, gr, gm1, rr, vv,
                            lowdose, scal, S, st);
        launch_tapcorr_acc(gm1, rr, sigma, lowdose ? gmb : nullptr, vv, -sigma, S * V, g->n_bins, half_len, tcorr,
                           tacc, fk ? fork_begin(fk, st) : st);
        // dL/dx_{k+1} += A^T dL/dr  (into gz, then swapped)
        backproject(g, gr, gz, 1, gx, scal2, S, ws, L, st);
        std::swap(gx, gz);
        // adjoint of the prox: final step, then the n_tv steps in reverse
        const float *trn = tp(tv_iters);
        launch_tv_final_bwd(z, trn, gx, gp, gz, gp2, N, S, scal, part, st);
        part += npx;
        for (int l = tv_iters - 1; l >= 0; --l) {
            launch_tv_step_bwd(z, tp(l), gp2, gz, gp, N, S, scal, part, st);
            part += npx;
            std::swap(gp, gp2);
        }
        std::swap(gp, gp2);   // gp: dL/dp_k
        // x_k enters through z_k only: dL/dx_k = dL/dz_k; dL/dmubar_k = -tau A dL/dz_k
        std::swap(gx, gz);
        launch_project_bands(g, gx, band, S, st);
        if (fk) fork_end(fk, st);   // the correlations are done with gmb, gm1, rr and vv
        launch_band_reduce_scaled(g, band, gmb, scal + S_RED0, S, st);
        std::swap(gm, gmu);   // dL/dmu_k
    }
    // mubar_0 = -sigma D b
    launch_tapcorr_acc(gmb, b, -sigma, nullptr, nullptr, 0.0, S * V, g->n_bins, half_len, tcorr, tacc, st);
    launch_pair_sums(pa, npx * ncall / 2, psum, scal, U_INV8ACC, U_LAMACC, st);
    // dL/dbeta = dL/dlambda dlambda/dbeta, dL/dlambda = lamacc + inv8acc d(1/(8 lam))/dlam
    if (lam > 0.0) launch_scalars(scal, SC_AXPY_SLOT, -1.0 / (8.0 * lam * lam), (double)U_INV8ACC, 0, U_LAMACC, st);
    launch_grad_out(tacc, nl, scal, U_LAMACC, lowdose ? tau : 0.0, grad, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("ct_unrolled_backward: %s", cudaGetErrorString(e));
        return CT_ERR_CUDA;
    }
    return CT_OK;
}
