/*
 * ct_oracle.c -- plain, slow, FP64 CPU reference of the ramp-preconditioned
 * primal-dual TV reconstruction of Kudo, Yamazaki, Nemoto and Takaki,
 * "A very fast iterative algorithm for TV-regularized image reconstruction
 * with applications to low-dose and few-view CT" (arXiv 1609.06041).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls
 * this file; the tests, the smoke check and the benchmark's CPU-baseline leg
 * load it through oracle/__init__.py to check and time the CUDA path.  It
 * shares no code, header or table with the CUDA sources.
 *
 * Every routine is written in the most direct form, with no blocking,
 * fusion or reordering beyond what the definition states.  Built with
 * OpenMP, the projector and the filter run their independent rays / views
 * on several threads and the backprojector gives each thread a band of
 * image rows; every output element is still formed by the same operations
 * in the same order as with one thread, so results do not depend on the
 * thread count (orc_set_threads).
 *
 * Conventions (the paper leaves the discretisation open; these are the
 * readings this project fixes):
 *   image  x[r*N + c], pixel centre (c - (N-1)/2, r - (N-1)/2), unit pixels;
 *   sinogram s[v*B + d], ray {(x,y): x cos t_v + y sin t_v = d - (B-1)/2};
 *   default angles t_v = v*pi/V; a view steps along rows when
 *   4v <= V or 4v >= 3V (custom angles: |cos t| >= |sin t|).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the projector, backprojector and filter (<= 0: all). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Geometry of one view                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    double c, s;   /* cos t, sin t */
    int rows;      /* 1: step along image rows, 0: along columns */
} view_t;

static view_t view_of(int v, int V, const double *angles)
{
    view_t w;
    double t;
    if (angles) {
        t = angles[v];
        w.c = cos(t);
        w.s = sin(t);
        w.rows = fabs(w.c) >= fabs(w.s);
    } else {
        t = (double)v * M_PI / (double)V;
        w.c = cos(t);
        w.s = sin(t);
        w.rows = (4 * v <= V) || (4 * v >= 3 * V);
    }
    return w;
}

static double pix(const double *x, int N, int r, int c)
{
    if (r < 0 || r >= N || c < 0 || c >= N) return 0.0;
    return x[(size_t)r * N + c];
}

/* ------------------------------------------------------------------ */
/* Forward projection A (Joseph): the system matrix of Eq. 1 for the   */
/* parallel-beam geometry of Sec. 2.1.                                 */
/* For a row-stepping view, each image row r contributes the linear    */
/* interpolation of that row at the column where the ray crosses the   */
/* row centre line, times the path length 1/|cos t| per row; columns   */
/* play the same part for column-stepping views.                       */
/* ------------------------------------------------------------------ */

void orc_project(int N, int V, int B, const double *angles,
                 const double *x, double *sino)
{
    const double h = 0.5 * (N - 1), hb = 0.5 * (B - 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < V; ++v) {
        view_t g = view_of(v, V, angles);
        for (int d = 0; d < B; ++d) {
            double s = d - hb, acc = 0.0;
            if (g.rows) {
                for (int r = 0; r < N; ++r) {
                    double y = r - h;
                    double u = (s - y * g.s) / g.c + h;   /* column coordinate */
                    double fl = floor(u), f = u - fl;
                    int i0 = (int)fl;
                    acc += (1.0 - f) * pix(x, N, r, i0) + f * pix(x, N, r, i0 + 1);
                }
                sino[(size_t)v * B + d] = acc / fabs(g.c);
            } else {
                for (int c = 0; c < N; ++c) {
                    double xc = c - h;
                    double u = (s - xc * g.c) / g.s + h;  /* row coordinate */
                    double fl = floor(u), f = u - fl;
                    int i0 = (int)fl;
                    acc += (1.0 - f) * pix(x, N, i0, c) + f * pix(x, N, i0 + 1, c);
                }
                sino[(size_t)v * B + d] = acc / fabs(g.s);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Backprojection A^T, written as the explicit scatter of each ray's   */
/* value into the pixels A reads, with the same weights (Eq. 19 uses   */
/* A^T).                                                               */
/* ------------------------------------------------------------------ */

/* adds val to pixel (r, c) if it lies in the image and in rows [r0, r1) */
static void add_pix(double *x, int N, int r, int c, double val, int r0, int r1)
{
    if (r < r0 || r >= r1 || c < 0 || c >= N) return;
    x[(size_t)r * N + c] += val;
}

/* Each thread owns the image rows [r0, r1) and visits the rays in the
 * serial order (view, then ray d, then step), so every pixel receives its
 * contributions in the same order as with one thread.  A row-stepping view
 * touches row r only at step r; a column-stepping view reaches rows near
 * u(d) = (s_d - x_c cos t) / sin t + h, which is linear in d, so at column c
 * only a short range of rays needs visiting (taken with a margin; the
 * per-ray arithmetic is unchanged and the row test decides). */
void orc_backproject(int N, int V, int B, const double *angles,
                     const double *sino, double *x)
{
    const double h = 0.5 * (N - 1), hb = 0.5 * (B - 1);
    memset(x, 0, sizeof(double) * (size_t)N * N);
#pragma omp parallel
    {
        int T = 1, t = 0;
#ifdef _OPENMP
        T = omp_get_num_threads();
        t = omp_get_thread_num();
#endif
        const int r0 = (int)((long long)N * t / T), r1 = (int)((long long)N * (t + 1) / T);
        for (int v = 0; v < V && r0 < r1; ++v) {
            view_t g = view_of(v, V, angles);
            if (g.rows) {
                for (int d = 0; d < B; ++d) {
                    double s = d - hb;
                    double val = sino[(size_t)v * B + d] / fabs(g.c);
                    for (int r = r0; r < r1; ++r) {
                        double y = r - h;
                        double u = (s - y * g.s) / g.c + h;
                        double fl = floor(u), f = u - fl;
                        int i0 = (int)fl;
                        add_pix(x, N, r, i0, (1.0 - f) * val, r0, r1);
                        add_pix(x, N, r, i0 + 1, f * val, r0, r1);
                    }
                }
            } else {
                for (int c = 0; c < N; ++c) {
                    double xc = c - h;
                    /* rays whose row coordinate u lies in [r0 - 2, r1 + 1] */
                    double da = (r0 - 2 - h) * g.s + hb + xc * g.c;
                    double db = (r1 + 1 - h) * g.s + hb + xc * g.c;
                    double dlo = floor(da < db ? da : db) - 1.0, dhi = ceil(da < db ? db : da) + 1.0;
                    int d0 = dlo < 0.0 ? 0 : (dlo > B ? B : (int)dlo);
                    int d1 = dhi < 0.0 ? -1 : (dhi > B - 1 ? B - 1 : (int)dhi);
                    for (int d = d0; d <= d1; ++d) {
                        double s = d - hb;
                        double val = sino[(size_t)v * B + d] / fabs(g.s);
                        double u = (s - xc * g.c) / g.s + h;
                        double fl = floor(u), f = u - fl;
                        int i0 = (int)fl;
                        add_pix(x, N, i0, c, (1.0 - f) * val, r0, r1);
                        add_pix(x, N, i0 + 1, c, f * val, r0, r1);
                    }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Preconditioner D = F^-1 H F along the detector axis of each view    */
/* (Eq. 24 for low-dose, Eq. 32 for few-view).                         */
/* Discretisation: period P = 2^ceil(log2(2B)), frequencies            */
/* w_j = 2 pi min(j, P-j)/P rad per bin, m = number of views over      */
/* 180 degrees.  The filter is the linear (zero-padded) convolution    */
/* with the taps t[k] = (1/P) sum_j H(w_j) cos(2 pi j k / P).          */
/* ------------------------------------------------------------------ */

int orc_fft_len(int B)
{
    int P = 1;
    while (P < 2 * B) P <<= 1;
    return P;
}

/* H(w): mode 0 smoothed ramp |w|/(2 m tau + kappa |w|) (Eq. 24);
 *       mode 1 pure ramp |w|/(2 m tau) (Eq. 32);
 *       modes 2 and 3 split the smoothed ramp into a low band and a high
 *       band, H_lo + H_hi = H (mode 0), for the shift-variant preconditioner
 *       (Sec. 5 names one approximating D = (tau A A^T + W^-1)^-1 of Eq. 23
 *       better; its form is this project's):
 *         H_lo = 2 m tau |w| / (2 m tau + kappa |w|)^2,
 *         H_hi = kappa w^2 / (2 m tau + kappa |w|)^2. */
static double H_of(int mode, double w, int m, double tau, double kappa)
{
    double aw = fabs(w), den = 2.0 * m * tau + kappa * aw;
    if (mode == 0) return aw / den;
    if (mode == 1) return aw / (2.0 * m * tau);
    if (mode == 2) return 2.0 * m * tau * aw / (den * den);
    return kappa * aw * aw / (den * den);
}

/* taps[k + half - 1] = t[k] for |k| <= half - 1, by the direct cosine sum. */
void orc_ramp_taps(int mode, int m, int P, double tau, double kappa,
                   int half, double *taps)
{
    for (int k = 0; k < half; ++k) {
        double acc = 0.0;
        for (int j = 0; j < P; ++j) {
            int jj = j < P - j ? j : P - j;
            double w = 2.0 * M_PI * jj / (double)P;
            acc += H_of(mode, w, m, tau, kappa) * cos(2.0 * M_PI * (double)j * k / (double)P);
        }
        taps[half - 1 + k] = acc / P;
        taps[half - 1 - k] = acc / P;
    }
}

/* out[v][d] = sum_{d'} t[d - d'] in[v][d'], taps of half length `half`
 * (2*half-1 values, centre at index half-1); zero outside the detector. */
void orc_filter(int V, int B, const double *taps, int half,
                const double *in, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < V; ++v) {
        const double *a = in + (size_t)v * B;
        double *o = out + (size_t)v * B;
        for (int d = 0; d < B; ++d) {
            double acc = 0.0;
            for (int e = 0; e < B; ++e) {
                int k = d - e;
                if (k <= -half || k >= half) continue;
                acc += taps[half - 1 + k] * a[e];
            }
            o[d] = acc;
        }
    }
}

/* The preconditioner applied in the iteration.  taps_hi == NULL: the
 * convolution D of Eqs. 24 / 32 with `taps`.  Otherwise the shift-variant
 * form D = T_lo + S T_hi S: `taps` holds the low band (H_lo), taps_hi the
 * high band (H_hi), and S = diag(s), s_i = sqrt(kappa w_i), scales the high
 * band so that, as the frequency grows, D tends to W = diag(w), the high-
 * frequency limit of (tau A A^T + W^-1)^-1 (Eq. 23), where Eq. 24 tends to
 * I/kappa.  With s = 1 (w_i = 1/kappa) it is the convolution of Eq. 24.
 * tmp: two scratch sinograms. */
static void apply_d(int V, int B, const double *taps, const double *taps_hi, int half,
                    const double *s, const double *in, double *out, double *tmp)
{
    orc_filter(V, B, taps, half, in, out);
    if (!taps_hi) return;
    size_t I = (size_t)V * B;
    double *t1 = tmp, *t2 = tmp + I;
    for (size_t i = 0; i < I; ++i) t1[i] = s[i] * in[i];
    orc_filter(V, B, taps_hi, half, t1, t2);
    for (size_t i = 0; i < I; ++i) out[i] += s[i] * t2[i];
}

void orc_apply_d(int V, int B, const double *taps, const double *taps_hi, int half,
                 const double *s, const double *in, double *out)
{
    double *tmp = malloc(sizeof(double) * 2 * (size_t)V * B);
    apply_d(V, B, taps, taps_hi, half, s, in, out, tmp);
    free(tmp);
}

/* ------------------------------------------------------------------ */
/* TV (Eq. 2) with forward differences, zero across the last column   */
/* and row: h_j^T x = x[r][c+1]-x[r][c], v_j^T x = x[r+1][c]-x[r][c].  */
/* div is defined as minus the adjoint of the gradient.                */
/* ------------------------------------------------------------------ */

void orc_grad(int N, const double *x, double *gx, double *gy)
{
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            size_t j = (size_t)r * N + c;
            gx[j] = (c < N - 1) ? x[j + 1] - x[j] : 0.0;
            gy[j] = (r < N - 1) ? x[j + N] - x[j] : 0.0;
        }
}

void orc_div(int N, const double *px, const double *py, double *out)
{
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            size_t j = (size_t)r * N + c;
            double dx = (c < N - 1 ? px[j] : 0.0) - (c > 0 ? px[j - 1] : 0.0);
            double dy = (r < N - 1 ? py[j] : 0.0) - (r > 0 ? py[j - N] : 0.0);
            out[j] = dx + dy;
        }
}

double orc_tv(int N, const double *x)
{
    size_t J = (size_t)N * N;
    double *gx = malloc(sizeof(double) * J), *gy = malloc(sizeof(double) * J);
    orc_grad(N, x, gx, gy);
    double acc = 0.0;
    for (size_t j = 0; j < J; ++j) acc += sqrt(gx[j] * gx[j] + gy[j] * gy[j]);
    free(gx);
    free(gy);
    return acc;
}

/* ------------------------------------------------------------------ */
/* prox of lam*TV + indicator(x >= 0) (Eq. 17): the dual projection    */
/* approach for TV denoising with the bound constraint, gradient-      */
/* projection form with step 1/(8 lam):                                */
/*   x_l = max(0, z + lam div p),  p <- Pi_{|p_j|<=1}(p + grad x_l/(8 lam)) */
/* repeated n_tv times from the given (warm-start) p, then             */
/*   x = max(0, z + lam div p).  lam = 0 gives x = max(0, z).         */
/* ------------------------------------------------------------------ */

void orc_tv_prox(int N, const double *z, double lam, int n_tv,
                 double *px, double *py, double *x)
{
    size_t J = (size_t)N * N;
    if (lam <= 0.0) {
        for (size_t j = 0; j < J; ++j) x[j] = z[j] > 0.0 ? z[j] : 0.0;
        return;
    }
    double *dv = malloc(sizeof(double) * J);
    double *gx = malloc(sizeof(double) * J), *gy = malloc(sizeof(double) * J);
    for (int it = 0; it < n_tv; ++it) {
        orc_div(N, px, py, dv);
        for (size_t j = 0; j < J; ++j) {
            double t = z[j] + lam * dv[j];
            x[j] = t > 0.0 ? t : 0.0;
        }
        orc_grad(N, x, gx, gy);
        for (size_t j = 0; j < J; ++j) {
            double qx = px[j] + gx[j] / (8.0 * lam);
            double qy = py[j] + gy[j] / (8.0 * lam);
            double nrm = sqrt(qx * qx + qy * qy);
            double s = nrm > 1.0 ? nrm : 1.0;
            px[j] = qx / s;
            py[j] = qy / s;
        }
    }
    orc_div(N, px, py, dv);
    for (size_t j = 0; j < J; ++j) {
        double t = z[j] + lam * dv[j];
        x[j] = t > 0.0 ? t : 0.0;
    }
    free(dv);
    free(gx);
    free(gy);
}

/* The same prox by the fast gradient projection (FGP) of Beck and      */
/* Teboulle (2009) on the dual field: the projected-gradient step above */
/* taken at an extrapolated point r, with the momentum of Nesterov:     */
/*   r_1 = p_0, t_1 = 1;  for k = 1..n_tv:                              */
/*     p_k = Pi(r_k + grad max(0, z + lam div r_k) / (8 lam)),          */
/*     t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,                           */
/*     r_{k+1} = p_k + ((t_k - 1) / t_{k+1}) (p_k - p_{k-1});           */
/*   x = max(0, z + lam div p_n).                                       */
/* p_0 (px, py on entry) warm-starts it; px, py receive p_n.            */
void orc_tv_prox_fgp(int N, const double *z, double lam, int n_tv,
                     double *px, double *py, double *x)
{
    size_t J = (size_t)N * N;
    if (lam <= 0.0) {
        for (size_t j = 0; j < J; ++j) x[j] = z[j] > 0.0 ? z[j] : 0.0;
        return;
    }
    double *dv = malloc(sizeof(double) * J);
    double *gx = malloc(sizeof(double) * J), *gy = malloc(sizeof(double) * J);
    double *rx = malloc(sizeof(double) * J), *ry = malloc(sizeof(double) * J);
    memcpy(rx, px, sizeof(double) * J);
    memcpy(ry, py, sizeof(double) * J);
    double t = 1.0;
    for (int it = 0; it < n_tv; ++it) {
        orc_div(N, rx, ry, dv);
        for (size_t j = 0; j < J; ++j) {
            double v = z[j] + lam * dv[j];
            x[j] = v > 0.0 ? v : 0.0;
        }
        orc_grad(N, x, gx, gy);
        double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double th = (t - 1.0) / t1;
        for (size_t j = 0; j < J; ++j) {
            double qx = rx[j] + gx[j] / (8.0 * lam);
            double qy = ry[j] + gy[j] / (8.0 * lam);
            double nrm = sqrt(qx * qx + qy * qy);
            double s = nrm > 1.0 ? nrm : 1.0;
            double nx = qx / s, ny = qy / s;      /* p_k */
            rx[j] = nx + th * (nx - px[j]);       /* r_{k+1}, px = p_{k-1} */
            ry[j] = ny + th * (ny - py[j]);
            px[j] = nx;
            py[j] = ny;
        }
        t = t1;
    }
    orc_div(N, px, py, dv);
    for (size_t j = 0; j < J; ++j) {
        double v = z[j] + lam * dv[j];
        x[j] = v > 0.0 ? v : 0.0;
    }
    free(dv);
    free(gx);
    free(gy);
    free(rx);
    free(ry);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (low-dose, Eqs. 18-20), Algorithm 1' (beta = 0) and     */
/* Algorithm 2 (few-view, Eqs. 29-31), in the order of their boxes:    */
/*   Step 1  k = 0: mu_bar = -sigma D b;                               */
/*           k > 0: mu_bar = 2 mu^k - mu^{k-1}                         */
/*                           [- sigma D W^-1 (mu^k - mu^{k-1}), Alg. 1]*/
/*   Step 2  x^{k+1} = prox_{tau g}(x^k - tau A^T mu_bar)              */
/*           (lam = tau*beta for Alg. 1, tau for Alg. 2)               */
/*   Step 3  mu^{k+1} = mu^k + sigma D (A x^{k+1} - b [- W^-1 mu^k])   */
/* mode 0 = Algorithm 1/1', mode 1 = Algorithm 2.  D is the Toeplitz   */
/* filter with the given taps (taps = {1}, half = 1 gives D = I, the   */
/* unpreconditioned iteration).  Iterations k0 .. k0+iters-1 run from  */
/* the state (x, mu, mu_prev, px, py); k0 = 0 starts from x = mu = p = 0. */
/* fgp: the prox by orc_tv_prox_fgp instead of orc_tv_prox.            */
/* trace[i] (optional) receives f(x) (Eq. 1) for mode 0 or ||Ax-b||    */
/* for mode 1 after iteration i.  mubar_out (optional, V*B) receives   */
/* the mu_bar that Step 1 of the last iteration formed.                */
/* ------------------------------------------------------------------ */

double orc_cost(int N, int V, int B, const double *angles, const double *b,
                const double *w, double beta, const double *x)
{
    size_t I = (size_t)V * B;
    double *ax = malloc(sizeof(double) * I);
    orc_project(N, V, B, angles, x, ax);
    double fid = 0.0;
    for (size_t i = 0; i < I; ++i) {
        double e = ax[i] - b[i];
        fid += (w ? w[i] : 1.0) * e * e;
    }
    free(ax);
    return beta * orc_tv(N, x) + 0.5 * fid;
}

double orc_residual(int N, int V, int B, const double *angles,
                    const double *b, const double *x)
{
    size_t I = (size_t)V * B;
    double *ax = malloc(sizeof(double) * I);
    orc_project(N, V, B, angles, x, ax);
    double acc = 0.0;
    for (size_t i = 0; i < I; ++i) acc += (ax[i] - b[i]) * (ax[i] - b[i]);
    free(ax);
    return sqrt(acc);
}

/* ------------------------------------------------------------------ */
/* The dual step of the epsilon-constrained few-view form               */
/*   min TV(x)  s.t.  ||Ax - b|| <= eps,  x >= 0    (Sec. 5)             */
/* (Sec. 5 names the form without its steps; here the indicator of the */
/* eps-ball replaces the equality constraint): with the ball's support  */
/* function in h, the dual step                                         */
/* in the metric of sigma D is the proximal map                         */
/*   nu = argmin_nu  se |nu| + 1/2 (nu - q)^T D^-1 (nu - q),  se = s eps, */
/* where q is the equality form's update mu + sigma D (A x - b) and D   */
/* is block diagonal over views with the B x B Toeplitz matrix T of the */
/* taps.  Optimality: (I + c T) nu = q with c = se / |nu|, or nu = 0    */
/* when |T^-1 q| <= se.  c |nu(c)| grows with c, so c is found by       */
/* bisection, each trial one dense Cholesky solve of I + c T for all    */
/* views (norms over the whole sinogram).                               */
/* ------------------------------------------------------------------ */

/* lower Cholesky factor of the n x n SPD matrix a (row-major, in place);
 * returns 0 if a pivot is not positive */
static int chol(double *a, int n)
{
    for (int j = 0; j < n; ++j) {
        double d = a[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
        if (!(d > 0.0)) return 0;
        d = sqrt(d);
        a[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = a[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
            a[(size_t)i * n + j] = v / d;
        }
    }
    return 1;
}

/* x = (L L^T)^-1 r */
static void chol_solve(const double *l, int n, const double *r, double *x)
{
    for (int i = 0; i < n; ++i) {
        double v = r[i];
        for (int k = 0; k < i; ++k) v -= l[(size_t)i * n + k] * x[k];
        x[i] = v / l[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double v = x[i];
        for (int k = i + 1; k < n; ++k) v -= l[(size_t)k * n + i] * x[k];
        x[i] = v / l[(size_t)i * n + i];
    }
}

/* out = (I + c T)^-1 q for every view (c < 0: T^-1 q); returns |out| over
 * the whole sinogram, or -1 if the matrix is not positive definite */
static double eps_solve(int V, int B, const double *taps, int half, double c, const double *q, double *out,
                        double *m)
{
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
            int k = i - j;
            double t = (k > -half && k < half) ? taps[half - 1 + k] : 0.0;
            m[(size_t)i * B + j] = c < 0.0 ? t : (i == j ? 1.0 : 0.0) + c * t;
        }
    if (!chol(m, B)) return -1.0;
    double n2 = 0.0;
    for (int v = 0; v < V; ++v) {
        chol_solve(m, B, q + (size_t)v * B, out + (size_t)v * B);
        for (int d = 0; d < B; ++d) n2 += out[(size_t)v * B + d] * out[(size_t)v * B + d];
    }
    return sqrt(n2);
}

void orc_eps_prox(int V, int B, const double *taps, int half, double se, const double *q, double *nu)
{
    size_t I = (size_t)V * B;
    if (!(se > 0.0)) {
        memcpy(nu, q, sizeof(double) * I);
        return;
    }
    double *m = malloc(sizeof(double) * (size_t)B * B);
    double qn = 0.0;
    for (size_t i = 0; i < I; ++i) qn += q[i] * q[i];
    qn = sqrt(qn);
    /* nu = 0 when |T^-1 q| <= se (T singular: the bound is infinite) */
    double tn = eps_solve(V, B, taps, half, -1.0, q, nu, m);
    if (qn == 0.0 || (tn >= 0.0 && tn <= se)) {
        memset(nu, 0, sizeof(double) * I);
        free(m);
        return;
    }
    /* |nu(c)| <= |q|, so c |nu(c)| <= se at c = se / |q| */
    double lo = se / qn, hi = 2.0 * lo;
    for (int it = 0; it < 400 && hi * eps_solve(V, B, taps, half, hi, q, nu, m) < se; ++it) {
        lo = hi;
        hi *= 2.0;
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        double c = 0.5 * (lo + hi);
        if (c * eps_solve(V, B, taps, half, c, q, nu, m) < se) lo = c;
        else hi = c;
    }
    eps_solve(V, B, taps, half, 0.5 * (lo + hi), q, nu, m);
    free(m);
}

void orc_pdtv(int N, int V, int B, const double *angles,
              const double *b, const double *w,
              const double *taps, const double *taps_hi, const double *sv, int half, int mode,
              double beta, double tau, double sigma, int n_tv, int fgp, double eps,
              int k0, int iters,
              double *x, double *mu, double *mu_prev, double *px, double *py,
              double *trace, double *mubar_out)
{
    /* eps > 0 (mode 1, taps_hi NULL): the epsilon-constrained form; Step 3
     * and Step 1 at k = 0 take the proximal map of orc_eps_prox */
    int epsf = mode == 1 && eps > 0.0;
    size_t I = (size_t)V * B, J = (size_t)N * N;
    double *mubar = malloc(sizeof(double) * I);
    double *t1 = malloc(sizeof(double) * I), *t2 = malloc(sizeof(double) * I);
    double *z = malloc(sizeof(double) * J);
    double *dtmp = malloc(sizeof(double) * 2 * I);
    double lam = (mode == 0) ? tau * beta : tau;
    if (k0 == 0) {
        memset(x, 0, sizeof(double) * J);
        memset(mu, 0, sizeof(double) * I);
        memset(mu_prev, 0, sizeof(double) * I);
        memset(px, 0, sizeof(double) * J);
        memset(py, 0, sizeof(double) * J);
    }
    for (int k = k0; k < k0 + iters; ++k) {
        /* Step 1: extrapolation */
        if (k == 0) {
            apply_d(V, B, taps, taps_hi, half, sv, b, t1, dtmp);
            for (size_t i = 0; i < I; ++i) mubar[i] = -sigma * t1[i];
            if (epsf) {
                memcpy(t2, mubar, sizeof(double) * I);
                orc_eps_prox(V, B, taps, half, sigma * eps, t2, mubar);
            }
        } else if (mode == 0) {
            for (size_t i = 0; i < I; ++i) t2[i] = (mu[i] - mu_prev[i]) / w[i];
            apply_d(V, B, taps, taps_hi, half, sv, t2, t1, dtmp);
            for (size_t i = 0; i < I; ++i)
                mubar[i] = 2.0 * mu[i] - mu_prev[i] - sigma * t1[i];
        } else {
            for (size_t i = 0; i < I; ++i) mubar[i] = 2.0 * mu[i] - mu_prev[i];
        }
        if (mubar_out && k == k0 + iters - 1) memcpy(mubar_out, mubar, sizeof(double) * I);
        /* Step 2: primal update through the prox of tau*g */
        orc_backproject(N, V, B, angles, mubar, z);
        for (size_t j = 0; j < J; ++j) z[j] = x[j] - tau * z[j];
        if (fgp) orc_tv_prox_fgp(N, z, lam, n_tv, px, py, x);
        else orc_tv_prox(N, z, lam, n_tv, px, py, x);
        /* Step 3: dual update */
        orc_project(N, V, B, angles, x, t2);
        for (size_t i = 0; i < I; ++i) {
            t2[i] -= b[i];
            if (mode == 0) t2[i] -= mu[i] / w[i];
        }
        apply_d(V, B, taps, taps_hi, half, sv, t2, t1, dtmp);
        for (size_t i = 0; i < I; ++i) {
            mu_prev[i] = mu[i];
            mu[i] = mu[i] + sigma * t1[i];
        }
        if (epsf) {
            memcpy(t2, mu, sizeof(double) * I);
            orc_eps_prox(V, B, taps, half, sigma * eps, t2, mu);
        }
        if (trace) {
            trace[k - k0] = (mode == 0)
                ? orc_cost(N, V, B, angles, b, w, beta, x)
                : orc_residual(N, V, B, angles, b, x);
        }
    }
    free(mubar);
    free(t1);
    free(t2);
    free(z);
    free(dtmp);
}

/* ------------------------------------------------------------------ */
/* Step-size setup (Alg. 1, Alg. 2 boxes): operator norms by the power */
/* method.  which = 0: ||A^T D A|| (equal to ||D^1/2 A A^T D^T/2||);   */
/* which = 1: ||W^-1/2 D W^-1/2|| (equal to ||D^1/2 W^-1 D^T/2||).      */
/* Starts from the all-ones vector; returns the last Rayleigh quotient.*/
/* ------------------------------------------------------------------ */

double orc_power_norm(int which, int N, int V, int B, const double *angles,
                      const double *taps, const double *taps_hi, const double *sv, int half,
                      const double *w, int iters)
{
    size_t I = (size_t)V * B, J = (size_t)N * N;
    size_t n = which == 0 ? J : I;
    double *v = malloc(sizeof(double) * n), *u = malloc(sizeof(double) * n);
    double *s1 = malloc(sizeof(double) * I), *s2 = malloc(sizeof(double) * I);
    double *dtmp = malloc(sizeof(double) * 2 * I);
    double lam = 0.0;
    for (size_t i = 0; i < n; ++i) v[i] = 1.0;
    for (int it = 0; it < iters; ++it) {
        double nv = 0.0;
        for (size_t i = 0; i < n; ++i) nv += v[i] * v[i];
        nv = sqrt(nv);
        for (size_t i = 0; i < n; ++i) v[i] /= nv;
        if (which == 0) {
            orc_project(N, V, B, angles, v, s1);
            apply_d(V, B, taps, taps_hi, half, sv, s1, s2, dtmp);
            orc_backproject(N, V, B, angles, s2, u);
        } else {
            for (size_t i = 0; i < I; ++i) s1[i] = v[i] / sqrt(w[i]);
            apply_d(V, B, taps, taps_hi, half, sv, s1, s2, dtmp);
            for (size_t i = 0; i < I; ++i) u[i] = s2[i] / sqrt(w[i]);
        }
        lam = 0.0;
        for (size_t i = 0; i < n; ++i) lam += v[i] * u[i];
        memcpy(v, u, sizeof(double) * n);
    }
    free(v);
    free(u);
    free(s1);
    free(s2);
    free(dtmp);
    return lam;
}

/* ------------------------------------------------------------------ */
/* Independent reference for limits: the Chambolle-Pock iteration on   */
/* K = [A; grad] with no inner loop, for                               */
/*   mode 0: min_{x>=0} beta TV(x) + 1/2 ||Ax - b||_W^2   (Eq. 1)       */
/*   mode 1: min_{x>=0} TV(x)  s.t.  Ax = b               (Eq. 25)      */
/*           (eps > 0: s.t. ||Ax - b|| <= eps, Sec. 5)                  */
/* Dual variables q (sinogram) and (gx, gy) (image pair):              */
/*   q  <- prox_{s F1*}(q + s A xb),  F1* = conj. of the fidelity      */
/*   g  <- project onto |g_j| <= beta of (g + s grad xb)               */
/*   x' <- max(0, x - t (A^T q - div g)),  xb = 2 x' - x.               */
/* Requires s t (||A||^2 + 8) < 1.  Runs `iters` iterations from zero.  */
/* ------------------------------------------------------------------ */

void orc_cp_reference(int N, int V, int B, const double *angles,
                      const double *b, const double *w, int mode,
                      double beta, double eps, double s, double t, int iters, double *x)
{
    size_t I = (size_t)V * B, J = (size_t)N * N;
    double *q = calloc(I, sizeof(double)), *ax = malloc(sizeof(double) * I);
    double *gxd = calloc(J, sizeof(double)), *gyd = calloc(J, sizeof(double));
    double *gx = malloc(sizeof(double) * J), *gy = malloc(sizeof(double) * J);
    double *xb = calloc(J, sizeof(double)), *xn = malloc(sizeof(double) * J);
    double *atq = malloc(sizeof(double) * J), *dv = malloc(sizeof(double) * J);
    double bnd = (mode == 0) ? beta : 1.0;
    memset(x, 0, sizeof(double) * J);
    for (int it = 0; it < iters; ++it) {
        orc_project(N, V, B, angles, xb, ax);
        if (mode == 1 && eps > 0.0) {
            /* Moreau: prox_{sF*}(y) = y - s P(y / s), P the projection onto
             * the ball of radius eps about b */
            double n2 = 0.0;
            for (size_t i = 0; i < I; ++i) {
                double u = (q[i] + s * ax[i]) / s - b[i];
                n2 += u * u;
            }
            double f = sqrt(n2) > eps ? eps / sqrt(n2) : 1.0;
            for (size_t i = 0; i < I; ++i) {
                double y = q[i] + s * ax[i];
                q[i] = y - s * (b[i] + f * (y / s - b[i]));
            }
        } else {
            for (size_t i = 0; i < I; ++i) {
                double y = q[i] + s * ax[i];
                if (mode == 0) q[i] = (y - s * b[i]) / (1.0 + s / w[i]);
                else q[i] = y - s * b[i];
            }
        }
        orc_grad(N, xb, gx, gy);
        for (size_t j = 0; j < J; ++j) {
            double a1 = gxd[j] + s * gx[j], a2 = gyd[j] + s * gy[j];
            double nrm = sqrt(a1 * a1 + a2 * a2);
            double sc = nrm > bnd ? bnd / nrm : 1.0;
            gxd[j] = a1 * sc;
            gyd[j] = a2 * sc;
        }
        orc_backproject(N, V, B, angles, q, atq);
        orc_div(N, gxd, gyd, dv);
        for (size_t j = 0; j < J; ++j) {
            double v = x[j] - t * (atq[j] - dv[j]);
            xn[j] = v > 0.0 ? v : 0.0;
        }
        for (size_t j = 0; j < J; ++j) {
            xb[j] = 2.0 * xn[j] - x[j];
            x[j] = xn[j];
        }
    }
    free(q); free(ax); free(gxd); free(gyd); free(gx); free(gy);
    free(xb); free(xn); free(atq); free(dv);
}
