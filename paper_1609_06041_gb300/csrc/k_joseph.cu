// k_joseph.cu -- Joseph forward projector A and its exact-transpose,
// pixel-driven backprojector A^T (the A and A^T of Eqs. 18-20 / 29-31).
#include "ctpd_internal.cuh"

namespace ctpd {

// ---------------------------------------------------------------------
// Forward projection, one thread per ray (v, d).  Row-stepping views read
// the image row by row; column-stepping views read the transposed image
// row by row, so both classes sweep contiguous memory and a warp (32
// neighbouring bins) touches neighbouring pixels of the same line.
// Each step: u, its floor i0 and fraction f, and (1-f) x[i0] + f x[i0+1]
// with zero outside the image.  Only the steps whose u can fall inside
// (-1, N) are visited (a conservative range, one step of margin).
// ---------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(128)
k_project(const float *__restrict__ x, const float *__restrict__ xT,
          const ViewP *__restrict__ views, int N, int V, int B,
          float *__restrict__ out, const float *__restrict__ b,
          const float *__restrict__ winv, const float *__restrict__ mu)
{
    // xT == NULL: column-stepping views read x with a stride of N (used by
    // the stand-alone projector; the solve keeps a transposed copy).
    const int v = blockIdx.y;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t img_off = (size_t)blockIdx.z * N * N;
    const size_t sino_off = (size_t)blockIdx.z * V * B;
    if (d >= B) return;
    const ViewP P = views[v];
    const float *img = ((P.rows || xT == nullptr) ? x : xT) + img_off;
    const int ss = (P.rows || xT != nullptr) ? N : 1;   // stride between steps
    const int su = (P.rows || xT != nullptr) ? 1 : N;   // stride along u
    const float h = 0.5f * (float)(N - 1);
    const float dp = (float)d - 0.5f * (float)(B - 1);

    // steps s with -1 < u(s) < N:  u(s) = h + dp*a + (s - h)*m
    int lo = 0, hi = N - 1;
    const float u0 = h + dp * P.a;     // u at s = h
    if (P.m != 0.0f) {
        float sa = (-1.0f - u0) / P.m + h, sb = ((float)N - u0) / P.m + h;
        float smin = fminf(sa, sb), smax = fmaxf(sa, sb);
        // clamp before converting: far-off rays give huge (or infinite) s
        smin = fminf(fmaxf(smin, -2.0f), (float)N + 2.0f);
        smax = fminf(fmaxf(smax, -3.0f), (float)N + 1.0f);
        lo = max(0, (int)floorf(smin) - 1);
        hi = min(N - 1, (int)ceilf(smax) + 1);
    } else if (!(u0 > -2.0f && u0 < (float)N + 1.0f)) {
        hi = -1;
    }
    float acc = 0.0f;
    for (int s = lo; s <= hi; ++s) {
        const float u = joseph_u(dp, P.a, (float)s - h, P.m, h);
        int i0;
        float f;
        joseph_split(u, i0, f);
        const float *row = img + (size_t)s * ss;
        const float x0 = (i0 >= 0 && i0 < N) ? __ldg(row + (size_t)i0 * su) : 0.0f;
        const float x1 = (i0 + 1 >= 0 && i0 + 1 < N) ? __ldg(row + (size_t)(i0 + 1) * su) : 0.0f;
        acc += __fmaf_rn(1.0f - f, x0, __fmul_rn(f, x1));
    }
    float val = acc * P.scale;
    const size_t o = sino_off + (size_t)v * B + d;
    if (MODE == 1) val = val - b[o] - winv[o] * mu[o];
    else if (MODE == 2) val = val - b[o];
    out[o] = val;
}

void launch_project(const Geometry *g, const float *x, const float *xT, float *out,
                    int mode, const float *b, const float *winv, const float *mu,
                    int batch, cudaStream_t st)
{
    dim3 blk(128), grd((g->n_bins + 127) / 128, g->n_views, batch);
    counted();
    if (mode == 0)
        k_project<0><<<grd, blk, 0, st>>>(x, xT, g->d_views, g->n, g->n_views, g->n_bins, out, b, winv, mu);
    else if (mode == 1)
        k_project<1><<<grd, blk, 0, st>>>(x, xT, g->d_views, g->n, g->n_views, g->n_bins, out, b, winv, mu);
    else
        k_project<2><<<grd, blk, 0, st>>>(x, xT, g->d_views, g->n, g->n_views, g->n_bins, out, b, winv, mu);
}

// ---------------------------------------------------------------------
// Backprojection, one thread per pixel (r, c), gathering over views.  For
// a view the pixel is the `j`-th pixel (along u) of step `s` (row r for a
// row-stepping view, column c for a column-stepping one).  The rays that
// can reach it have u(d, s) in [j-1, j+1), i.e. d within |inv_a| of the
// pixel's own detector coordinate; each candidate recomputes u with the
// same joseph_u as the projector and takes weight 1-f if floor(u) = j,
// f if floor(u) = j-1.  The candidate window carries a 1e-3 bin margin, so
// rounding never drops a ray the projector uses.
// ---------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256)
k_backproject(const float *__restrict__ y, float *__restrict__ out,
              const ViewP *__restrict__ views, int N, int V, int B,
              const float *__restrict__ xin, const double *__restrict__ scal)
{
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int r = blockIdx.y * 8 + threadIdx.y;
    if (r >= N || c >= N) return;
    const size_t img_off = (size_t)blockIdx.z * N * N;
    const float *ys = y + (size_t)blockIdx.z * V * B;
    const float h = 0.5f * (float)(N - 1);
    const float hb = 0.5f * (float)(B - 1);
    float acc = 0.0f;
    for (int v = 0; v < V; ++v) {
        const ViewP P = views[v];
        const int s = P.rows ? r : c;
        const int j = P.rows ? c : r;
        const float sp = (float)s - h;
        const float t = __fmul_rn(sp, P.m);
        const float e = ((float)j - h - t) * P.inv_a + hb;   // detector coordinate of the pixel
        const float wdt = fabsf(P.inv_a) + 1e-3f;
        const int dlo = max(0, (int)ceilf(e - wdt));
        const int dhi = min(B - 1, (int)floorf(e + wdt));
        const float *yv = ys + (size_t)v * B;
        float av = 0.0f;
        for (int d = dlo; d <= dhi; ++d) {
            const float u = joseph_u((float)d - hb, P.a, sp, P.m, h);
            int i0;
            float f;
            joseph_split(u, i0, f);
            const float wgt = (i0 == j) ? (1.0f - f) : ((i0 + 1 == j) ? f : 0.0f);
            av += wgt * __ldg(yv + d);
        }
        acc += av * P.scale;
    }
    const size_t o = img_off + (size_t)r * N + c;
    if (MODE == 0) out[o] = acc;
    else out[o] = xin[o] - (float)scal[S_TAU] * acc;
}

void launch_backproject(const Geometry *g, const float *y, float *out, int mode,
                        const float *xin, const double *scal, int batch, cudaStream_t st)
{
    dim3 blk(32, 8), grd((g->n + 31) / 32, (g->n + 7) / 8, batch);
    counted();
    if (mode == 0)
        k_backproject<0><<<grd, blk, 0, st>>>(y, out, g->d_views, g->n, g->n_views, g->n_bins, xin, scal);
    else
        k_backproject<1><<<grd, blk, 0, st>>>(y, out, g->d_views, g->n, g->n_views, g->n_bins, xin, scal);
}

// 32x32 tiles through shared memory (padded against bank conflicts).
__global__ void k_transpose(const float *__restrict__ x, float *__restrict__ xT, int N)
{
    __shared__ float tile[32][33];
    const size_t off = (size_t)blockIdx.z * N * N;
    int c = blockIdx.x * 32 + threadIdx.x;
    for (int k = threadIdx.y; k < 32; k += 8) {
        int r = blockIdx.y * 32 + k;
        if (r < N && c < N) tile[k][threadIdx.x] = x[off + (size_t)r * N + c];
    }
    __syncthreads();
    int r = blockIdx.y * 32 + threadIdx.x;
    for (int k = threadIdx.y; k < 32; k += 8) {
        int cc = blockIdx.x * 32 + k;
        if (r < N && cc < N) xT[off + (size_t)cc * N + r] = tile[threadIdx.x][k];
    }
}

void launch_transpose(const float *x, float *xT, int n, int batch, cudaStream_t st)
{
    dim3 blk(32, 8), grd((n + 31) / 32, (n + 31) / 32, batch);
    counted();
    k_transpose<<<grd, blk, 0, st>>>(x, xT, n);
}

}  // namespace ctpd
