// k_tv.cu -- prox of tau*g (Eq. 17): argmin_{x>=0} lam TV(x) + 1/2 ||x - z||^2
// by projected-gradient steps on the TV dual field p = (px, py), |p_j| <= 1:
//     x_l = max(0, z + lam div p),   p <- Pi(p + grad x_l / (8 lam)),
// then x = max(0, z + lam div p).  grad is the forward difference (zero
// across the last row/column), div = -grad^T.  lam = 0 gives max(0, z).
//
// Temporal blocking: one block owns a tile of tc x tr pixels and holds it
// with a halo of H = steps + 1 pixels on every side.  Each step spoils one
// more ring of the halo (its outermost cells see zeros instead of their
// neighbours), so after `steps` steps the tile holds exactly what a
// whole-image iteration would give, with no grid-wide synchronisation and
// one pass over global memory per call.  p is double-buffered (p_in ->
// p_out) because neighbouring blocks read the old p in their halos.
//
// The held region is 64 columns (lane l owns columns 2l, 2l+1) by up to
// TV_ROWS rows (warp w owns rows w + 16 j), so tc = 64 - 2H.  Every cell's
// z, p and x stay in registers for the whole call; left/right neighbours
// come from the adjacent lane by shuffle, and each phase publishes the one
// field its vertical neighbours need (x for the dual step, p_y for the
// divergence) in shared memory.  Outside the image, and where a forward
// difference does not exist (p_x on the last column, p_y on the last row),
// p is zero and stays zero: the dual step's factor is 0 there, so the
// divergence needs no boundary tests.
#include <algorithm>

#include "ctpd_internal.cuh"

namespace ctpd {

constexpr int TV_WARPS = 16;
constexpr int TV_THREADS = TV_WARPS * 32;
constexpr int TV_J = 5;                     // region rows per warp
constexpr int TV_ROWS = TV_WARPS * TV_J;    // 80
constexpr int TV_MAX_STEPS = 16;            // H = 17: 30 interior columns
constexpr int TV_MIN_TR = 16;               // fewest interior rows per tile

int tv_max_steps() { return TV_MAX_STEPS; }

struct TvTiles {
    int tc, tr, ncb, nrb;
};

// Column tiles are as wide as the region allows; rows are split so that the
// tiles of one image about fill the GPU once (one block per SM), but no
// narrower than TV_MIN_TR rows and no taller than the region.
static TvTiles tv_tiles(int N, int steps, int n_sm, int min_tr)
{
    const int H = steps + 1;
    TvTiles t;
    t.tc = 64 - 2 * H;
    t.ncb = (N + t.tc - 1) / t.tc;
    const int tr_max = TV_ROWS - 2 * H;
    int nrb = std::max(1, n_sm / t.ncb);
    nrb = std::min(nrb, (N + min_tr - 1) / min_tr);
    nrb = std::max(nrb, (N + tr_max - 1) / tr_max);
    t.tr = (N + nrb - 1) / nrb;
    t.nrb = (N + t.tr - 1) / t.tr;
    return t;
}

// FGP: the fast gradient projection (Beck and Teboulle): each step is the
// projected-gradient step taken at r = p + theta (p - p_prev) instead of p,
// with theta_k = (t_k - 1) / t_{k+1}, t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
// (momentum restarted at every call).  Each cell keeps p_prev as well, and
// the field published for the divergence is r_y (p_y after the last step).
template <bool FGP>
__global__ void __launch_bounds__(TV_THREADS, 1)
k_tv(const float *__restrict__ z, const float *__restrict__ p_in, float *__restrict__ p_out,
     float *__restrict__ x, int N, int steps, int final_, int tc, int tr, const double *__restrict__ scal)
{
    // row li of the region at index (li + 1) * 32 + lane; rows -1 and
    // beyond the region read zeros
    __shared__ float2 pub_x[(TV_ROWS + 2) * 32];
    __shared__ float2 pub_y[(TV_ROWS + 2) * 32];
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int H = steps + 1, Sr = tr + 2 * H;
    const int R0 = blockIdx.y * tr - H, C0 = blockIdx.x * tc - H;
    const int c0 = C0 + 2 * lane;   // image columns c0, c0 + 1 of this lane
    const size_t NN = (size_t)N * N;
    const float lam = fscal(scal, F_LAMBDA);
    const float inv8 = fscal(scal, F_INV8LAM);
    // forward differences: along x on columns 0..N-2, along y on columns 0..N-1
    const bool cx0 = (unsigned)c0 < (unsigned)(N - 1), cx1 = (unsigned)(c0 + 1) < (unsigned)(N - 1);
    const bool cy0 = (unsigned)c0 < (unsigned)N, cy1 = (unsigned)(c0 + 1) < (unsigned)N;

    for (int i = threadIdx.x; i < (TV_ROWS + 2) * 32; i += TV_THREADS) {
        pub_x[i] = make_float2(0.0f, 0.0f);
        pub_y[i] = make_float2(0.0f, 0.0f);
    }
    float zr[TV_J][2], pxr[TV_J][2], pyr[TV_J][2], xr[TV_J][2];
    float pxo[TV_J][2], pyo[TV_J][2];   // FGP: p of the previous step
    unsigned rowx = 0, rowy = 0;   // bit j: row in the image / row with a y difference
#pragma unroll
    for (int j = 0; j < TV_J; ++j) {
        const int li = w + TV_WARPS * j, rr = R0 + li;
        const bool rin = li < Sr && (unsigned)rr < (unsigned)N;
        const bool ryd = li < Sr && (unsigned)rr < (unsigned)(N - 1);
        rowx |= (unsigned)rin << j;
        rowy |= (unsigned)ryd << j;
        zr[j][0] = zr[j][1] = pxr[j][0] = pxr[j][1] = pyr[j][0] = pyr[j][1] = 0.0f;
        xr[j][0] = xr[j][1] = 0.0f;
        if (rin) {
            const size_t gi = (size_t)rr * N + c0;   // c0 may be -1..: only valid columns are read
            if (cy0) zr[j][0] = z[gi];
            if (cy1) zr[j][1] = z[gi + 1];
            if (cx0) pxr[j][0] = p_in[gi];
            if (cx1) pxr[j][1] = p_in[gi + 1];
            if (ryd && cy0) pyr[j][0] = p_in[NN + gi];
            if (ryd && cy1) pyr[j][1] = p_in[NN + gi + 1];
        }
    }
#pragma unroll
    for (int j = 0; j < TV_J; ++j) {
        pxo[j][0] = pxr[j][0];
        pxo[j][1] = pxr[j][1];
        pyo[j][0] = pyr[j][0];
        pyo[j][1] = pyr[j][1];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TV_J; ++j) {
        const int li = w + TV_WARPS * j;
        if (li < Sr) pub_y[(li + 1) * 32 + lane] = make_float2(pyr[j][0], pyr[j][1]);
    }
    __syncthreads();

    if (lam > 0.0f) {
        float t = 1.0f, th = 0.0f;   // FGP: t_k and theta_{k-1} (theta_0 = 0)
        for (int it = 0; it < steps; ++it) {
            // x = max(0, z + lam div r), r = p (GP) or p + theta (p - p_prev) (FGP)
#pragma unroll
            for (int j = 0; j < TV_J; ++j) {
                const int li = w + TV_WARPS * j;
                if (li < Sr) {
                    const float2 pa = pub_y[li * 32 + lane];   // r_y of row li - 1
                    const float rx0 = FGP ? fmaf(th, pxr[j][0] - pxo[j][0], pxr[j][0]) : pxr[j][0];
                    const float rx1 = FGP ? fmaf(th, pxr[j][1] - pxo[j][1], pxr[j][1]) : pxr[j][1];
                    const float ry0 = FGP ? fmaf(th, pyr[j][0] - pyo[j][0], pyr[j][0]) : pyr[j][0];
                    const float ry1 = FGP ? fmaf(th, pyr[j][1] - pyo[j][1], pyr[j][1]) : pyr[j][1];
                    float pl = __shfl_up_sync(FULL, rx1, 1);
                    if (lane == 0) pl = 0.0f;
                    const float d0 = (rx0 - pl) + (ry0 - pa.x);
                    const float d1 = (rx1 - rx0) + (ry1 - pa.y);
                    xr[j][0] = fmaxf(0.0f, fmaf(lam, d0, zr[j][0]));
                    xr[j][1] = fmaxf(0.0f, fmaf(lam, d1, zr[j][1]));
                    pub_x[(li + 1) * 32 + lane] = make_float2(xr[j][0], xr[j][1]);
                }
            }
            __syncthreads();
            // FGP: theta_k for the next extrapolation
            const float t1 = FGP ? 0.5f * (1.0f + sqrtf(fmaf(4.0f * t, t, 1.0f))) : 1.0f;
            const float thn = FGP ? (t - 1.0f) / t1 : 0.0f;
            const bool last = it + 1 == steps;
            // p = Pi(p + grad x / (8 lam)), Pi(q) = q / max(1, |q|)
#pragma unroll
            for (int j = 0; j < TV_J; ++j) {
                const int li = w + TV_WARPS * j;
                if (li < Sr) {
                    const float2 xb = pub_x[(li + 2) * 32 + lane];   // x of row li + 1
                    const float xrt = __shfl_down_sync(FULL, xr[j][0], 1);
                    const bool rx = (rowx >> j) & 1u, ry = (rowy >> j) & 1u;
                    const float mx0 = (rx && cx0) ? inv8 : 0.0f, mx1 = (rx && cx1) ? inv8 : 0.0f;
                    const float my0 = (ry && cy0) ? inv8 : 0.0f, my1 = (ry && cy1) ? inv8 : 0.0f;
                    const float rx0 = FGP ? fmaf(th, pxr[j][0] - pxo[j][0], pxr[j][0]) : pxr[j][0];
                    const float rx1 = FGP ? fmaf(th, pxr[j][1] - pxo[j][1], pxr[j][1]) : pxr[j][1];
                    const float ry0 = FGP ? fmaf(th, pyr[j][0] - pyo[j][0], pyr[j][0]) : pyr[j][0];
                    const float ry1 = FGP ? fmaf(th, pyr[j][1] - pyo[j][1], pyr[j][1]) : pyr[j][1];
                    const float qx0 = fmaf(xr[j][1] - xr[j][0], mx0, rx0);
                    const float qx1 = fmaf(xrt - xr[j][1], mx1, rx1);
                    const float qy0 = fmaf(xb.x - xr[j][0], my0, ry0);
                    const float qy1 = fmaf(xb.y - xr[j][1], my1, ry1);
                    const float s0 = fminf(1.0f, rsqrtf(fmaf(qx0, qx0, qy0 * qy0)));
                    const float s1 = fminf(1.0f, rsqrtf(fmaf(qx1, qx1, qy1 * qy1)));
                    if (FGP) {
                        pxo[j][0] = pxr[j][0];
                        pxo[j][1] = pxr[j][1];
                        pyo[j][0] = pyr[j][0];
                        pyo[j][1] = pyr[j][1];
                    }
                    pxr[j][0] = qx0 * s0;
                    pxr[j][1] = qx1 * s1;
                    pyr[j][0] = qy0 * s0;
                    pyr[j][1] = qy1 * s1;
                    if (FGP && !last)   // r_y of the next step
                        pub_y[(li + 1) * 32 + lane] =
                            make_float2(fmaf(thn, pyr[j][0] - pyo[j][0], pyr[j][0]),
                                        fmaf(thn, pyr[j][1] - pyo[j][1], pyr[j][1]));
                    else
                        pub_y[(li + 1) * 32 + lane] = make_float2(pyr[j][0], pyr[j][1]);
                }
            }
            __syncthreads();
            t = t1;
            th = thn;
        }
    }

    // the tile interior: p, and x = max(0, z + lam div p) on the last chunk
#pragma unroll
    for (int j = 0; j < TV_J; ++j) {
        const int li = w + TV_WARPS * j, rr = R0 + li;
        if (li >= H && li < H + tr && rr < N) {
            const float2 pa = pub_y[li * 32 + lane];
            float pl = __shfl_up_sync(FULL, pxr[j][1], 1);
            if (lane == 0) pl = 0.0f;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int lj = 2 * lane + e, cc = C0 + lj;
                if (lj >= H && lj < H + tc && cc < N) {
                    const size_t gi = (size_t)rr * N + cc;
                    if (lam > 0.0f) {
                        p_out[gi] = pxr[j][e];
                        p_out[NN + gi] = pyr[j][e];
                    }
                    if (final_) {
                        const float dv = e == 0 ? (pxr[j][0] - pl) + (pyr[j][0] - pa.x)
                                                : (pxr[j][1] - pxr[j][0]) + (pyr[j][1] - pa.y);
                        x[gi] = fmaxf(0.0f, fmaf(lam, dv, zr[j][e]));
                    }
                }
            }
        }
    }
}

void launch_tv(const float *z, const float *p_in, float *p_out, float *x,
               int n, int n_sm, int min_rows, int steps, int final_, const double *scal, cudaStream_t st, bool fgp)
{
    const TvTiles t = tv_tiles(n, steps, n_sm, min_rows > 0 ? min_rows : TV_MIN_TR);
    counted();
    if (fgp)
        k_tv<true><<<dim3(t.ncb, t.nrb), TV_THREADS, 0, st>>>(z, p_in, p_out, x, n, steps, final_, t.tc, t.tr, scal);
    else
        k_tv<false><<<dim3(t.ncb, t.nrb), TV_THREADS, 0, st>>>(z, p_in, p_out, x, n, steps, final_, t.tc, t.tr, scal);
}

void kernel_attrs_tv() {}


// =====================================================================
// Whole-image single steps of the same projected-gradient iteration, and
// their adjoints, for the differentiable unrolled solve.  One thread per
// pixel, blockIdx.z = image of a batch; p = (px, py) stored as two N x N
// planes.  The adjoints use div = -grad^T, the mask of max(0, .), and the
// Jacobian of the unit-ball projection Pi(q) = q / max(1, |q|), which is I
// inside the ball and (I - qhat qhat^T) / |q| outside it.
// =====================================================================
namespace {

__device__ __forceinline__ float tv_div(const float *px, const float *py, int r, int c, int N)
{
    const size_t j = (size_t)r * N + c;
    return ((c < N - 1 ? px[j] : 0.0f) - (c > 0 ? px[j - 1] : 0.0f)) +
           ((r < N - 1 ? py[j] : 0.0f) - (r > 0 ? py[j - N] : 0.0f));
}

// s = z + lam div p (before the max(0, .))
__device__ __forceinline__ float tv_s(const float *z, const float *px, const float *py, int r, int c, int N, float lam)
{
    return z[(size_t)r * N + c] + lam * tv_div(px, py, r, c, N);
}

// q = p + inv8 grad max(0, s) at (r, c)
__device__ __forceinline__ float2 tv_q(const float *z, const float *px, const float *py, int r, int c, int N,
                                       float lam, float inv8)
{
    const size_t j = (size_t)r * N + c;
    const float x0 = fmaxf(0.0f, tv_s(z, px, py, r, c, N, lam));
    const float gx = c < N - 1 ? fmaxf(0.0f, tv_s(z, px, py, r, c + 1, N, lam)) - x0 : 0.0f;
    const float gy = r < N - 1 ? fmaxf(0.0f, tv_s(z, px, py, r + 1, c, N, lam)) - x0 : 0.0f;
    return make_float2(px[j] + gx * inv8, py[j] + gy * inv8);
}

// J_Pi(q)^T g
__device__ __forceinline__ float2 proj_adj(float2 q, float2 g)
{
    const float n2 = fmaf(q.x, q.x, q.y * q.y);
    if (n2 <= 1.0f) return g;
    const float inv = rsqrtf(n2);
    const float hx = q.x * inv, hy = q.y * inv;
    const float d = hx * g.x + hy * g.y;
    return make_float2((g.x - hx * d) * inv, (g.y - hy * d) * inv);
}

__device__ __forceinline__ void block_sum_to(double v, double *partials)
{
    __shared__ double red[256];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    if (t == 0)
        partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

}  // namespace

// p_out = Pi(p_in + inv8 grad max(0, z + lam div p_in))
__global__ void __launch_bounds__(256)
k_tv_step(const float *__restrict__ z, const float *__restrict__ p_in, float *__restrict__ p_out, int N,
          const double *__restrict__ scal)
{
    const int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    if (r >= N || c >= N) return;
    const size_t NN = (size_t)N * N, j = (size_t)r * N + c;
    const float *zz = z + blockIdx.z * NN;
    const float *px = p_in + blockIdx.z * 2 * NN, *py = px + NN;
    float *ox = p_out + blockIdx.z * 2 * NN, *oy = ox + NN;
    const float lam = fscal(scal, F_LAMBDA), inv8 = fscal(scal, F_INV8LAM);
    const float2 q = tv_q(zz, px, py, r, c, N, lam, inv8);
    const float sc = fminf(1.0f, rsqrtf(fmaf(q.x, q.x, q.y * q.y)));
    ox[j] = q.x * sc;
    oy[j] = q.y * sc;
}

// x = max(0, z + lam div p)
__global__ void __launch_bounds__(256)
k_tv_final(const float *__restrict__ z, const float *__restrict__ p, float *__restrict__ x, int N,
           const double *__restrict__ scal)
{
    const int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    if (r >= N || c >= N) return;
    const size_t NN = (size_t)N * N;
    const float *px = p + blockIdx.z * 2 * NN, *py = px + NN;
    x[blockIdx.z * NN + (size_t)r * N + c] =
        fmaxf(0.0f, tv_s(z + blockIdx.z * NN, px, py, r, c, N, fscal(scal, F_LAMBDA)));
}

// Adjoint of x = max(0, s), s = z + lam div p, with the adjoint gp_next of p
// flowing in from later: gs = gx [s > 0]; gz = gs; gp = gp_next - lam grad gs;
// partial sums of <gs, div p> (the lam derivative).
__global__ void __launch_bounds__(256)
k_tv_final_bwd(const float *__restrict__ z, const float *__restrict__ p, const float *__restrict__ gx,
               const float *__restrict__ gp_next, float *__restrict__ gz, float *__restrict__ gp, int N,
               const double *__restrict__ scal, double *__restrict__ part_lam)
{
    const int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    double contrib = 0.0;
    if (r < N && c < N) {
        const size_t NN = (size_t)N * N, j = (size_t)r * N + c;
        const float *zz = z + blockIdx.z * NN, *g = gx + blockIdx.z * NN;
        const float *px = p + blockIdx.z * 2 * NN, *py = px + NN;
        const float lam = fscal(scal, F_LAMBDA);
        auto gs_at = [&](int rr, int cc) {
            return tv_s(zz, px, py, rr, cc, N, lam) > 0.0f ? g[(size_t)rr * N + cc] : 0.0f;
        };
        const float gs0 = gs_at(r, c);
        const float gsr = c < N - 1 ? gs_at(r, c + 1) : 0.0f;
        const float gsd = r < N - 1 ? gs_at(r + 1, c) : 0.0f;
        gz[blockIdx.z * NN + j] = gs0;
        const float *gnx = gp_next + blockIdx.z * 2 * NN, *gny = gnx + NN;
        float *ox = gp + blockIdx.z * 2 * NN, *oy = ox + NN;
        ox[j] = gnx[j] - lam * (c < N - 1 ? gsr - gs0 : 0.0f);
        oy[j] = gny[j] - lam * (r < N - 1 ? gsd - gs0 : 0.0f);
        contrib = (double)gs0 * (double)tv_div(px, py, r, c, N);
    }
    block_sum_to(contrib, part_lam);
}

// Adjoint of one step p' = Pi(q), q = p + inv8 grad x, x = max(0, s), part a:
// gq = J_Pi(q)^T gp_next, and partial sums of <gq, grad x> (the inv8 derivative).
__global__ void __launch_bounds__(256)
k_tv_step_bwd_a(const float *__restrict__ z, const float *__restrict__ p, const float *__restrict__ gp_next,
                float *__restrict__ gq, int N, const double *__restrict__ scal, double *__restrict__ part_inv8)
{
    const int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    double contrib = 0.0;
    if (r < N && c < N) {
        const size_t NN = (size_t)N * N, j = (size_t)r * N + c;
        const float *zz = z + blockIdx.z * NN;
        const float *px = p + blockIdx.z * 2 * NN, *py = px + NN;
        const float lam = fscal(scal, F_LAMBDA), inv8 = fscal(scal, F_INV8LAM);
        const float2 q = tv_q(zz, px, py, r, c, N, lam, inv8);
        const float *gnx = gp_next + blockIdx.z * 2 * NN, *gny = gnx + NN;
        const float2 g = proj_adj(q, make_float2(gnx[j], gny[j]));
        float *ox = gq + blockIdx.z * 2 * NN, *oy = ox + NN;
        ox[j] = g.x;
        oy[j] = g.y;
        // grad x = (q - p) / inv8 without the division: recompute it
        const float x0 = fmaxf(0.0f, tv_s(zz, px, py, r, c, N, lam));
        const float gxv = c < N - 1 ? fmaxf(0.0f, tv_s(zz, px, py, r, c + 1, N, lam)) - x0 : 0.0f;
        const float gyv = r < N - 1 ? fmaxf(0.0f, tv_s(zz, px, py, r + 1, c, N, lam)) - x0 : 0.0f;
        contrib = (double)g.x * gxv + (double)g.y * gyv;
    }
    block_sum_to(contrib, part_inv8);
}

// Part b: gx = -inv8 div gq; gs = gx [s > 0]; gz += gs; gp = gq - lam grad gs;
// partial sums of <gs, div p> (the lam derivative).
__global__ void __launch_bounds__(256)
k_tv_step_bwd_b(const float *__restrict__ z, const float *__restrict__ p, const float *__restrict__ gq,
                float *__restrict__ gz, float *__restrict__ gp, int N, const double *__restrict__ scal,
                double *__restrict__ part_lam)
{
    const int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    double contrib = 0.0;
    if (r < N && c < N) {
        const size_t NN = (size_t)N * N, j = (size_t)r * N + c;
        const float *zz = z + blockIdx.z * NN;
        const float *px = p + blockIdx.z * 2 * NN, *py = px + NN;
        const float *qx = gq + blockIdx.z * 2 * NN, *qy = qx + NN;
        const float lam = fscal(scal, F_LAMBDA), inv8 = fscal(scal, F_INV8LAM);
        auto gs_at = [&](int rr, int cc) {
            const float gxv = -inv8 * tv_div(qx, qy, rr, cc, N);
            return tv_s(zz, px, py, rr, cc, N, lam) > 0.0f ? gxv : 0.0f;
        };
        const float gs0 = gs_at(r, c);
        const float gsr = c < N - 1 ? gs_at(r, c + 1) : 0.0f;
        const float gsd = r < N - 1 ? gs_at(r + 1, c) : 0.0f;
        gz[blockIdx.z * NN + j] += gs0;
        float *ox = gp + blockIdx.z * 2 * NN, *oy = ox + NN;
        ox[j] = qx[j] - lam * (c < N - 1 ? gsr - gs0 : 0.0f);
        oy[j] = qy[j] - lam * (r < N - 1 ? gsd - gs0 : 0.0f);
        contrib = (double)gs0 * (double)tv_div(px, py, r, c, N);
    }
    block_sum_to(contrib, part_lam);
}

namespace {
dim3 tv_px_grid(int n, int batch) { return dim3((n + 31) / 32, (n + 7) / 8, batch); }
}

size_t tv_px_blocks(int n, int batch) { return (size_t)((n + 31) / 32) * ((n + 7) / 8) * batch; }

void launch_tv_step(const float *z, const float *p_in, float *p_out, int n, int batch, const double *scal,
                    cudaStream_t st)
{
    counted();
    k_tv_step<<<tv_px_grid(n, batch), dim3(32, 8), 0, st>>>(z, p_in, p_out, n, scal);
}

void launch_tv_final(const float *z, const float *p, float *x, int n, int batch, const double *scal, cudaStream_t st)
{
    counted();
    k_tv_final<<<tv_px_grid(n, batch), dim3(32, 8), 0, st>>>(z, p, x, n, scal);
}

void launch_tv_final_bwd(const float *z, const float *p, const float *gx, const float *gp_next, float *gz,
                         float *gp, int n, int batch, const double *scal, double *part_lam, cudaStream_t st)
{
    counted();
    k_tv_final_bwd<<<tv_px_grid(n, batch), dim3(32, 8), 0, st>>>(z, p, gx, gp_next, gz, gp, n, scal, part_lam);
}

void launch_tv_step_bwd(const float *z, const float *p, const float *gp_next, float *gq, float *gz, float *gp,
                        int n, int batch, const double *scal, double *part_inv8, double *part_lam, cudaStream_t st)
{
    counted(2);
    k_tv_step_bwd_a<<<tv_px_grid(n, batch), dim3(32, 8), 0, st>>>(z, p, gp_next, gq, n, scal, part_inv8);
    k_tv_step_bwd_b<<<tv_px_grid(n, batch), dim3(32, 8), 0, st>>>(z, p, gq, gz, gp, n, scal, part_lam);
}

}  // namespace ctpd
