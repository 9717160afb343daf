// k_tv.cu -- prox of tau*g (Eq. 17): argmin_{x>=0} lam TV(x) + 1/2 ||x - z||^2
// by projected-gradient steps on the TV dual field p = (px, py), |p_j| <= 1:
//     x_l = max(0, z + lam div p),   p <- Pi(p + grad x_l / (8 lam)),
// then x = max(0, z + lam div p).  grad is the forward difference (zero
// across the last row/column), div = -grad^T.  lam = 0 gives max(0, z).
//
// Temporal blocking: one block owns a tile of tc x tr pixels and holds it
// with a halo of H >= steps + 1 pixels on every side.  Each step spoils one
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

#include "body_tv.cuh"

namespace ctpd {

int tv_max_steps() { return TV_MAX_STEPS; }

struct TvTiles {
    int tc, tr, ncb, nrb;
};

// Column tiles are as wide as the region allows; rows are split so that the
// tiles of one image about fill the GPU once (one block per SM), but no
// narrower than TV_MIN_TR rows and no taller than the region.
static TvTiles tv_tiles(int N, int steps, int n_sm, int min_tr, bool even = false, int rows = TV_ROWS)
{
    const int H = tv_halo(steps, even);
    TvTiles t;
    t.tc = 64 - 2 * H;
    t.ncb = (N + t.tc - 1) / t.tc;
    const int tr_max = rows - 2 * H;
    int nrb = std::max(1, n_sm / t.ncb);
    nrb = std::min(nrb, (N + min_tr - 1) / min_tr);
    nrb = std::max(nrb, (N + tr_max - 1) / tr_max);
    t.tr = (N + nrb - 1) / nrb;
    t.nrb = (N + t.tr - 1) / t.tr;
    return t;
}

template <bool FGP, bool TRAJ>
__global__ void __launch_bounds__(TV_THREADS, 1)
k_tv(const float *__restrict__ z, const float *__restrict__ p_in, float *__restrict__ p_out,
     float *__restrict__ x, int N, int steps, int final_, int tc, int tr, const double *__restrict__ scal,
     float *__restrict__ traj)
{
    __shared__ float2 pub_x[(TV_ROWS + 2) * 32];
    __shared__ float2 pub_y[(TV_ROWS + 2) * 32];
    pdl_wait();
    tv_body<FGP, TRAJ>(whole_block(), blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z, pub_x, pub_y, z, p_in, p_out, x,
                       N, steps, final_, tc, tr, scal, traj);
}

void tv_tile_shape(int n, int steps, int n_sm, int min_rows, int *tc, int *tr, int *ncb, int *nrb, int rows)
{
    const TvTiles t = tv_tiles(n, steps, std::max(1, n_sm), min_rows > 0 ? min_rows : TV_MIN_TR, false,
                               rows > 0 ? rows : TV_ROWS);
    *tc = t.tc;
    *tr = t.tr;
    *ncb = t.ncb;
    *nrb = t.nrb;
}

void launch_tv(const float *z, const float *p_in, float *p_out, float *x,
               int n, int n_sm, int min_rows, int steps, int final_, const double *scal, cudaStream_t st, bool fgp,
               int batch, float *traj)
{
    // a batch fills the GPU with its images: the tiles of one image only
    // need to cover n_sm / batch SMs
    const TvTiles t = tv_tiles(n, steps, std::max(1, n_sm / std::max(1, batch)), min_rows > 0 ? min_rows : TV_MIN_TR,
                               traj != nullptr);
    const dim3 grid(t.ncb, t.nrb, std::max(1, batch));
    counted();
    auto kern = traj ? k_tv<false, true> : fgp ? k_tv<true, false> : k_tv<false, false>;
    launch_kernel(kern, grid, dim3(TV_THREADS), 0, st, z, p_in, p_out, x, n, steps, final_, t.tc, t.tr, scal, traj);
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

// Block sums of the per-thread float terms va, vb: a fixed shuffle tree per
// warp, then the block's warp sums in order (compensated FP32, FSum) into
// part[2 block], part[2 block + 1].  launch_pair_sums adds the partials of
// many launches at the end.  Blocks of 256 threads.
__device__ __forceinline__ void block_pair_to(float va, float vb, float *part)
{
    __shared__ float wa[8], wb[8];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        va += __shfl_down_sync(0xffffffffu, va, o);
        vb += __shfl_down_sync(0xffffffffu, vb, o);
    }
    if ((t & 31) == 0) {
        wa[t >> 5] = va;
        wb[t >> 5] = vb;
    }
    __syncthreads();
    if (t == 0) {
        FSum sa{0.0f, 0.0f}, sb{0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            fsum_add(sa, wa[k]);
            fsum_add(sb, wb[k]);
        }
        part[2 * blk] = sa.s + sa.c;
        part[2 * blk + 1] = sb.s + sb.c;
    }
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
               const double *__restrict__ scal, float *__restrict__ part)
{
    const int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    float contrib = 0.0f;
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
        contrib = gs0 * tv_div(px, py, r, c, N);
    }
    block_pair_to(0.0f, contrib, part);
}

// Adjoint of one step p' = Pi(q), q = p + inv8 grad x, x = max(0, s),
// s = z + lam div p, with the adjoint gp_next of p' flowing in from later:
//   gq = J_Pi(q)^T gp_next;   gx = -inv8 div gq;   gs = gx [s > 0];
//   gz += gs;   gp = gq - lam grad gs;
// and the derivative terms <gq, grad x> (for inv8) and <gs, div p> (for
// lam).  One block per BT_W x BT_H tile: p is staged with a halo of two,
// s with a halo of one (one more column and row on the far side), gq with
// a halo of one and gs one column and row past the tile, each phase
// reading only shared memory and the phase before.  The tile is 28 columns
// wide so that every staged row fits one warp: lane = column, warp = row.
constexpr int BT_W = 28, BT_H = 16;
constexpr int BP_H = BT_H + 4;   // p: origin (r0 - 2, c0 - 2), 32 columns
constexpr int BS_H = BT_H + 3;   // s: origin (r0 - 1, c0 - 1), 31 columns
constexpr int BQ_H = BT_H + 2;   // gq: origin (r0 - 1, c0 - 1), 30 columns
constexpr int BG_H = BT_H + 1;   // gs: origin (r0, c0), 29 columns

// INT: the tile and its halos lie inside the image, one cell away from the
// last row and column (r0 >= 2, c0 >= 2, r0 + BT_H + 3 <= N, c0 + 31 <= N),
// so every bounds and boundary test below is true and is left out.
struct BwdTile {   // the staged regions (one per block, shared by both paths)
    float PX[BP_H][32], PY[BP_H][32], SS[BS_H][32], QX[BQ_H][32], QY[BQ_H][32], GS[BG_H][32];
};

template <bool INT>
__device__ __forceinline__ void tv_step_bwd_tile(BwdTile &t, const float *__restrict__ z, const float *__restrict__ px,
                                                 const float *__restrict__ py, const float *__restrict__ gnx,
                                                 const float *__restrict__ gny, float *__restrict__ gz,
                                                 float *__restrict__ ox, float *__restrict__ oy, int N, int r0,
                                                 int c0, float lam, float inv8, float &c_inv8, float &c_lam)
{
    auto &PX = t.PX;
    auto &PY = t.PY;
    auto &SS = t.SS;
    auto &QX = t.QX;
    auto &QY = t.QY;
    auto &GS = t.GS;
    const int lx = threadIdx.x, ly = threadIdx.y;
    auto in_img = [&](int v) { return INT || (unsigned)v < (unsigned)N; };
    auto below_last = [&](int v) { return INT || v < N - 1; };   // a forward difference exists
    auto above_first = [&](int v) { return INT || v > 0; };
    // image column of this lane in each region, and whether it is inside
    const int bp = c0 - 2 + lx, bs = c0 - 1 + lx, bg = c0 + lx;
    const bool inp = in_img(bp), ins = lx < 31 && in_img(bs);
    const bool inq = lx < 30 && in_img(bs), ing = lx < 29 && in_img(bg);
    // div p at image cell (a, b) = region p cell (i, j) (zero outside the image)
    auto div_p = [&](int i, int j, int a, int b) {
        return ((below_last(b) ? PX[i][j] : 0.0f) - (above_first(b) ? PX[i][j - 1] : 0.0f)) +
               ((below_last(a) ? PY[i][j] : 0.0f) - (above_first(a) ? PY[i - 1][j] : 0.0f));
    };

    for (int i = ly; i < BP_H; i += 8) {
        const int a = r0 - 2 + i;
        const bool in = inp && in_img(a);
        const size_t gi = (size_t)a * N + bp;
        PX[i][lx] = in ? px[gi] : 0.0f;
        PY[i][lx] = in ? py[gi] : 0.0f;
    }
    // every global load of the block goes out before the first barrier
    float zr[3], gnr[3][2], gzr[2];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int i = ly + 8 * m, a = r0 - 1 + i;
        const bool in = ins && in_img(a);
        const size_t gi = (size_t)a * N + bs;
        zr[m] = (i < BS_H && in) ? z[gi] : 0.0f;
        gnr[m][0] = (i < BQ_H && lx < 30 && in) ? gnx[gi] : 0.0f;
        gnr[m][1] = (i < BQ_H && lx < 30 && in) ? gny[gi] : 0.0f;
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int a = r0 + ly + 8 * m;
        gzr[m] = (lx < BT_W && (INT || (bg < N && a < N))) ? gz[(size_t)a * N + bg] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 3; ++m) {   // s = z + lam div p
        const int i = ly + 8 * m, a = r0 - 1 + i;
        if (i < BS_H && lx < 31)
            SS[i][lx] = (ins && in_img(a)) ? fmaf(lam, div_p(i + 1, lx + 1, a, bs), zr[m]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 3; ++m) {   // gq = J_Pi(q)^T gp_next
        const int i = ly + 8 * m, a = r0 - 1 + i;
        if (i >= BQ_H) break;
        float2 g = make_float2(0.0f, 0.0f);
        if (inq && in_img(a)) {
            const float x0 = fmaxf(0.0f, SS[i][lx]);
            const float gxv = below_last(bs) ? fmaxf(0.0f, SS[i][lx + 1]) - x0 : 0.0f;
            const float gyv = below_last(a) ? fmaxf(0.0f, SS[i + 1][lx]) - x0 : 0.0f;
            const float2 q = make_float2(PX[i + 1][lx + 1] + gxv * inv8, PY[i + 1][lx + 1] + gyv * inv8);
            g = proj_adj(q, make_float2(gnr[m][0], gnr[m][1]));
            if (i >= 1 && i <= BT_H && lx >= 1 && lx <= BT_W) c_inv8 = fmaf(g.x, gxv, fmaf(g.y, gyv, c_inv8));
        }
        if (lx < 30) {
            QX[i][lx] = g.x;
            QY[i][lx] = g.y;
        }
    }
    __syncthreads();
    for (int i = ly; i < BG_H; i += 8) {   // gs = [s > 0] (-inv8 div gq)
        const int a = r0 + i;
        float v = 0.0f;
        if (ing && in_img(a) && SS[i + 1][lx + 1] > 0.0f) {
            const float d = ((below_last(bg) ? QX[i + 1][lx + 1] : 0.0f) - (above_first(bg) ? QX[i + 1][lx] : 0.0f)) +
                            ((below_last(a) ? QY[i + 1][lx + 1] : 0.0f) - (above_first(a) ? QY[i][lx + 1] : 0.0f));
            v = -inv8 * d;
        }
        if (lx < 29) GS[i][lx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int i = ly + 8 * m, a = r0 + i;
        if (lx < BT_W && (INT || (bg < N && a < N))) {
            const size_t gi = (size_t)a * N + bg;
            const float gs0 = GS[i][lx];
            gz[gi] = gzr[m] + gs0;
            ox[gi] = QX[i + 1][lx + 1] - lam * (below_last(bg) ? GS[i][lx + 1] - gs0 : 0.0f);
            oy[gi] = QY[i + 1][lx + 1] - lam * (below_last(a) ? GS[i + 1][lx] - gs0 : 0.0f);
            c_lam = fmaf(gs0, div_p(i + 2, lx + 2, a, bg), c_lam);
        }
    }
}

__global__ void __launch_bounds__(256, 6)
k_tv_step_bwd(const float *__restrict__ z, const float *__restrict__ p, const float *__restrict__ gp_next,
              float *__restrict__ gz, float *__restrict__ gp, int N, const double *__restrict__ scal,
              float *__restrict__ part)
{
    const int r0 = blockIdx.y * BT_H, c0 = blockIdx.x * BT_W;
    const size_t NN = (size_t)N * N;
    const float *px = p + blockIdx.z * 2 * NN;
    const float *gnx = gp_next + blockIdx.z * 2 * NN;
    float *ox = gp + blockIdx.z * 2 * NN;
    const float lam = fscal(scal, F_LAMBDA), inv8 = fscal(scal, F_INV8LAM);
    __shared__ BwdTile tile;
    float c_inv8 = 0.0f, c_lam = 0.0f;
    if (r0 >= 2 && c0 >= 2 && r0 + BT_H + 3 <= N && c0 + 31 <= N)
        tv_step_bwd_tile<true>(tile, z + blockIdx.z * NN, px, px + NN, gnx, gnx + NN, gz + blockIdx.z * NN, ox, ox + NN,
                               N, r0, c0, lam, inv8, c_inv8, c_lam);
    else
        tv_step_bwd_tile<false>(tile, z + blockIdx.z * NN, px, px + NN, gnx, gnx + NN, gz + blockIdx.z * NN, ox, ox + NN,
                                N, r0, c0, lam, inv8, c_inv8, c_lam);
    block_pair_to(c_inv8, c_lam, part);
}

namespace {
dim3 tv_px_grid(int n, int batch) { return dim3((n + 31) / 32, (n + 7) / 8, batch); }
}

// partials (two floats per block) of the adjoint kernels: the larger grid
size_t tv_px_blocks(int n, int batch)
{
    const size_t px = (size_t)((n + 31) / 32) * ((n + 7) / 8), tl = (size_t)((n + BT_W - 1) / BT_W) * ((n + BT_H - 1) / BT_H);
    return 2 * std::max(px, tl) * batch;
}

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
                         float *gp, int n, int batch, const double *scal, float *part, cudaStream_t st)
{
    counted();
    k_tv_final_bwd<<<tv_px_grid(n, batch), dim3(32, 8), 0, st>>>(z, p, gx, gp_next, gz, gp, n, scal, part);
}

void launch_tv_step_bwd(const float *z, const float *p, const float *gp_next, float *gz, float *gp, int n,
                        int batch, const double *scal, float *part, cudaStream_t st)
{
    counted();
    k_tv_step_bwd<<<dim3((n + BT_W - 1) / BT_W, (n + BT_H - 1) / BT_H, batch), dim3(32, 8), 0, st>>>(
        z, p, gp_next, gz, gp, n, scal, part);
}

// scal[slot_a] += sum of part[2 i], scal[slot_b] += sum of part[2 i + 1],
// i < npairs, in a fixed order and compensated FP32: PS_BLOCKS blocks add
// contiguous runs, one warp adds their results; the one thread then adds
// the two totals to the double slots.
constexpr int PS_BLOCKS = 152;

__global__ void __launch_bounds__(256) k_pair_sums(const float *__restrict__ part, size_t npairs, float *out)
{
    const size_t per = (npairs + gridDim.x - 1) / gridDim.x, lo = blockIdx.x * per;
    const size_t hi = lo + per < npairs ? lo + per : npairs;
    FSum a{0.0f, 0.0f}, b{0.0f, 0.0f};
    for (size_t i = lo + threadIdx.x; i < hi; i += 256) {
        const float2 v = reinterpret_cast<const float2 *>(part)[i];
        fsum_add(a, v.x);
        fsum_add(b, v.y);
    }
    __shared__ FSum ra[256], rb[256];
    ra[threadIdx.x] = a;
    rb[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            fsum_merge(ra[threadIdx.x], ra[threadIdx.x + o]);
            fsum_merge(rb[threadIdx.x], rb[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[4 * blockIdx.x] = ra[0].s;
        out[4 * blockIdx.x + 1] = ra[0].c;
        out[4 * blockIdx.x + 2] = rb[0].s;
        out[4 * blockIdx.x + 3] = rb[0].c;
    }
}

// one warp: strided lanes, then a fixed shuffle tree
__global__ void k_pair_final(const float *__restrict__ r, int nb, double *scal, int slot_a, int slot_b)
{
    FSum a{0.0f, 0.0f}, b{0.0f, 0.0f};
    for (int i = threadIdx.x; i < nb; i += 32) {
        fsum_merge(a, FSum{r[4 * i], r[4 * i + 1]});
        fsum_merge(b, FSum{r[4 * i + 2], r[4 * i + 3]});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fsum_merge(a, FSum{__shfl_down_sync(0xffffffffu, a.s, o), __shfl_down_sync(0xffffffffu, a.c, o)});
        fsum_merge(b, FSum{__shfl_down_sync(0xffffffffu, b.s, o), __shfl_down_sync(0xffffffffu, b.c, o)});
    }
    if (threadIdx.x == 0) {
        scal[slot_a] += (double)a.s + (double)a.c;
        scal[slot_b] += (double)b.s + (double)b.c;
    }
}

size_t pair_sums_scratch_floats() { return 4 * PS_BLOCKS; }

void launch_pair_sums(const float *part, size_t npairs, float *scratch, double *scal, int slot_a, int slot_b,
                      cudaStream_t st)
{
    counted(2);
    k_pair_sums<<<PS_BLOCKS, 256, 0, st>>>(part, npairs, scratch);
    k_pair_final<<<1, 32, 0, st>>>(scratch, PS_BLOCKS, scal, slot_a, slot_b);
}

}  // namespace ctpd
