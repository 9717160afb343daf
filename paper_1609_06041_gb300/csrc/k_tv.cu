// k_tv.cu -- prox of tau*g (Eq. 17): argmin_{x>=0} lam TV(x) + 1/2 ||x - z||^2
// by projected-gradient steps on the TV dual field p = (px, py), |p_j| <= 1:
//     x_l = max(0, z + lam div p),   p <- Pi(p + grad x_l / (8 lam)),
// then x = max(0, z + lam div p).  grad is the forward difference (zero
// across the last row/column), div = -grad^T.  lam = 0 gives max(0, z).
//
// Temporal blocking: one block owns a TV_T x TV_T tile and loads it with a
// halo of (steps + 1) pixels.  Each step invalidates one more ring of the
// halo, so after `steps` steps the tile interior holds exactly what a
// whole-image iteration would give, with no grid-wide synchronisation and
// one pass over global memory per call.  p is double-buffered (p_in ->
// p_out) because neighbouring blocks read the old p in their halos.
#include "ctpd_internal.cuh"

namespace ctpd {

constexpr int TV_T = 32;
constexpr int TV_MAX_STEPS = 24;   // S = 32 + 2*25 = 82: 4*82*82*4 B = 105 KB

int tv_max_steps() { return TV_MAX_STEPS; }

static size_t tv_smem(int steps)
{
    int S = TV_T + 2 * (steps + 1);
    return sizeof(float) * 4 * (size_t)S * S;
}

constexpr int TV_THREADS = 512;   // 32 x 16

__global__ void __launch_bounds__(TV_THREADS)
k_tv(const float *__restrict__ z, const float *__restrict__ p_in, float *__restrict__ p_out,
     float *__restrict__ x, int N, int steps, int final_,
     const double *__restrict__ scal)
{
    extern __shared__ float sm[];
    const int H = steps + 1;
    const int S = TV_T + 2 * H;
    float *sz = sm, *spx = sm + S * S, *spy = spx + S * S, *sx = spy + S * S;
    const int R0 = blockIdx.y * TV_T - H, C0 = blockIdx.x * TV_T - H;
    const size_t NN = (size_t)N * N;
    const float lam = (float)scal[S_LAMBDA];
    const float inv8 = (float)scal[S_INV8LAM];
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 16
    constexpr int TY = TV_THREADS / 32;

    for (int li = ty; li < S; li += TY) {
        const int rr = R0 + li;
        for (int lj = tx; lj < S; lj += 32) {
            const int cc = C0 + lj;
            const bool in = rr >= 0 && rr < N && cc >= 0 && cc < N;
            const size_t gi = (size_t)rr * N + cc;
            const int i = li * S + lj;
            sz[i] = in ? z[gi] : 0.0f;
            spx[i] = in ? p_in[gi] : 0.0f;
            spy[i] = in ? p_in[NN + gi] : 0.0f;
            sx[i] = 0.0f;
        }
    }
    __syncthreads();

    if (lam > 0.0f) {
        for (int it = 0; it < steps; ++it) {
            // x_l = max(0, z + lam div p) on rows/cols >= 1 of the region
            for (int li = 1 + ty; li < S; li += TY) {
                const int rr = R0 + li;
                for (int lj = 1 + tx; lj < S; lj += 32) {
                    const int cc = C0 + lj;
                    const int i = li * S + lj;
                    const float dvx = (cc < N - 1 ? spx[i] : 0.0f) - (cc > 0 ? spx[i - 1] : 0.0f);
                    const float dvy = (rr < N - 1 ? spy[i] : 0.0f) - (rr > 0 ? spy[i - S] : 0.0f);
                    sx[i] = fmaxf(0.0f, sz[i] + lam * (dvx + dvy));
                }
            }
            __syncthreads();
            // p <- Pi(p + grad x / (8 lam)) on rows/cols 1 .. S-2
            for (int li = 1 + ty; li < S - 1; li += TY) {
                const int rr = R0 + li;
                for (int lj = 1 + tx; lj < S - 1; lj += 32) {
                    const int cc = C0 + lj;
                    const int i = li * S + lj;
                    const float gx = (cc < N - 1) ? sx[i + 1] - sx[i] : 0.0f;
                    const float gy = (rr < N - 1) ? sx[i + S] - sx[i] : 0.0f;
                    const float qx = spx[i] + gx * inv8;
                    const float qy = spy[i] + gy * inv8;
                    // divide by max(1, |q|)
                    const float sc = fminf(1.0f, rsqrtf(fmaf(qx, qx, qy * qy)));
                    spx[i] = qx * sc;
                    spy[i] = qy * sc;
                }
            }
            __syncthreads();
        }
    }

    // write back the tile interior
    for (int li = H + ty; li < H + TV_T; li += TY) {
        const int rr = R0 + li;
        for (int lj = H + tx; lj < H + TV_T; lj += 32) {
            const int cc = C0 + lj;
            const int i = li * S + lj;
            if (rr < N && cc < N) {
                const size_t gi = (size_t)rr * N + cc;
                if (lam > 0.0f) {
                    p_out[gi] = spx[i];
                    p_out[NN + gi] = spy[i];
                }
                if (final_) {
                    const float dvx = (cc < N - 1 ? spx[i] : 0.0f) - (cc > 0 ? spx[i - 1] : 0.0f);
                    const float dvy = (rr < N - 1 ? spy[i] : 0.0f) - (rr > 0 ? spy[i - S] : 0.0f);
                    const float xv = fmaxf(0.0f, sz[i] + lam * (dvx + dvy));
                    x[gi] = xv;
                }
            }
        }
    }
}

void launch_tv(const float *z, const float *p_in, float *p_out, float *x,
               int n, int steps, int final_, const double *scal, cudaStream_t st)
{
    dim3 blk(32, TV_THREADS / 32), grd((n + TV_T - 1) / TV_T, (n + TV_T - 1) / TV_T);
    counted();
    k_tv<<<grd, blk, tv_smem(steps), st>>>(z, p_in, p_out, x, n, steps, final_, scal);
}

void kernel_attrs_tv()
{
    cudaFuncSetAttribute(k_tv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tv_smem(TV_MAX_STEPS));
}


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
    const float lam = (float)scal[S_LAMBDA], inv8 = (float)scal[S_INV8LAM];
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
        fmaxf(0.0f, tv_s(z + blockIdx.z * NN, px, py, r, c, N, (float)scal[S_LAMBDA]));
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
        const float lam = (float)scal[S_LAMBDA];
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
        const float lam = (float)scal[S_LAMBDA], inv8 = (float)scal[S_INV8LAM];
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
        const float lam = (float)scal[S_LAMBDA], inv8 = (float)scal[S_INV8LAM];
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
