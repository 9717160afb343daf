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

}  // namespace ctpd
