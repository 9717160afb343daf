// body_tv.cuh -- body of the temporally blocked, register-resident TV prox
// (Eq. 17) shared by its kernel (k_tv.cu) and the persistent batched kernel
// (persist.cu).
#pragma once

#include "ctpd_internal.cuh"

namespace ctpd {

constexpr int TV_WARPS = 16;
constexpr int TV_THREADS = TV_WARPS * 32;
constexpr int TV_J = 5;                     // region rows per warp
constexpr int TV_ROWS = TV_WARPS * TV_J;    // 80
constexpr int TV_MAX_STEPS = 16;            // H = 17: 30 interior columns
constexpr int TV_MIN_TR = 16;               // fewest interior rows per tile


// Halo: steps + 1; the trajectory variant rounds it up to even, so that tile
// origins (and every lane's column pair) fall on even columns: with N even
// each pair of its many stores is one aligned 8-byte store.
__host__ __device__ __forceinline__ int tv_halo(int steps, bool even) { return even ? (steps + 2) & ~1 : steps + 1; }

// bz selects the image of a batch (z, x: N x N each; p: 2 N x N).
// traj, when not NULL, receives p after each of the first steps - 1 steps:
// step l + 1 (l = 0 .. steps - 2) at traj + (l * gz + image) * 2 N N.
//
// FGP: the fast gradient projection (Beck and Teboulle): each step is the
// projected-gradient step taken at r = p + theta (p - p_prev) instead of p,
// with theta_k = (t_k - 1) / t_{k+1}, t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
// (momentum restarted at every call).  Each cell keeps p_prev as well, and
// the field published for the divergence is r_y (p_y after the last step).
// Body of tile (bx, by) of image bz of a batch of gz images, on the
// TV_THREADS threads of context cb; J rows per warp (the region holds
// TV_WARPS J rows, TV_ROWS by default); pub_x and pub_y: (TV_WARPS J + 2) * 32
// float2 of shared memory each (row li of the region at index
// (li + 1) * 32 + lane; rows -1 and beyond the region read zeros).
template <bool FGP, bool TRAJ, class Ctx, int J = TV_J>
__device__ __forceinline__ void tv_body(const Ctx &cb, int bx, int by, int bz, int gz, float2 *pub_x, float2 *pub_y,
                                        const float *z, const float *p_in, float *p_out, float *x, int N,
                                        int steps, int final_, int tc, int tr, const double *scal, float *traj)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = cb.tid() & 31, w = cb.tid() >> 5;
    const int H = tv_halo(steps, TRAJ), Sr = tr + 2 * H;
    const bool vec2 = TRAJ && (N & 1) == 0;   // column pairs 8-byte aligned
    const int R0 = by * tr - H, C0 = bx * tc - H;
    const int c0 = C0 + 2 * lane;   // image columns c0, c0 + 1 of this lane
    const size_t NN = (size_t)N * N, img = bz;
    z += img * NN;
    p_in += img * 2 * NN;
    p_out += img * 2 * NN;
    if (final_) x += img * NN;
    const float lam = fscal(scal, F_LAMBDA);
    const float inv8 = fscal(scal, F_INV8LAM);
    // forward differences: along x on columns 0..N-2, along y on columns 0..N-1
    const bool cx0 = (unsigned)c0 < (unsigned)(N - 1), cx1 = (unsigned)(c0 + 1) < (unsigned)(N - 1);
    const bool cy0 = (unsigned)c0 < (unsigned)N, cy1 = (unsigned)(c0 + 1) < (unsigned)N;

    for (int i = cb.tid(); i < (TV_WARPS * J + 2) * 32; i += TV_THREADS) {
        pub_x[i] = make_float2(0.0f, 0.0f);
        pub_y[i] = make_float2(0.0f, 0.0f);
    }
    float zr[J][2], pxr[J][2], pyr[J][2], xr[J][2];
    float pxo[J][2], pyo[J][2];   // FGP: p of the previous step
    unsigned rowx = 0, rowy = 0;   // bit j: row in the image / row with a y difference
#pragma unroll
    for (int j = 0; j < J; ++j) {
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
    for (int j = 0; j < J; ++j) {
        pxo[j][0] = pxr[j][0];
        pxo[j][1] = pxr[j][1];
        pyo[j][0] = pyr[j][0];
        pyo[j][1] = pyr[j][1];
    }
    cb.sync();
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int li = w + TV_WARPS * j;
        if (li < Sr) pub_y[(li + 1) * 32 + lane] = make_float2(pyr[j][0], pyr[j][1]);
    }
    cb.sync();

    if (lam > 0.0f) {
        float t = 1.0f, th = 0.0f;   // FGP: t_k and theta_{k-1} (theta_0 = 0)
        for (int it = 0; it < steps; ++it) {
            // x = max(0, z + lam div r), r = p (GP) or p + theta (p - p_prev) (FGP)
#pragma unroll
            for (int j = 0; j < J; ++j) {
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
            cb.sync();
            // FGP: theta_k for the next extrapolation
            const float t1 = FGP ? 0.5f * (1.0f + sqrtf(fmaf(4.0f * t, t, 1.0f))) : 1.0f;
            const float thn = FGP ? (t - 1.0f) / t1 : 0.0f;
            const bool last = it + 1 == steps;
            // p = Pi(p + grad x / (8 lam)), Pi(q) = q / max(1, |q|)
#pragma unroll
            for (int j = 0; j < J; ++j) {
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
            if (TRAJ && !last) {   // the tile interior's p after this step
                float *tp = traj + ((size_t)it * gz + img) * 2 * NN;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int li = w + TV_WARPS * j, rr = R0 + li;
                    if (li >= H && li < H + tr && rr < N) {
                        if (vec2) {   // H, tc even: both columns of the pair are interior, or neither
                            const int lj = 2 * lane, cc = C0 + lj;
                            if (lj >= H && lj < H + tc && cc < N) {
                                const size_t gi = (size_t)rr * N + cc;
                                *reinterpret_cast<float2 *>(tp + gi) = make_float2(pxr[j][0], pxr[j][1]);
                                *reinterpret_cast<float2 *>(tp + NN + gi) = make_float2(pyr[j][0], pyr[j][1]);
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int lj = 2 * lane + e, cc = C0 + lj;
                                if (lj >= H && lj < H + tc && cc < N) {
                                    const size_t gi = (size_t)rr * N + cc;
                                    tp[gi] = pxr[j][e];
                                    tp[NN + gi] = pyr[j][e];
                                }
                            }
                        }
                    }
                }
            }
            cb.sync();
            t = t1;
            th = thn;
        }
    }

    // the tile interior: p, and x = max(0, z + lam div p) on the last chunk
#pragma unroll
    for (int j = 0; j < J; ++j) {
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

}  // namespace ctpd
