// eps.cu -- the epsilon-constrained few-view form (Sec. 5):
//     min TV(x)  subject to  ||Ax - b|| <= eps,  x >= 0.
//
// The dual step of Algorithm 2 becomes a proximal map (the ball's support
// function replaces the linear h of Eq. 28): with q the equality form's
// update mu + sigma D (A x - b),
//     nu = argmin  sigma eps |nu| + 1/2 (nu - q)^T D^-1 (nu - q),
// whose optimality condition is (I + c D) nu = q with c = sigma eps / |nu|,
// or nu = 0 when |D^-1 q| <= sigma eps.  D acts on each view with one B x B
// symmetric Toeplitz matrix T = Q diag(lambda) Q^T, so in T's eigenbasis the
// map is diagonal: w = Q^T q per view, nu = Q diag(1 / (1 + c lambda)) w,
// and c solves the scalar equation c^2 sum_j W2_j / (1 + c lambda_j)^2 =
// (sigma eps)^2 with W2_j = sum_v w_vj^2.
//
// Q and lambda come from an FP64 eigendecomposition on the host (once per
// geometry and taps, cached by the caller); per iteration the device runs
// two B x B GEMMs over the views, one column reduction and a one-warp
// Newton solve for c.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ctpd_internal.cuh"

namespace ctpd {

// ---------------------------------------------------------------------
// Host: symmetric eigendecomposition (FP64)
// ---------------------------------------------------------------------
namespace {

// a (n x n, row-major, symmetric) = z diag(d) z^T; z's columns are the
// eigenvectors.  Householder reduction to tridiagonal form (the reflectors
// accumulated backwards into z), then implicit symmetric QR steps with the
// Wilkinson shift on the tridiagonal, each rotation also applied to z.
// Returns false if the QR steps do not converge.
bool sym_eig(std::vector<double> &a, int n, std::vector<double> &d, std::vector<double> &z)
{
    d.assign(n, 0.0);
    std::vector<double> e(std::max(n - 1, 1), 0.0);
    std::vector<std::vector<double>> refl(std::max(n - 2, 0));
    std::vector<double> p(n), w(n);
    auto A = [&](int i, int j) -> double & { return a[(size_t)i * n + j]; };
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;   // reflector acts on rows / columns k+1 .. n-1
        std::vector<double> &v = refl[k];
        v.assign(m, 0.0);
        double xn = 0.0;
        for (int i = 0; i < m; ++i) xn += A(k + 1 + i, k) * A(k + 1 + i, k);
        xn = sqrt(xn);
        if (xn == 0.0) {
            e[k] = 0.0;
            continue;
        }
        const double x0 = A(k + 1, k), alpha = x0 >= 0.0 ? -xn : xn;
        for (int i = 0; i < m; ++i) v[i] = A(k + 1 + i, k);
        v[0] -= alpha;
        double vn = 0.0;
        for (int i = 0; i < m; ++i) vn += v[i] * v[i];
        vn = sqrt(vn);
        for (int i = 0; i < m; ++i) v[i] /= vn;
        // A22 <- H A22 H, H = I - 2 v v^T:  p = A22 v, w = p - (v.p) v,
        // A22 -= 2 (v w^T + w v^T)
        double vp = 0.0;
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += A(k + 1 + i, k + 1 + j) * v[j];
            p[i] = s;
            vp += v[i] * s;
        }
        for (int i = 0; i < m; ++i) w[i] = p[i] - vp * v[i];
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) A(k + 1 + i, k + 1 + j) -= 2.0 * (v[i] * w[j] + w[i] * v[j]);
        e[k] = alpha;
    }
    for (int k = 0; k < n; ++k) d[k] = A(k, k);
    if (n >= 2) e[n - 2] = A(n - 1, n - 2);   // below the last reflector
    // z = H_0 H_1 ... H_{n-3}, accumulated from the last reflector
    z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) z[(size_t)i * n + i] = 1.0;
    for (int k = n - 3; k >= 0; --k) {
        const std::vector<double> &v = refl[k];
        if (v.empty()) continue;
        const int m = n - k - 1;
        for (int j = k + 1; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += v[i] * z[(size_t)(k + 1 + i) * n + j];
            for (int i = 0; i < m; ++i) z[(size_t)(k + 1 + i) * n + j] -= 2.0 * s * v[i];
        }
    }
    // implicit QR on (d, e), deflating from the bottom
    int hi = n - 1, guard = 0;
    while (hi > 0) {
        if (++guard > 60 * n + 100) return false;
        // deflate negligible off-diagonals
        if (fabs(e[hi - 1]) <= 1e-15 * (fabs(d[hi - 1]) + fabs(d[hi])) || e[hi - 1] == 0.0) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && !(fabs(e[lo - 1]) <= 1e-15 * (fabs(d[lo - 1]) + fabs(d[lo])))) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        // Wilkinson shift from the trailing 2 x 2
        const double dl = 0.5 * (d[hi - 1] - d[hi]), eh = e[hi - 1];
        const double mu = d[hi] - eh * eh / (dl + (dl >= 0.0 ? 1.0 : -1.0) * hypot(dl, eh));
        double x = d[lo] - mu, y = e[lo];
        for (int k = lo; k < hi; ++k) {
            const double r = hypot(x, y);
            const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : y / r;
            if (k > lo) e[k - 1] = r;
            const double a0 = d[k], b0 = e[k], c0 = d[k + 1];
            d[k] = c * c * a0 + 2.0 * c * s * b0 + s * s * c0;
            d[k + 1] = s * s * a0 - 2.0 * c * s * b0 + c * c * c0;
            e[k] = c * s * (c0 - a0) + (c * c - s * s) * b0;
            if (k + 1 < hi) {   // the bulge below the block's next off-diagonal
                y = s * e[k + 1];
                e[k + 1] *= c;
                x = e[k];
            }
            for (int i = 0; i < n; ++i) {
                const double zk = z[(size_t)i * n + k], zk1 = z[(size_t)i * n + k + 1];
                z[(size_t)i * n + k] = c * zk + s * zk1;
                z[(size_t)i * n + k + 1] = -s * zk + c * zk1;
            }
        }
    }
    return true;
}

}  // namespace

// T[i][j] = t[|i - j|] (n x n): T commutes with the exchange J, so its
// eigenvectors split into symmetric ones [u; (b); J u] and antisymmetric
// ones [u; (0); -J u], from two symmetric problems of half the size:
//   m = floor(n / 2), A = T[0:m, 0:m], (C J)[i][j] = T[i][n - 1 - j];
//   antisymmetric:  A - C J  (m x m);
//   symmetric:      A + C J  (n even) or [[A + C J, r2 c], [r2 c^T, t0]]
//                   (n odd, c = T[0:m, m], r2 = sqrt 2).
bool toeplitz_eig(const double *t, int n, double *q, double *lambda)
{
    if (n < 1) return false;
    const int m = n / 2, odd = n & 1, ms = m + odd;
    auto T = [&](int i, int j) { return t[i > j ? i - j : j - i]; };
    const double r2 = sqrt(2.0);
    std::vector<double> as((size_t)ms * ms), aa((size_t)m * m), ds, zs, da, za;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            as[(size_t)i * ms + j] = T(i, j) + T(i, n - 1 - j);
            aa[(size_t)i * m + j] = T(i, j) - T(i, n - 1 - j);
        }
    if (odd) {
        for (int i = 0; i < m; ++i) as[(size_t)i * ms + m] = as[(size_t)m * ms + i] = r2 * T(i, m);
        as[(size_t)m * ms + m] = T(m, m);
    }
    if (!sym_eig(as, ms, ds, zs)) return false;
    if (m > 0 && !sym_eig(aa, m, da, za)) return false;
    std::fill(q, q + (size_t)n * n, 0.0);
    const double h = 1.0 / r2;
    for (int k = 0; k < ms; ++k) {   // symmetric eigenvectors: columns 0 .. ms-1
        lambda[k] = ds[k];
        for (int i = 0; i < m; ++i) {
            const double u = zs[(size_t)i * ms + k] * h;
            q[(size_t)i * n + k] = u;
            q[(size_t)(n - 1 - i) * n + k] = u;
        }
        if (odd) q[(size_t)m * n + k] = zs[(size_t)m * ms + k];
    }
    for (int k = 0; k < m; ++k) {    // antisymmetric: columns ms .. n-1
        lambda[ms + k] = da[k];
        for (int i = 0; i < m; ++i) {
            const double u = za[(size_t)i * m + k] * h;
            q[(size_t)i * n + ms + k] = u;
            q[(size_t)(n - 1 - i) * n + ms + k] = -u;
        }
    }
    return true;
}

// ---------------------------------------------------------------------
// Device: the per-iteration map
// ---------------------------------------------------------------------
constexpr int EG_T = 32;    // output tile (views x columns) and K tile
constexpr int EG_KS = 8;    // most K chunks of the split GEMM
constexpr int EG_PF = 4;    // K tiles whose global loads are in flight together
constexpr int EPS_ROOT_T = 512;   // threads of the multiplier's solve

// K chunks: enough blocks for about two per SM (few views give few tiles)
int eps_ksplit(const Geometry *g)
{
    const int tiles = ((g->n_bins + EG_T - 1) / EG_T) * ((g->n_views + EG_T - 1) / EG_T);
    return std::max(1, std::min(EG_KS, (2 * g->n_sm + tiles - 1) / tiles));
}

size_t eps_partial_floats(const Geometry *g) { return (size_t)eps_ksplit(g) * g->n_views * g->n_bins; }

// part[z][v][c] = sum over k in chunk z of X[v][k] s_k Qop[k][c], Qop = Q
// (TRANS false) or Q^T; s = NULL: 1.  16 x 16 threads, 2 x 2 outputs each,
// K staged through shared memory in tiles of 32; blockIdx.z = K chunk.
template <bool TRANS>
__global__ void __launch_bounds__(256)
k_eps_gemm(const float *__restrict__ X, const float *__restrict__ Q, const float *__restrict__ s,
           float *__restrict__ part, int V, int B, int kchunk)
{
    __shared__ float xs[EG_T][EG_T + 1], qs[EG_T][EG_T + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int v0 = blockIdx.y * EG_T, c0 = blockIdx.x * EG_T;
    const int kb = blockIdx.z * kchunk, ke = min(B, kb + kchunk);
    float acc[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    // the K tiles of the chunk go through shared memory one at a time, but
    // the global loads of up to EG_PF of them are issued before the first
    // is stored, so that their L2 round trips overlap
    for (int kg = kb; kg < ke; kg += EG_PF * EG_T) {
        float xr[EG_PF][4], qr[EG_PF][4];
#pragma unroll
        for (int t = 0; t < EG_PF; ++t) {
            const int k0 = kg + t * EG_T;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = ty + 16 * (e >> 1), j = tx + 16 * (e & 1);
                const int v = v0 + i, k = k0 + j;
                xr[t][e] = (k0 < ke && v < V && k < ke) ? X[(size_t)v * B + k] * (s ? s[k] : 1.0f) : 0.0f;
                // the element qs[.][.] of this (i, j) below: Q[c][kk] read along kk (TRANS), Q[kk][c] along c
                if (TRANS) {
                    const int c = c0 + i, kk = k0 + j;
                    qr[t][e] = (k0 < ke && c < B && kk < ke) ? Q[(size_t)c * B + kk] : 0.0f;
                } else {
                    const int kk = k0 + i, c = c0 + j;
                    qr[t][e] = (k0 < ke && c < B && kk < ke) ? Q[(size_t)kk * B + c] : 0.0f;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < EG_PF; ++t) {
            if (kg + t * EG_T >= ke) break;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = ty + 16 * (e >> 1), j = tx + 16 * (e & 1);
                xs[i][j] = xr[t][e];
                // qs[kk][cc] = Qop[k0 + kk][c0 + cc]
                if (TRANS) qs[j][i] = qr[t][e];
                else qs[i][j] = qr[t][e];
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < EG_T; ++kk) {
                const float x0 = xs[ty][kk], x1 = xs[ty + 16][kk];
                const float q0 = qs[kk][tx], q1 = qs[kk][tx + 16];
                acc[0][0] = fmaf(x0, q0, acc[0][0]);
                acc[0][1] = fmaf(x0, q1, acc[0][1]);
                acc[1][0] = fmaf(x1, q0, acc[1][0]);
                acc[1][1] = fmaf(x1, q1, acc[1][1]);
            }
            __syncthreads();
        }
    }
    float *pz = part + (size_t)blockIdx.z * V * B;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int v = v0 + ty + 16 * a, c = c0 + tx + 16 * b;
            if (v < V && c < B) pz[(size_t)v * B + c] = acc[a][b];
        }
}

// after the first map: w[v][j] = sum_z part[z][v][j] (chunks in order) and
// w2[j] = sum_v w[v][j]^2 (views v = y, y + 8, ... per thread row y, then
// the eight rows in order); blocks of 32 columns x 8 view rows
__global__ void __launch_bounds__(256)
k_eps_sum_w2(const float *__restrict__ part, int ks, int V, int B, float *__restrict__ w, float *__restrict__ w2)
{
    __shared__ float r[8][33];
    const int cx = threadIdx.x, vy = threadIdx.y, j = blockIdx.x * 32 + cx;
    const size_t VB = (size_t)V * B;
    float a2 = 0.0f;
    if (j < B)
        for (int v = vy; v < V; v += 8) {
            float pz[EG_KS];
#pragma unroll
            for (int z = 0; z < EG_KS; ++z) pz[z] = z < ks ? part[z * VB + (size_t)v * B + j] : 0.0f;
            float a = 0.0f;
#pragma unroll
            for (int z = 0; z < EG_KS; ++z) a += pz[z];
            w[(size_t)v * B + j] = a;
            a2 = fmaf(a, a, a2);
        }
    r[vy][cx] = a2;
    __syncthreads();
    if (vy == 0 && j < B) {
        float t = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += r[k][cx];
        w2[j] = t;
    }
}

// after the second map: out = sum_z part[z] (chunks in order), out2 =
// 2 out - mu0
__global__ void k_eps_sum_out(const float *__restrict__ part, int ks, size_t n, float *__restrict__ out,
                              float *__restrict__ out2, const float *__restrict__ mu0)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float pz[EG_KS];
#pragma unroll
        for (int z = 0; z < EG_KS; ++z) pz[z] = z < ks ? part[z * n + i] : 0.0f;
        float a = 0.0f;
#pragma unroll
        for (int z = 0; z < EG_KS; ++z) a += pz[z];
        out[i] = a;
        if (out2) out2[i] = 2.0f * a - mu0[i];
    }
}

// out = X s (per column j; in place allowed), out2 = 2 out - mu0: the map
// when D = I
__global__ void k_eps_scale(const float *X, const float *__restrict__ s, float *out,
                            float *__restrict__ out2, const float *__restrict__ mu0, int V, int B)
{
    const size_t n = (size_t)V * B;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float v = X[i] * s[i % B];
        out[i] = v;
        if (out2) out2[i] = 2.0f * v - mu0[i];
    }
}

// w2[j] = sum_v W[v][j]^2 (views in order)
__global__ void k_eps_w2(const float *__restrict__ W, int V, int B, float *__restrict__ w2)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B) return;
    float a = 0.0f;
    for (int v = 0; v < V; ++v) {
        const float x = W[(size_t)v * B + j];
        a = fmaf(x, x, a);
    }
    w2[j] = a;
}

// One block; each evaluation of f and g is spread over its threads.  se = sigma eps.  With u = 1 / c the condition
// c |nu(c)| = se reads f(u) = sum_j W2_j / (u + l_j)^2 = se^2 (l_j =
// max(lambda_j, 0); lambda = NULL: 1), the secular equation of a
// trust-region step: f falls from f(0) (infinite when some l_j = 0 carries
// energy) to 0.  If f(0) <= se^2, nu = 0.  Otherwise u solves
// psi(u) = 1 / sqrt(f(u)) - 1 / se = 0; psi is concave and increasing, so
// Newton steps from a point where psi < 0 climb to the root without
// overshooting (Hebden; More and Sorensen).  The start is the last step's
// u when psi < 0 there, else u = 0 (or the smallest l_j > 0 / 1e6 when
// f(0) is infinite, halved until psi < 0).  Stops at |sqrt(f) - se| <=
// 2e-6 se, the FP32 map's own accuracy.  All FP32, the sums in a fixed
// order (a butterfly per warp, then the warps in order).  Writes s_j = u / (u + l_j) = 1 / (1 + c l_j), or 0; u is
// kept as a float in the double slot scal[S_EPSC].
__global__ void __launch_bounds__(EPS_ROOT_T)
k_eps_root(const float *__restrict__ w2g, const float *__restrict__ lambda, int B, double *scal,
           float eps, float *__restrict__ s)
{
    // W2 and l staged once (n_bins <= 4096); every evaluation is spread over
    // the whole block: each thread sums its terms, the warps' sums meet in
    // shared memory, and every thread adds the EPS_ROOT_T / 32 warp sums in
    // the same order, so all threads hold the same f, g and take the same
    // Newton steps
    __shared__ float w2[4096], ls[4096];
    __shared__ float red[2][EPS_ROOT_T / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < B; j += EPS_ROOT_T) {
        w2[j] = w2g[j];
        ls[j] = lambda ? fmaxf(lambda[j], 0.0f) : 1.0f;
    }
    __syncthreads();
    float *uslot = reinterpret_cast<float *>(scal + S_EPSC);
    const float se = fscal(scal, F_SIGMA) * eps, se2 = se * se;
    auto wsum = [](float v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    // block sums of two per-thread values, the same in every thread
    auto bsum2 = [&](float a, float b, float &sa, float &sb) {
        a = wsum(a);
        b = wsum(b);
        if (lane == 0) {
            red[0][warp] = a;
            red[1][warp] = b;
        }
        __syncthreads();
        sa = 0.0f;
        sb = 0.0f;
#pragma unroll
        for (int q = 0; q < EPS_ROOT_T / 32; ++q) {
            sa += red[0][q];
            sb += red[1][q];
        }
        __syncthreads();   // red is reused by the next sum
    };
    // f(u) and g(u) = sum_j W2_j / (u + l_j)^3
    auto eval = [&](float u, float &f, float &g) {
        float a = 0.0f, b = 0.0f;
        for (int j = tid; j < B; j += EPS_ROOT_T) {
            const float inv = __fdividef(1.0f, u + ls[j]), t = w2[j] * inv * inv;
            a += t;
            b = fmaf(t, inv, b);
        }
        bsum2(a, b, f, g);
    };
    float f0 = 0.0f, lmin = 3.0e38f, unbf = 0.0f;
    for (int j = tid; j < B; j += EPS_ROOT_T) {
        const float lj = ls[j], wj = w2[j];
        if (lj > 0.0f) {
            f0 += wj / (lj * lj);
            lmin = fminf(lmin, lj);
        } else if (wj > 0.0f) {
            unbf = 1.0f;
        }
    }
    float unbs;
    bsum2(f0, unbf, f0, unbs);
    const bool unb = unbs > 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    if (lane == 0) red[0][warp] = lmin;
    __syncthreads();
    lmin = 3.0e38f;
#pragma unroll
    for (int q = 0; q < EPS_ROOT_T / 32; ++q) lmin = fminf(lmin, red[0][q]);
    __syncthreads();
    float u = 0.0f;
    bool zero = false, all = false;
    if (!(se > 0.0f)) {
        all = true;   // c = 0: s = 1
    } else if (!unb && f0 <= se2) {
        zero = true;
    } else {
        float f, g;
        const float up = *uslot;
        if (up > 0.0f) {
            eval(up, f, g);
            if (f > se2) u = up;
        }
        if (u == 0.0f && unb) {
            u = (lmin < 3.0e38f ? lmin : 1.0f) * 1e-6f;
            for (int k = 0; k < 120 && u > 0.0f; ++k, u *= 0.5f) {
                eval(u, f, g);
                if (f > se2) break;
            }
        }
        for (int k = 0; k < 40; ++k) {
            eval(u, f, g);
            const float nrm = sqrtf(f);
            if (fabsf(nrm - se) <= 2e-6f * se || !(g > 0.0f)) break;
            // psi = 1/nrm - 1/se, psi' = g / nrm^3
            const float un = u - (1.0f / nrm - 1.0f / se) * nrm * nrm * nrm / g;
            u = un > 0.0f ? un : 0.5f * u;
        }
    }
    for (int j = tid; j < B; j += EPS_ROOT_T) s[j] = all ? 1.0f : zero ? 0.0f : __fdividef(u, u + ls[j]);
    __syncthreads();   // every thread has read the previous u
    if (tid == 0) *uslot = (zero || all) ? 0.0f : u;
}

void launch_eps_step(const Geometry *g, const float *q, float *out, float *out2, const float *mu0, const float *Q,
                     const float *lambda, double eps, double *scal, float *wbuf, float *s, float *w2, float *part,
                     cudaStream_t st)
{
    const int V = g->n_views, B = g->n_bins;
    const size_t n = (size_t)V * B;
    const unsigned eblocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
    if (Q) {
        const int ks = eps_ksplit(g), kchunk = ((B + ks - 1) / ks + EG_T - 1) / EG_T * EG_T;
        const dim3 tb(16, 16), grid((B + EG_T - 1) / EG_T, (V + EG_T - 1) / EG_T, ks);
        counted(5);
        k_eps_gemm<false><<<grid, tb, 0, st>>>(q, Q, nullptr, part, V, B, kchunk);
        k_eps_sum_w2<<<(B + 31) / 32, dim3(32, 8), 0, st>>>(part, ks, V, B, wbuf, w2);
        k_eps_root<<<1, EPS_ROOT_T, 0, st>>>(w2, lambda, B, scal, (float)eps, s);
        k_eps_gemm<true><<<grid, tb, 0, st>>>(wbuf, Q, s, part, V, B, kchunk);
        k_eps_sum_out<<<eblocks, 256, 0, st>>>(part, ks, n, out, out2, mu0);
    } else {
        counted(3);
        k_eps_w2<<<(B + 127) / 128, 128, 0, st>>>(q, V, B, w2);
        k_eps_root<<<1, EPS_ROOT_T, 0, st>>>(w2, nullptr, B, scal, (float)eps, s);
        k_eps_scale<<<eblocks, 256, 0, st>>>(q, s, out, out2, mu0, V, B);
    }
}

// ---------------------------------------------------------------------
// Per-geometry cache of D's eigenbasis, keyed by (precond, tau as given):
// the taps, and so T, depend only on those and the geometry.  Entries are
// never replaced, so a solve's kernels may still read one while another
// thread adds a new entry.
// ---------------------------------------------------------------------
namespace {

struct EpsEntry {
    int precond;
    double tau;
    float *q, *lambda;
};

struct EpsCache {
    std::mutex mu;
    std::vector<EpsEntry> entries;
};

}  // namespace

ct_status eps_basis(const Geometry *g, int precond, double tau_key, const float *taps, cudaStream_t st,
                    const float **q, const float **lambda)
{
    Geometry *gm = const_cast<Geometry *>(g);
    {
        static std::mutex create_mu;
        std::lock_guard<std::mutex> lock(create_mu);
        if (!gm->eps_cache) gm->eps_cache = new EpsCache();
    }
    EpsCache *c = static_cast<EpsCache *>(gm->eps_cache);
    std::lock_guard<std::mutex> lock(c->mu);
    for (const EpsEntry &e : c->entries)
        if (e.precond == precond && e.tau == tau_key) {
            *q = e.q;
            *lambda = e.lambda;
            return CT_OK;
        }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        set_error("ct_pdtv_solve: the first error-tolerant solve for this geometry, precond and tau computes D's "
                  "eigenbasis on the host and cannot run inside stream capture; run it once uncaptured");
        return CT_ERR_ARG;
    }
    const int B = g->n_bins;
    std::vector<float> ht(2 * (size_t)B - 1);
    cudaError_t err = cudaMemcpyAsync(ht.data(), taps, sizeof(float) * ht.size(), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) {
        set_error("ct_pdtv_solve: reading the taps: %s", cudaGetErrorString(err));
        return CT_ERR_CUDA;
    }
    std::vector<double> t(B), qd((size_t)B * B), ld(B);
    for (int k = 0; k < B; ++k) t[k] = ht[B - 1 + k];
    if (!toeplitz_eig(t.data(), B, qd.data(), ld.data())) {
        set_error("ct_pdtv_solve: the eigendecomposition of D did not converge");
        return CT_ERR_NONFINITE;
    }
    std::vector<float> qf(qd.begin(), qd.end()), lf(ld.begin(), ld.end());
    EpsEntry e{precond, tau_key, nullptr, nullptr};
    err = cudaMalloc((void **)&e.q, sizeof(float) * qf.size());
    if (err == cudaSuccess) err = cudaMalloc((void **)&e.lambda, sizeof(float) * lf.size());
    if (err == cudaSuccess) err = cudaMemcpy(e.q, qf.data(), sizeof(float) * qf.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(e.lambda, lf.data(), sizeof(float) * lf.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        if (e.q) cudaFree(e.q);
        if (e.lambda) cudaFree(e.lambda);
        cudaGetLastError();
        set_error("ct_pdtv_solve: storing D's eigenbasis: %s", cudaGetErrorString(err));
        return err == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA;
    }
    c->entries.push_back(e);
    *q = e.q;
    *lambda = e.lambda;
    return CT_OK;
}

bool eps_basis_ready(const Geometry *g, int precond, double tau_key)
{
    if (precond == 0) return true;   // D = I: no basis
    EpsCache *c = static_cast<EpsCache *>(g->eps_cache);
    if (!c) return false;
    std::lock_guard<std::mutex> lock(c->mu);
    for (const EpsEntry &e : c->entries)
        if (e.precond == precond && e.tau == tau_key) return true;
    return false;
}

void eps_cache_free(Geometry *g)
{
    EpsCache *c = static_cast<EpsCache *>(g->eps_cache);
    if (!c) return;
    for (const EpsEntry &e : c->entries) {
        cudaFree(e.q);
        cudaFree(e.lambda);
    }
    delete c;
    g->eps_cache = nullptr;
}

}  // namespace ctpd

extern "C" ct_status ct_sym_toeplitz_eig(const double *t, int n, double *q, double *lambda)
{
    ctpd::set_error("%s", "");
    if (!t || !q || !lambda || n < 1) {
        ctpd::set_error("ct_sym_toeplitz_eig: bad argument");
        return CT_ERR_ARG;
    }
    if (!ctpd::toeplitz_eig(t, n, q, lambda)) {
        ctpd::set_error("ct_sym_toeplitz_eig: the QR iteration did not converge");
        return CT_ERR_NONFINITE;
    }
    return CT_OK;
}
