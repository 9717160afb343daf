// autotune.cu -- ct_geometry_autotune / ct_geometry_get_tuning /
// ct_geometry_set_tuning: launch shapes per geometry picked by measurement.
//
// Five shapes are tuned, each by timing every candidate on synthetic data
// of the geometry's size with CUDA events (one warm-up launch, then the mean
// of three):
//   - the projector's view items per block (k_project_quad: 64 threads per
//     view pair, pg pairs share one staged band pair), pg = 4 .. 16, jointly
//     with its steps per pass of a ray walk (2, or 4 with pg <= 12) and its
//     form (one band pair per block, or the work-balanced k_project_qbal
//     with 8, 12 or 16 items' threads per block);
//   - the backprojector's base-view slices (grid.z), 1 .. 8, for its
//     cluster form (k_backproject_orbit_cl: the slices' blocks add their
//     sums through distributed shared memory) and for its slice-image form
//     (one partial image per slice and k_orbit_reduce, taken by solves run
//     side by side and by the persistent batched kernel);
//   - the TV prox's fewest interior rows per tile (k_tv), 4 .. 64, which
//     sets how many tiles one image is cut into;
// and, with the work-balanced projector form, its unit ranges for one image
// balanced from measured block times (qbal_balance).
// Each choice changes only the launch shape and the order in which
// independent partial sums are formed, never the arithmetic of a sample.
#include <stdio.h>

#include "ctpd_internal.cuh"

using namespace ctpd;

namespace {

struct Buffers {
    void *p[8] = {};
    int n = 0;
    cudaError_t alloc(float **out, size_t floats)
    {
        cudaError_t e = cudaMalloc((void **)out, sizeof(float) * (floats ? floats : 1));
        if (e == cudaSuccess) p[n++] = *out;
        return e;
    }
    ~Buffers()
    {
        for (int i = 0; i < n; ++i) cudaFree(p[i]);
    }
};

// mean time of three launches of f after one warm-up, in ms (negative on error)
template <class F>
float time_launches(F f, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    f();
    cudaEventRecord(e0, st);
    for (int i = 0; i < 3; ++i) f();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    return cudaGetLastError() == cudaSuccess ? ms / 3.0f : -1.0f;
}

bool quad_path(const Geometry *g) { return g->vpair && g->n % 32 == 0 && g->n + 3 <= 640; }

}  // namespace

extern "C" ct_status ct_geometry_get_tuning(const ct_geometry *g, int *items_per_block, int *proj_rows,
                                            int *orbit_slices, int *tv_rows, int *proj_form)
{
    if (!g) {
        set_error("ct_geometry_get_tuning: NULL geometry");
        return CT_ERR_ARG;
    }
    if (items_per_block) *items_per_block = g->tune_pg;
    if (proj_rows) *proj_rows = g->tune_qrows;
    if (orbit_slices) *orbit_slices = g->tune_orb;
    if (tv_rows) *tv_rows = g->tune_tv;
    if (proj_form) *proj_form = g->tune_qbal;
    return CT_OK;
}

extern "C" ct_status ct_geometry_set_tuning(ct_geometry *g, int items_per_block, int proj_rows, int orbit_slices,
                                            int tv_rows, int proj_form)
{
    if (!g) {
        set_error("ct_geometry_set_tuning: NULL geometry");
        return CT_ERR_ARG;
    }
    if (proj_rows != 0 && proj_rows != 2 && proj_rows != 4) {
        set_error("ct_geometry_set_tuning: proj_rows must be 0, 2 or 4");
        return CT_ERR_ARG;
    }
    if (items_per_block != 0 && (items_per_block < 4 || items_per_block > (proj_rows == 4 ? 12 : 16))) {
        set_error("ct_geometry_set_tuning: items_per_block must be 0 or in [4, 16] ([4, 12] with proj_rows 4)");
        return CT_ERR_ARG;
    }
    if (orbit_slices != 0 && !orbit_slices_ok(g, orbit_slices)) {
        set_error("ct_geometry_set_tuning: orbit_slices must be 0 or in [1, 8] with at most 1024 base views "
                  "per slice");
        return CT_ERR_ARG;
    }
    if (tv_rows != 0 && (tv_rows < 4 || tv_rows > 64)) {
        set_error("ct_geometry_set_tuning: tv_rows must be 0 or in [4, 64]");
        return CT_ERR_ARG;
    }
    if (proj_form < 0 || proj_form > 2) {
        set_error("ct_geometry_set_tuning: proj_form must be 0, 1 or 2");
        return CT_ERR_ARG;
    }
    g->tune_pg = items_per_block;
    g->tune_qrows = proj_rows;
    g->tune_orb = g->tune_orb_si = orbit_slices;
    g->tune_tv = tv_rows;
    g->tune_qbal = proj_form;
    graph_cache_clear(g);
    return CT_OK;
}

extern "C" ct_status ct_geometry_autotune(ct_geometry *g, int batch, void *stream)
{
    set_error("%s", "");
    if (!g || batch < 1 || batch > 64) {
        set_error("ct_geometry_autotune: NULL geometry or batch outside [1, 64]");
        return CT_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int N = g->n;
    const size_t J = (size_t)N * N, I = (size_t)g->n_views * g->n_bins;
    const int old_pg = g->tune_pg, old_rows = g->tune_qrows, old_orb = g->tune_orb, old_tv = g->tune_tv;
    const int old_orb_si = g->tune_orb_si;
    const int old_qbal = g->tune_qbal;
    Buffers buf;
    float *x = nullptr, *sino = nullptr, *band = nullptr, *orb = nullptr, *img = nullptr, *tvb = nullptr;
    float *scalf = nullptr;
    cudaError_t e = buf.alloc(&x, J * batch);
    if (e == cudaSuccess) e = buf.alloc(&sino, I * batch);
    if (e == cudaSuccess) e = buf.alloc(&band, (size_t)proj_bands(N) * I * batch);
    if (e == cudaSuccess) e = buf.alloc(&orb, orbit_partial_floats(g, batch));
    if (e == cudaSuccess) e = buf.alloc(&img, J * batch);
    if (e == cudaSuccess) e = buf.alloc(&tvb, 6 * J);   // z, p_in (2J), p_out (2J), x
    if (e == cudaSuccess) e = buf.alloc(&scalf, 2 * (size_t)S_COUNT);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        set_error("ct_geometry_autotune: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA;
    }
    double *scal = reinterpret_cast<double *>(scalf);
    cudaMemsetAsync(scal, 0, sizeof(double) * S_COUNT, st);
    launch_scalars(scal, SC_SET, 1.0, 0, 0, S_TAU, st);
    launch_scalars(scal, SC_SET, 0.05, 0, 0, S_LAMBDA, st);
    launch_scalars(scal, SC_SET, 1.0 / (8.0 * 0.05), 0, 0, S_INV8LAM, st);
    launch_fill(x, 0.5f, J * batch, st);
    launch_fill(sino, 1.0f, I * batch, st);
    launch_fill(tvb, 0.0f, 6 * J, st);
    launch_fill(tvb, 0.5f, J, st);

    ct_status result = CT_OK;
    float t;
    if (quad_path(g)) {
        float best = -1.0f;
        int best_pg = 0, best_rows = 0, best_form = 1;
        for (int form = 1; form <= 2 && result == CT_OK; ++form) {
            for (int rows = 2; rows <= 4 && result == CT_OK; rows += 2) {
                for (int pg = form == 1 ? 4 : 8; pg <= (rows == 4 ? 12 : 16) && result == CT_OK;
                     pg += form == 1 ? 1 : 4) {
                    g->tune_pg = pg;
                    g->tune_qrows = rows;
                    g->tune_qbal = form;
                    t = time_launches([&] { launch_project_bands(g, x, band, batch, st); }, st, e0, e1);
                    if (t < 0.0f) result = CT_ERR_CUDA;
                    else if (best < 0.0f || t < best) {
                        best = t;
                        best_pg = pg;
                        best_rows = rows;
                        best_form = form;
                    }
                }
            }
        }
        g->tune_pg = best_pg;
        g->tune_qrows = best_rows;
        g->tune_qbal = best_form;
        // the balanced form's unit ranges for one image, from measured block times
        if (result == CT_OK) result = qbal_balance(g, x, band, st);
    }
    // the orbit backprojector's slices, for each of its two forms: slices
    // added in a thread-block cluster (single solves) and slice images with
    // a reduction pass (solves run side by side, the persistent kernel)
    for (int form = 0; form < 2 && result == CT_OK && orbit_ok(g); ++form) {
        const bool cl = form == 0;
        int &slot = cl ? g->tune_orb : g->tune_orb_si;
        float best = -1.0f;
        int best_sl = 0;
        for (int nsl = 1; nsl <= 8 && result == CT_OK; ++nsl) {
            if (!orbit_slices_ok(g, nsl)) continue;
            slot = nsl;
            t = time_launches([&] { launch_backproject_orbit(g, sino, img, 0, nullptr, scal, batch, orb, st, cl); },
                              st, e0, e1);
            if (t < 0.0f) result = CT_ERR_CUDA;
            else if (best < 0.0f || t < best) {
                best = t;
                best_sl = nsl;
            }
        }
        slot = best_sl;
    }
    if (result == CT_OK) {
        float best = -1.0f;
        int best_rows = 0;
        for (int rows = 4; rows <= 64 && result == CT_OK; rows *= 2) {
            t = time_launches([&] { launch_tv(tvb, tvb + J, tvb + 3 * J, tvb + 5 * J, N, g->n_sm, rows, 10, 1, scal,
                                              st); },
                              st, e0, e1);
            if (t < 0.0f) result = CT_ERR_CUDA;
            else if (best < 0.0f || t < best) {
                best = t;
                best_rows = rows;
            }
        }
        g->tune_tv = best_rows;
    }
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    graph_cache_clear(g);
    if (result != CT_OK) {
        g->tune_pg = old_pg;
        g->tune_qrows = old_rows;
        g->tune_orb = old_orb;
        g->tune_orb_si = old_orb_si;
        g->tune_tv = old_tv;
        g->tune_qbal = old_qbal;
        cudaError_t le = cudaGetLastError();
        set_error("ct_geometry_autotune: %s", cudaGetErrorString(le));
        return result;
    }
    return CT_OK;
}
