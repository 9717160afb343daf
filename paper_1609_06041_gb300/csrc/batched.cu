// batched.cu -- ct_pdtv_solve_batched: many independent slices (their own
// geometry, data, mode and parameters) solved in one call.
//
// The call forks the caller's stream onto a pool of streams (one pool per
// device, created on first use and kept until exit) with events, hands the
// slices to the pool streams largest first, each to the stream with the
// least work so far (work ~ N^2 V (iterations + Lanczos steps)), and joins
// every pool stream back into the caller's stream.  The fork and join are stream-ordered event waits,
// so the whole call can be captured into one CUDA graph.  When every slice
// qualifies for the persistent form, the pool runs only the slices' setups
// and one persistent launch after the join runs all their iterations
// (persist.cu); otherwise the pool runs each slice's whole single-slice
// solve, so small slices that cannot fill the GPU alone run side by side.
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ctpd_internal.cuh"

namespace {

constexpr int POOL_STREAMS = 16;
constexpr int MAX_DEVICES = 64;

struct Pool {
    bool ready = false;
    cudaStream_t s[POOL_STREAMS];
    cudaEvent_t fork;
    cudaEvent_t join[POOL_STREAMS];
    // held from the fork record to the last join wait: a call's pool
    // streams then wait on its own fork record, and its stream on its own
    // join records, when several host threads call at once
    std::mutex mu;
};

std::mutex g_pool_mu;
Pool g_pools[MAX_DEVICES];

ct_status pool_for_current(Pool **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return CT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    Pool &p = g_pools[dev];
    if (!p.ready) {
        cudaError_t e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming);
        for (int i = 0; i < POOL_STREAMS && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return CT_ERR_CUDA;
        }
        p.ready = true;
    }
    *out = &p;
    return CT_OK;
}

}  // namespace

extern "C" ct_status ct_pdtv_solve_batched(int n, const ct_geometry *const *geoms, const float *const *b,
                                           const float *const *w, const ct_pdtv_params *params,
                                           float *const *x_out, void *const *workspaces,
                                           ct_pdtv_report *reports, void *stream)
{
    ctpd::set_error("%s", "");
    if (n < 0 || (n > 0 && (!geoms || !b || !params || !x_out || !workspaces))) {
        ctpd::set_error("ct_pdtv_solve_batched: bad argument");
        return CT_ERR_ARG;
    }
    if (n == 0) return CT_OK;
    for (int i = 0; i < n; ++i) {
        if (!geoms[i] || !b[i] || !x_out[i] || !workspaces[i] || params[i].resume ||
            (params[i].mode == CT_LOWDOSE && (!w || !w[i]))) {
            ctpd::set_error("ct_pdtv_solve_batched: slice %d: missing geometry, data, output or workspace "
                            "(or resume set)", i);
            return CT_ERR_ARG;
        }
    }
    Pool *pool = nullptr;
    if (pool_for_current(&pool) != CT_OK) {
        ctpd::set_error("ct_pdtv_solve_batched: cannot create the stream pool");
        return CT_ERR_CUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int used = n < POOL_STREAMS ? n : POOL_STREAMS;
    // the persistent form: every slice qualifies and shares the iteration count
    bool persistent = ctpd::batched_form() == CT_BATCH_AUTO;
    int dev = -1;
    cudaGetDevice(&dev);
    for (int i = 0; i < n && persistent; ++i)
        persistent = geoms[i]->device == dev && ctpd::persistent_slice_ok(geoms[i], &params[i], params[0].iters);
    std::vector<ct_pdtv_params> setup;
    if (persistent) {
        // the pool runs each slice's setup and Step 1 at k = 0 (no iteration)
        setup.assign(params, params + n);
        for (auto &p : setup) p.iters = 0;
    }
    std::unique_lock<std::mutex> lock(pool->mu);
    cudaEventRecord(pool->fork, st);
    for (int i = 0; i < used; ++i) cudaStreamWaitEvent(pool->s[i], pool->fork, 0);
    // largest first onto the least-loaded stream: the streams end close
    // together instead of the last large slices running alone
    std::vector<int> order(n), stream_of(n);
    std::vector<double> work(n), load(used, 0.0);
    for (int i = 0; i < n; ++i) {
        const ct_geometry *g = geoms[i];
        const int its = persistent ? 0 : params[i].iters;
        const int nlz = params[i].sigma > 0.0 ? 0 : (params[i].norm_iters > 0 ? params[i].norm_iters : 12);
        order[i] = i;
        work[i] = (double)g->n * g->n * g->n_views * (double)(its + nlz + 1);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    for (int i : order) {
        const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        stream_of[i] = j;
        load[j] += work[i];
    }
    ct_status result = CT_OK;
    for (int k = 0; k < n && result == CT_OK; ++k) {
        const int i = order[k];
        result = ctpd::pdtv_solve(geoms[i], b[i], w ? w[i] : nullptr, persistent ? &setup[i] : &params[i], x_out[i],
                                  workspaces[i], nullptr, pool->s[stream_of[i]], false);
        if (result != CT_OK) {
            char msg[400];
            snprintf(msg, sizeof(msg), "%s", ct_last_error());
            ctpd::set_error("ct_pdtv_solve_batched: slice %d: %s", i, msg);
        }
    }
    // join: the caller's stream waits for every pool stream that was used
    for (int i = 0; i < used; ++i) {
        cudaEventRecord(pool->join[i], pool->s[i]);
        cudaStreamWaitEvent(st, pool->join[i], 0);
    }
    lock.unlock();
    if (result != CT_OK) return result;
    // the iterations of every slice: one persistent launch on the caller's stream
    if (persistent) {
        result = ctpd::launch_persistent(n, geoms, b, params, x_out, workspaces, st);
        if (result != CT_OK) return result;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctpd::set_error("ct_pdtv_solve_batched: %s", cudaGetErrorString(e));
        return CT_ERR_CUDA;
    }
    if (reports) {
        // scalars of each slice, read back after the caller's stream completes
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            ctpd::set_error("ct_pdtv_solve_batched: %s", cudaGetErrorString(e));
            return CT_ERR_CUDA;
        }
        ct_status first = CT_OK;
        char msg[400] = "";
        for (int i = 0; i < n; ++i) {
            result = ctpd::read_report(workspaces[i], &reports[i]);
            if (result != CT_OK && first == CT_OK) {
                first = result;
                snprintf(msg, sizeof(msg), "slice %d: %s", i, ct_last_error());
            }
        }
        if (first != CT_OK) {
            ctpd::set_error("ct_pdtv_solve_batched: %s", msg);
            return first;
        }
    }
    return CT_OK;
}
