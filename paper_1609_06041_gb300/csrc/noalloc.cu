// noalloc.cu -- ct_ramp_filter_noalloc: the ramp filter without any device
// allocation, for callers that must not allocate (see include/ctpd.h).
//
// ct_ramp_filter needs a scratch buffer for the frequency response of the
// taps (n_fft complex values); it takes that buffer from the stream-ordered
// allocator.  This variant keeps the scratch in a file-scope device array
// instead, sized for the largest transform of the frequency-domain filter.
#include <mutex>

#include "ctpd_internal.cuh"

namespace {

// Frequency response of the taps.  Every GPU that loads the library holds
// this array (64 KiB) until the process exits.  All calls share it.
constexpr int NOALLOC_MAX_P = ctpd::FFT_MAX_P;
static __device__ __align__(256) float2 g_noalloc_hhat[NOALLOC_MAX_P];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
float2 *g_hhat_ptr[MAX_DEVICES] = {};

// Device address of g_noalloc_hhat on the current device, looked up once
// per device (host code only has a host-side stand-in for the symbol).
ct_status scratch_address(float2 **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return CT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_hhat_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_hhat);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return CT_ERR_CUDA;
        }
        g_hhat_ptr[dev] = static_cast<float2 *>(p);
    }
    *out = g_hhat_ptr[dev];
    return CT_OK;
}

}  // namespace

extern "C" ct_status ct_ramp_filter_noalloc(const ct_geometry *geom, const float *taps, int half_len,
                                            const float *in, float *out, int batch, void *stream)
{
    const ctpd::Geometry *g = geom;
    ctpd::set_error("%s", "");
    if (!g || half_len < 1 || half_len > g->n_bins || batch < 0 || batch > 65535) {
        ctpd::set_error("ct_ramp_filter_noalloc: bad argument");
        return CT_ERR_ARG;
    }
    if (g->n_fft > NOALLOC_MAX_P) {
        ctpd::set_error("ct_ramp_filter_noalloc: n_bins %d needs a %d-point transform; the allocation-free "
                        "filter supports at most %d points (n_bins <= %d)",
                        g->n_bins, g->n_fft, NOALLOC_MAX_P, NOALLOC_MAX_P / 2);
        return CT_ERR_ARG;
    }
    if (batch == 0) return CT_OK;
    if (!taps || !in || !out || in == out) {
        ctpd::set_error("ct_ramp_filter_noalloc: bad pointer");
        return CT_ERR_ARG;
    }
    // the scratch array's address and the geometry's twiddle table must
    // belong to the same GPU: the geometry's
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        ctpd::set_error("ct_ramp_filter_noalloc: cudaGetDevice failed");
        return CT_ERR_CUDA;
    }
    if (dev != g->device) {
        ctpd::set_error("ct_ramp_filter_noalloc: the current device is %d but the geometry lives on device %d",
                        dev, g->device);
        return CT_ERR_ARG;
    }
    float2 *hhat = nullptr;
    if (scratch_address(&hhat) != CT_OK) {
        ctpd::set_error("ct_ramp_filter_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return CT_ERR_CUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // k_hhat writes all n_fft entries, so the shared array needs no clearing
    ctpd::launch_hhat(g, taps, half_len, hhat, st);
    ctpd::launch_filter_fft(g, hhat, in, out, nullptr, nullptr, 0, nullptr, batch, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctpd::set_error("ct_ramp_filter_noalloc: %s", cudaGetErrorString(e));
        return CT_ERR_CUDA;
    }
    return CT_OK;
}
