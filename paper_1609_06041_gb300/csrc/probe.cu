// probe.cu -- measured FP32 FMA throughput of the device, the denominator of
// the roofline fraction reported for the FMA-carrying operators.  Not part
// of the paper's method: a fixed FMA-only kernel timed with CUDA events.
//
// Every thread runs 16 independent FMA chains (scalar fma.rn.f32, or eight
// packed fma.rn.f32x2 pairs), enough independent work per warp to keep the
// FMA pipes busy; the chains converge to c / (1 - b), so no value
// overflows or turns denormal, and the sum is stored only under a
// condition the values never meet, so no work is dropped.
#include "ctpd_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 16;

template <bool PACKED>
__global__ void __launch_bounds__(PROBE_THREADS)
k_fma_probe(float *sink, int iters, float b, float c)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = (float)(threadIdx.x & 7) * 1.0e-3f + (float)i;
    if constexpr (PACKED) {
        unsigned long long bb, cc, av[PROBE_CHAINS / 2];
        asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
        asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS / 2; ++i) asm("mov.b64 %0, {%1, %2};" : "=l"(av[i]) : "f"(a[2 * i]), "f"(a[2 * i + 1]));
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS / 2; ++i)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(av[i]) : "l"(bb), "l"(cc));
        }
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS / 2; ++i) asm("mov.b64 {%0, %1}, %2;" : "=f"(a[2 * i]), "=f"(a[2 * i + 1]) : "l"(av[i]));
    } else {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[i]) : "f"(b), "f"(c));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == -1.0f) sink[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;   // never true: chains stay positive
}

}  // namespace

extern "C" ct_status ct_probe_fp32_fma(int packed, double *tflops, void *stream)
{
    ctpd::set_error("%s", "");
    if (!tflops) {
        ctpd::set_error("ct_probe_fp32_fma: NULL output");
        return CT_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = sms * 8;   // 64 warps per SM
    const int iters = 4096;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sink, sizeof(float) * blocks * PROBE_THREADS, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        ctpd::counted();
        if (packed) k_fma_probe<true><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters, 0.999f, 1.0e-3f);
        else k_fma_probe<false><<<blocks, PROBE_THREADS, 0, st>>>(sink, iters, 0.999f, 1.0e-3f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best_ms == 0.0f || ms < best_ms)) best_ms = ms;   // rep 0 warms up
    }
    if (sink) cudaFreeAsync(sink, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || best_ms <= 0.0f) {
        cudaGetLastError();
        ctpd::set_error("ct_probe_fp32_fma: %s", cudaGetErrorString(e));
        return CT_ERR_CUDA;
    }
    const double flops = 2.0 * PROBE_CHAINS * (double)iters * blocks * PROBE_THREADS;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return CT_OK;
}
