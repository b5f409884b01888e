// Throughput probes for the roofline denominators of the forward kernel,
// which is bound by the FP32 and MUFU (special-function) pipes rather than by
// HBM or the tensor cores.  Each probe runs independent dependency chains on
// every resident warp of every SM and counts operations per second.
#include <cuda_runtime.h>

#include "aem_internal.h"

namespace aem {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) fma32_probe(float *sink, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3f + c;
    const float m = 0.999999f, b = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) fma64_probe(double *sink, int iters) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3 + c;
    const double m = 0.999999, b = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.0) sink[0] = s;
}

// ex2 of a negated operand keeps every chain bounded in (0.5, 1].
__global__ void __launch_bounds__(kProbeThreads) mufu_probe(float *sink, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 0.5f + 0.01f * c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float v;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(-a[c]));
            a[c] = v;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.f) sink[0] = s;
}

// The forward recursion's special-function mix per layer-step: two rsqrt,
// one rcp, one ex2, one sin and one cos (their rates differ: ex2 issues at
// twice the rate of the others on this part).
__global__ void __launch_bounds__(kProbeThreads) mufu_mix_probe(float *sink, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 0.5f + 0.01f * c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float v = a[c], r;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(r));
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(-r));
            asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
            asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(r));
            a[c] = v;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.f) sink[0] = s;
}

template <class Kern, class... Args>
int time_kernel(Kern k, int grid, float *ms, Args... args) {
    cudaEvent_t e0, e1;
    AEM_CUDA_TRY(cudaEventCreate(&e0));
    AEM_CUDA_TRY(cudaEventCreate(&e1));
    k<<<grid, kProbeThreads>>>(args...);  // warm-up
    AEM_CUDA_TRY(cudaGetLastError());
    AEM_CUDA_TRY(cudaEventRecord(e0));
    k<<<grid, kProbeThreads>>>(args...);
    AEM_CUDA_TRY(cudaEventRecord(e1));
    AEM_CUDA_TRY(cudaEventSynchronize(e1));
    AEM_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return AEM_OK;
}

}  // namespace
}  // namespace aem

using namespace aem;

extern "C" int aem_probe_peaks(double *fp32_fma_per_s, double *mufu_per_s, double *fp64_fma_per_s,
                               double *mufu_mix_per_s) {
    int dev = 0, sms = 0;
    AEM_CUDA_TRY(cudaGetDevice(&dev));
    AEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * (2048 / kProbeThreads);
    const double threads = (double)grid * kProbeThreads;
    float *sink = nullptr;
    AEM_CUDA_TRY(cudaMalloc(&sink, 64));
    int rc = AEM_OK;
    float ms = 0.f;
    const int it32 = 1 << 14, itmufu = 1 << 11, it64 = 1 << 9;
    if ((rc = time_kernel(fma32_probe, grid, &ms, sink, it32))) goto done;
    if (fp32_fma_per_s) *fp32_fma_per_s = threads * it32 * kChains / (ms * 1e-3);
    if ((rc = time_kernel(mufu_probe, grid, &ms, sink, itmufu))) goto done;
    if (mufu_per_s) *mufu_per_s = threads * itmufu * kChains / (ms * 1e-3);
    if ((rc = time_kernel(fma64_probe, grid, &ms, (double *)sink, it64))) goto done;
    if (fp64_fma_per_s) *fp64_fma_per_s = threads * it64 * kChains / (ms * 1e-3);
    if ((rc = time_kernel(mufu_mix_probe, grid, &ms, sink, itmufu / 4))) goto done;
    if (mufu_mix_per_s) *mufu_mix_per_s = threads * (itmufu / 4) * kChains * 6.0 / (ms * 1e-3);
done:
    cudaFree(sink);
    return rc;
}
