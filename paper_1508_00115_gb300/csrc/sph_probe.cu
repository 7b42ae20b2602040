// sph_probe.cu -- throughput probe of the plain FP32 pipes, the ceiling of the pair
// kernels (the density and force sums are not dense contractions, so their roofline
// is the FP32 FMA rate, not the tensor cores).
//
// Every thread runs kChains independent FMA recurrences a <- a * b + c for `iters`
// rounds: enough independent work per warp to cover the FMA latency, and enough
// resident warps per scheduler to keep the pipe busy; the loop is unrolled so that
// its control instructions take ~2 % of the issue slots.  The result is stored only if
// it equals a value it cannot take, so the arithmetic stays but nothing is written.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sph {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr int kChains = 16;

__device__ float g_probe_sink;

__global__ void __launch_bounds__(kProbeThreads) k_ffma(int iters, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.2345e-30f) g_probe_sink = s;
}

}  // namespace sph

extern "C" int sph_fp32_peak(void *cuda_stream, int32_t iters, int32_t reps, double *tflops_out, float *ms_out)
{
    using namespace sph;
    if (iters < 1 || reps < 1 || !tflops_out) return SPH_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return SPH_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = sms * kProbeBlocksPerSm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SPH_ERR_CUDA;
    }
    // b < 1 and c small keep the recurrences finite (they converge to c / (1 - b))
    const float b = 0.999999f, c = 1e-7f;
    k_ffma<<<blocks, kProbeThreads, 0, st>>>(iters, b, c);  // warm-up (clocks, code load)
    float best = 0.f;
    int rc = SPH_OK;
    for (int r = 0; r < reps && rc == SPH_OK; ++r) {
        float ms = 0.f;
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = SPH_ERR_CUDA;
        k_ffma<<<blocks, kProbeThreads, 0, st>>>(iters, b, c);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = SPH_ERR_CUDA;
        if (rc == SPH_OK && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kProbeThreads;
    *tflops_out = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return SPH_OK;
}
