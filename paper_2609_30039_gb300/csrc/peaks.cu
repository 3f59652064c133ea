// Arithmetic-rate probe for the FP64 roofline (instrumentation; the paper has no counterpart).
//
// The FP64 path of the Yee step moves 2x the FP32 bytes, but on this part its arithmetic rate
// may bind first: each cell-step issues ~25 FP64 instructions (adds, multiplies, fused
// multiply-adds) plus 12 per CPML slab membership.  The roof of that path is therefore
// min(HBM bandwidth / bytes, FP64 instruction rate / instructions); this probe measures the
// second rate with independent fused multiply-add chains that keep every FP64 pipe busy.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdtd.h"

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread (hide the pipe latency)
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = 1e-3 * (threadIdx.x + q);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = __fma_rn(x[q], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += x[q];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" fdtd_status fdtd_measure_fp64_rate(void* stream, double* fma_per_s, double* best_ms) {
    if (!fma_per_s || !best_ms) return FDTD_EINVAL;
    *fma_per_s = 0.0;
    *best_ms = 0.0;
    const cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fp64_fma, kProbeThreads, 0) != cudaSuccess)
        return FDTD_ECUDA;
    const int blocks = sms * (per > 0 ? per : 1);
    const int iters = 2048;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        return FDTD_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fdtd_status rc = FDTD_OK;
    float best = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FDTD_ECUDA;
    for (int rep = 0; rep < 6 && rc == FDTD_OK; ++rep) {   // the first run warms up
        cudaEventRecord(e0, st);
        k_fp64_fma<<<blocks, kProbeThreads, 0, st>>>(out, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = FDTD_ECUDA;
            break;
        }
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != FDTD_OK || best <= 0.f) return rc == FDTD_OK ? FDTD_ECUDA : rc;
    const double fmas = (double)blocks * kProbeThreads * (double)iters * kChains;
    *best_ms = best;
    *fma_per_s = fmas / (best * 1e-3);
    return FDTD_OK;
}
