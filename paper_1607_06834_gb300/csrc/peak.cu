// FP64 FMA throughput of the current device (roofline denominator of the
// FP64-ALU-bound stencil): independent DFMA chains in every thread of a grid
// of 8 CTAs per SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "rok.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void dfma_kernel(double *sink, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-9 + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) sink[threadIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace

extern "C" rok_status rok_fp64_fma_peak(double *tflops, int repeats)
{
    if (!tflops || repeats < 1) return ROK_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ROK_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ROK_ERR_CUDA;
    double *sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return ROK_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = 8 * sms, threads = 256;
    dfma_kernel<<<blocks, threads>>>(sink, 0.9999999, 1e-7);   // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < repeats; ++r) dfma_kernel<<<blocks, threads>>>(sink, 0.9999999, 1e-7);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || ms <= 0.f) return ROK_ERR_CUDA;
    const double flops = 2.0 * kChains * (double)kIters * blocks * threads * repeats;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return ROK_OK;
}
