// FP64 throughput probe (declared in include/lbm.h): the ceilings of the
// step kernels that are bound by the FP64 pipe rather than by HBM - the ELBM
// root solve (FP64 in every storage format) and FP64 storage.  Measurement
// support only; the paper's method has no counterpart.
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kFmaIters = 4096;
constexpr int kLogIters = 256;

// kChains independent chains of fused multiply-adds, kFmaIters deep.
__global__ void __launch_bounds__(kProbeThreads) dfma_probe(double* sink, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-9 * (threadIdx.x + j);
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678) sink[0] = s;  // keeps the chains live
}

// Four independent log() evaluations per iteration on distinct arguments.
__global__ void __launch_bounds__(kProbeThreads) log_probe(double* sink, double step) {
    double x[4], acc = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = 1.0 + 1e-6 * (blockIdx.x * kProbeThreads + threadIdx.x) + 0.25 * j;
    for (int it = 0; it < kLogIters; ++it) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc += log(x[j]);
            x[j] += step;
        }
    }
    if (acc == 12345.678) sink[0] = acc;
}

}  // namespace

extern "C" lbm_status lbm_fp64_rates(double* dfma_flops, double* log_per_s, void* stream) {
    if (!dfma_flops && !log_per_s) return LBM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ERR_CUDA;
    const int blocks = nsm * 8;
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbm_status st = LBM_OK;
    if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = LBM_ERR_CUDA;
    float ms = 0.f;
    // each probe: one warm-up launch, then one timed launch
    if (st == LBM_OK && dfma_flops) {
        dfma_probe<<<blocks, kProbeThreads, 0, s>>>(sink, 0.999999, 1e-7);
        cudaEventRecord(e0, s);
        dfma_probe<<<blocks, kProbeThreads, 0, s>>>(sink, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            st = LBM_ERR_CUDA;
        else
            *dfma_flops = 2.0 * kChains * (double)kFmaIters * blocks * kProbeThreads / (ms * 1e-3);
    }
    if (st == LBM_OK && log_per_s) {
        log_probe<<<blocks, kProbeThreads, 0, s>>>(sink, 1e-7);
        cudaEventRecord(e0, s);
        log_probe<<<blocks, kProbeThreads, 0, s>>>(sink, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            st = LBM_ERR_CUDA;
        else
            *log_per_s = 4.0 * kLogIters * (double)blocks * kProbeThreads / (ms * 1e-3);
    }
    if (cudaGetLastError() != cudaSuccess) st = LBM_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}
