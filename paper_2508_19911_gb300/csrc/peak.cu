// Measured throughput of the SM's fused multiply-add pipes: the denominator
// of the roofline fractions reported for the ALU-bound kernels (the FP64
// flux and reconstruction, their FP32 counterparts in the mixed path).
// The paper has no counterpart; GB300's FP64 vector rate is far below its
// FP32 rate, and its nominal figure is confirmed here on the device itself.
//
// One launch of independent FMA chains: every thread carries kChains
// accumulators x_i <- x_i * a + b, so the pipe, not the dependency latency,
// bounds the kernel; the grid is a multiple of the SM count so that every
// SM does the same work. FLOP/s = 2 x FMAs / event-timed duration.
#include <cuda_runtime.h>

#include "common.cuh"
#include "gks.h"

namespace gks {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T *__restrict__ sink, int iters,
                                                             T a, T b) {
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x) * T(1e-3) + T(i);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    // a store the compiler cannot drop and that never happens at run time
    // for the constants the host passes (the chains stay near their start)
    if (s == T(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int sms, int iters, cudaStream_t s, T *sink, double *flops, double *ms_out) {
    const int blocks = sms * kBlocksPerSm;
    const T a = T(0.999999), b = T(1e-6);
    fma_chain_kernel<T><<<blocks, kThreads, 0, s>>>(sink, iters / 8, a, b);  // warm-up
    if (cudaGetLastError() != cudaSuccess) return GKS_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GKS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GKS_ERR_CUDA;
    }
    float best = 0.f;
    int rc = GKS_OK;
    for (int rep = 0; rep < 3 && rc == GKS_OK; ++rep) {
        cudaEventRecord(e0, s);
        fma_chain_kernel<T><<<blocks, kThreads, 0, s>>>(sink, iters, a, b);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = GKS_ERR_CUDA;
        float ms = 0.f;
        if (rc == GKS_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = GKS_ERR_CUDA;
        if (rc == GKS_OK && (rep == 0 || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GKS_OK) return rc;
    const double fmas = (double)blocks * kThreads * (double)iters * 16.0 * kChains;
    *flops = 2.0 * fmas / (best * 1e-3);
    *ms_out = best;
    return GKS_OK;
}

}  // namespace
}  // namespace gks

extern "C" int gks_fma_rate(int precision, void *cuda_stream, double *flops, double *ms) {
    if (!flops || !ms || (precision != GKS_PREC_FP64 && precision != GKS_PREC_MIXED))
        return GKS_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GKS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GKS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the sink is never written for the constants used (see the kernel);
    // it is a valid buffer of the grid's size all the same
    const size_t count = (size_t)sms * gks::kBlocksPerSm * gks::kThreads;
    void *sink = nullptr;
    if (cudaMalloc(&sink, count * sizeof(double)) != cudaSuccess) return GKS_ERR_NOMEM;
    // ~30 ms per launch at GB300's nominal rates (2 FP64 and 128 FP32 FMA
    // per clock per SM)
    const int rc = precision == GKS_PREC_FP64
                       ? gks::run<double>(sms, 1024, s, (double *)sink, flops, ms)
                       : gks::run<float>(sms, 1024 * 64, s, (float *)sink, flops, ms);
    cudaFree(sink);
    return rc;
}
