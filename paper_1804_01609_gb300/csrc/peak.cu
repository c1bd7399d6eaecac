// FP64 FMA throughput of the device, the denominator of the stencil-solve roofline. The
// measured peak HBM copy and BF16 GEMM rates come from outside the library; GB300's FP64 rate
// is not among them, so it is measured here: every thread runs kChains independent chains of
// dependent FMAs (enough warps and chains in flight to keep every SM's FP64 units busy), and
// the rate is 2 x FMAs / time. No counterpart in the paper: a measurement utility.
#include "common.cuh"

namespace rbfsl {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma_rate_kernel(int64_t iters, double seed, double *sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (threadIdx.x + c) * 1e-7;
    const double m = 1.0 - 1e-12, d = 1e-13;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678) sink[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace rbfsl

extern "C" int rbfsl_fp64_fma_rate(int64_t iters, double *tflops, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(iters >= 1 && tflops, "fp64_fma_rate: bad arguments");
    int dev = 0, sms = 0;
    RBFSL_CUDA_TRY(cudaGetDevice(&dev));
    RBFSL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    double *sink = nullptr;
    RBFSL_CUDA_TRY(cudaMalloc(&sink, sizeof(double)));
    const unsigned blocks = (unsigned)(sms * 8);  // 8 blocks x 8 warps per SM
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_rate_kernel<<<blocks, 256, 0, s>>>(iters / 8 + 1, 1.0, sink);  // warm-up
    cudaEventRecord(e0, s);
    fma_rate_kernel<<<blocks, 256, 0, s>>>(iters, 1.0, sink);
    cudaEventRecord(e1, s);
    int rc = launch_status("fp64_fma_rate");
    float ms = 0.f;
    if (rc == RBFSL_OK) {
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = RBFSL_ECUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != RBFSL_OK) return rc;
    const double fmas = (double)blocks * 256.0 * (double)iters * kChains;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return RBFSL_OK;
}
