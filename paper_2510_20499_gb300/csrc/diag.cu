// bp_fp64_rate: the device's FP64 fused multiply-add throughput, the denominator of the FP64
// pipe fraction the benchmark reports beside the HBM fraction (propagation spends one FP64
// multiply-add per nonzero of its activities).  Every thread runs eight independent chains of
// dependent FMAs, so the FP64 pipe, not latency, bounds the kernel.
#include "bp_host.h"

namespace gpubp {
namespace {

constexpr int kChains = 8;

__global__ void k_fp64_fma(double* out, int iters, double b, double c) {
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (threadIdx.x + i) * 1e-3;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == 12345.678) out[0] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace
}  // namespace gpubp

using namespace gpubp;

extern "C" int bp_fp64_rate(double* tflops, void* stream) {
    if (!tflops) {
        set_error("bp_fp64_rate: null argument");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    BP_CUDA_TRY(cudaGetDevice(&dev));
    BP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double* out = nullptr;
    BP_CUDA_TRY(cudaMallocAsync(&out, sizeof(double), s));
    cudaEvent_t e0, e1;
    BP_CUDA_TRY(cudaEventCreate(&e0));
    BP_CUDA_TRY(cudaEventCreate(&e1));
    k_fp64_fma<<<blocks, threads, 0, s>>>(out, 64, 1.0000001, 0.999999);   // warm-up
    float best = 0.0f;
    for (int rep = 0; rep < 5; ++rep) {
        BP_CUDA_TRY(cudaEventRecord(e0, s));
        k_fp64_fma<<<blocks, threads, 0, s>>>(out, iters, 1.0000001, 0.999999);
        BP_CUDA_TRY(cudaEventRecord(e1, s));
        BP_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        BP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep == 0 || ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BP_CUDA_TRY(cudaFreeAsync(out, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return BP_OK;
}
