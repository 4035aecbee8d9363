// peak_fp64.cu -- measured FP64 fused multiply-add throughput of the current GPU: the ALU
// ceiling of the FP64 stencil, whose few flops per byte still exceed this part's FP64 rate
// per byte of HBM bandwidth.  Measurement support, not part of the sweep.
#include <cuda_runtime.h>

#include "../../include/mf.h"
#include "mf_internal.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma_rate(double *sink, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * c + 1e-9 * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) sink[0] = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" int mf_fp64_fma_rate(double *tflops, void *stream) {
    if (!tflops) return mfk::set_error(MF_EINVAL, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = mfk::sm_count() * 8;
    const int iters = 4096;
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
        cudaEventRecord(e0, s);
        k_dfma_rate<<<blocks, kThreads, 0, s>>>(sink, iters, 0.9999999, 1e-7);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return mfk::set_error(MF_ECUDA, cudaGetErrorString(e));
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return 0;
}
