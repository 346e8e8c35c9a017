// probe.cu -- measurement of the device's FP64 fused multiply-add rate, the
// denominator of the FP64 path's roofline (the update is bound by the FP64
// pipe, not by HBM). Each thread runs 8 independent FMA chains so the pipe,
// not the dependency latency, limits the rate.
#include "hamr_internal.h"

namespace hamr {
namespace {

constexpr int CHAINS = 8;
constexpr int ITERS = 4096;

__global__ void k_fp64_fma(double* out, double a, double b) {
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += x[c];
    if (s == 123.456) out[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

cudaError_t measure_fp64_peak(cudaStream_t s, double* gflops) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double));
    if (e != cudaSuccess) return e;
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_fp64_fma<<<blocks, threads, 0, s>>>(out, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(a, s);
    const int reps = 5;
    for (int r = 0; r < reps; r++) k_fp64_fma<<<blocks, threads, 0, s>>>(out, 0.999999, 1e-7);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * CHAINS * (double)ITERS * threads * (double)blocks * reps;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return cudaGetLastError();
}

}  // namespace hamr
