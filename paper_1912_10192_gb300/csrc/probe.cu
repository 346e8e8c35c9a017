// probe.cu -- measurement of the device's FP64 fused multiply-add rate, the
// denominator of the FP64 path's roofline (the update is bound by the FP64
// pipe, not by HBM). Each thread runs 8 independent FMA chains so the pipe,
// not the dependency latency, limits the rate. Also the self-check of the
// integer-pipe binary32 <-> binary64 conversions (cvt.cuh) against the
// hardware ones.
#include "cvt.cuh"
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

// widening: every binary32 bit pattern, each thread a contiguous range of `per`
__global__ void k_check_widen(unsigned long long per, unsigned long long* bad, unsigned long long* first) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nbad = 0;
    for (unsigned long long q = t * per; q < (t + 1) * per && q < (1ull << 32); q++) {
        const float f = __uint_as_float((unsigned)q);
        const double w = widen(f), h = (double)f;
        const long long a = __double_as_longlong(w), b = __double_as_longlong(h);
        if (a != b && !(isnan(w) && isnan(h))) {  // NaN payloads are the implementation's
            if (nbad == 0) atomicCAS(first, ~0ull, q);
            nbad++;
        }
    }
    if (nbad) atomicAdd(bad, nbad);
}

// narrowing: around every binary32 value x (bit patterns q), the binary64 values x, x +- 1 and 2
// binary64 units, the midpoint to the next binary32 value and its binary64 neighbours (the ties and
// the values just beside them); plus `nrand` binary64 bit patterns from a splitmix64 sequence
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool narrow_differs(double x) {
    const float a = narrow(x), b = __double2float_rn(x);
    return __float_as_uint(a) != __float_as_uint(b) && !(isnan(a) && isnan(b));
}

__global__ void k_check_narrow(unsigned long long per, unsigned long long nrand, unsigned long long seed,
                               unsigned long long* bad, unsigned long long* first) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nbad = 0;
    auto check = [&](long long bits) {
        if (narrow_differs(__longlong_as_double(bits))) {
            if (nbad == 0) atomicCAS(first, ~0ull, (unsigned long long)bits);
            nbad++;
        }
    };
    for (unsigned long long q = t * per; q < (t + 1) * per && q < (1ull << 32); q++) {
        const float f = __uint_as_float((unsigned)q);
        const long long d = __double_as_longlong((double)f);
        for (int k = -2; k <= 2; k++) check(d + k);
        const long long mid = d + (1ll << 28);  // half a binary32 unit above x (same sign as x)
        for (int k = -1; k <= 1; k++) check(mid + k);
    }
    for (unsigned long long r = t; r < nrand; r += (unsigned long long)gridDim.x * blockDim.x)
        check((long long)mix64(seed + r));
    if (nbad) atomicAdd(bad, nbad);
}

}  // namespace

cudaError_t check_conversions(unsigned long long nrand, unsigned long long seed, unsigned long long out[4]) {
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    const unsigned long long init[4] = {0ull, ~0ull, 0ull, ~0ull};
    cudaMemcpy(d, init, sizeof(init), cudaMemcpyHostToDevice);
    const int threads = 256, blocks = 4096;
    const unsigned long long per = (1ull << 32) / ((unsigned long long)threads * blocks);
    k_check_widen<<<blocks, threads>>>(per, d, d + 1);
    k_check_narrow<<<blocks, threads>>>(per, nrand, seed, d + 2, d + 3);
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, d, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e;
}

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
