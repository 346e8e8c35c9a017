// c2p.cu -- the standalone inversion entry point (Sec. 2.6): one thread per
// state, the metric evaluated analytically at each state's position.
#include "c2p.cuh"
#include "hamr_internal.h"
#include "metric.cuh"

namespace hamr {
namespace {

__global__ void k_con2prim(hamr_c2p_desc d, int64_t n, const double* __restrict__ U, const double* __restrict__ B,
                           const double* __restrict__ x1, const double* __restrict__ x2, double* __restrict__ prim,
                           int32_t* __restrict__ status, int32_t* __restrict__ iters) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    FullMetric M;
    metric_at(d.metric, d.a, x1[s], x2[s], M);
    Metric<double> m;
    to_sparse(M, m);
    double u[NCONS], bc[3], pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NCONS; q++) u[q] = U[q * n + s];
#pragma unroll
    for (int q = 0; q < 3; q++) bc[q] = B[q * n + s];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pr[q] = prim[q * n + s];
    pr[B1] = bc[0];
    pr[B2] = bc[1];
    pr[B3] = bc[2];
    int it = 0;
    const int st = invert(u, bc, m, d.gam, pr, &it, (d.flags & HAMR_C2P_ENTROPY_ONLY) != 0);
#pragma unroll
    for (int q = 0; q < NPRIM; q++) prim[q * n + s] = pr[q];
    status[s] = st;
    if (iters) iters[s] = it;
}

}  // namespace

cudaError_t launch_con2prim(const hamr_c2p_desc& d, int64_t n, const double* U, const double* B, const double* x1,
                            const double* x2, double* prim, int32_t* status, int32_t* iters, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int bs = 128;
    k_con2prim<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(d, n, U, B, x1, x2, prim, status, iters);
    return cudaGetLastError();
}

}  // namespace hamr
