// c2p.cu -- the standalone inversion entry point (Sec. 2.6): one thread per
// state, the metric evaluated analytically at each state's position.
#include "c2p.cuh"
#include "hamr_internal.h"
#include "metric.cuh"
#include "mlp.cuh"

namespace hamr {
namespace {

template <bool MLP>
__global__ void __launch_bounds__(128) k_con2prim(hamr_c2p_desc d, const uint8_t* __restrict__ img, int* err,
                                                  int64_t n, const double* __restrict__ U,
                                                  const double* __restrict__ B, const double* __restrict__ x1,
                                                  const double* __restrict__ x2, double* __restrict__ prim,
                                                  int32_t* __restrict__ status, int32_t* __restrict__ iters) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = s < n;
    if (!MLP && !active) return;
    Metric<double> m;
    double u[NCONS], bc[3], pr[NPRIM];
    if (active) {
        FullMetric M;
        metric_at(d.metric, d.a, x1[s], x2[s], M);
        to_sparse(M, m);
#pragma unroll
        for (int q = 0; q < NCONS; q++) u[q] = U[q * n + s];
#pragma unroll
        for (int q = 0; q < 3; q++) bc[q] = B[q * n + s];
#pragma unroll
        for (int q = 0; q < NPRIM; q++) pr[q] = prim[q * n + s];
        pr[B1] = bc[0];
        pr[B2] = bc[1];
        pr[B3] = bc[2];
    }
    const bool entropy_only = (d.flags & HAMR_C2P_ENTROPY_ONLY) != 0;
    const bool rescue = (d.flags & HAMR_C2P_MLP_RESCUE) != 0;
    C2PWork w;
    if (active)
        c2p_prepare(u, bc, m, d.gam, pr, w, (d.flags & HAMR_C2P_AITKEN) ? HAMR_INV_AITKEN : HAMR_INV_NEWTON,
                    (d.flags & HAMR_C2P_MIXED) ? 1 : 0);
    if (MLP && !entropy_only) {  // the 128 states of the CTA through the network (mlp.cuh)
        if (rescue && active) c2p_attempt_plain(w, d.gam);
        if (__syncthreads_or(active && !w.ok)) {
            extern __shared__ __align__(16) uint8_t mlp_smem[];
            MlpCta C;
            mlp_begin(C, mlp_smem, img);
            float f[MLP_NIN], y[MLP_NOUT];
            if (active) mlp_features(w.S, u[C_RHO], u[C_ENT], m, x1[s], d.gam, f);
            const bool ran = mlp_infer(C, f, active, y);
            mlp_end(C);
            if (!C.ok && threadIdx.x == 0 && err) atomicExch(err, 1);
            if (active && ran && !w.ok) {
                double g2[2];
                mlp_guess(w.S.D, y, g2);
                c2p_attempt(w, d.gam, g2[0], g2[1]);
            }
        }
    }
    if (!active) return;
    if (!entropy_only && !(MLP && rescue)) c2p_attempt_plain(w, d.gam);
    const int st = c2p_finish(w, u, m, d.gam, pr);
    const int it = w.its;
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
    const unsigned nb = (unsigned)((n + bs - 1) / bs);
    if ((d.flags & (HAMR_C2P_MLP | HAMR_C2P_MLP_RESCUE)) && d.mlp)
        k_con2prim<true><<<nb, bs, MLP_SMEM_BYTES, s>>>(d, mlp_image(d.mlp), mlp_error_ptr(d.mlp), n, U, B, x1, x2,
                                                        prim, status, iters);
    else
        k_con2prim<false><<<nb, bs, 0, s>>>(d, nullptr, nullptr, n, U, B, x1, x2, prim, status, iters);
    return cudaGetLastError();
}

}  // namespace hamr
