// geom.cu -- geometry tables of a block (Liska et al. 2019, Sec. 2.2).
//
// The Kerr metric is evaluated analytically in Kerr-Schild coordinates and
// carried to the internal coordinates x1 = log r, x2 = theta, x3 = phi with
// the exact Jacobian dr/dx1 = r. Christoffel symbols are finite differences
// of the internal-coordinate metric: 4th-order central differences with
// step h = 1e-3 in x1 and x2 (the metric does not depend on t or phi); the
// same derivatives are also stored themselves for the FP64 source term.
// Tables are 2-D over the padded (i, j) plane because the metric is
// stationary and axisymmetric; each component is one contiguous plane.
#include "grmhd.cuh"
#include "hamr_internal.h"
#include "metric.cuh"

namespace hamr {

namespace {

constexpr double CONN_H = 1.0e-3;

__device__ void store_metric(double* __restrict__ tab, long stride, long q, const FullMetric& M, bool pole) {
    tab[G_00 * stride + q] = M.g[0][0];
    tab[G_01 * stride + q] = M.g[0][1];
    tab[G_03 * stride + q] = M.g[0][3];
    tab[G_11 * stride + q] = M.g[1][1];
    tab[G_13 * stride + q] = M.g[1][3];
    tab[G_22 * stride + q] = M.g[2][2];
    tab[G_33 * stride + q] = M.g[3][3];
    tab[GI_00 * stride + q] = M.gi[0][0];
    tab[GI_01 * stride + q] = M.gi[0][1];
    tab[GI_11 * stride + q] = M.gi[1][1];
    tab[GI_13 * stride + q] = M.gi[1][3];
    tab[GI_22 * stride + q] = M.gi[2][2];
    tab[GI_33 * stride + q] = pole ? 0.0 : M.gi[3][3];
    tab[G_DET * stride + q] = pole ? 0.0 : M.gdet;
    tab[G_ALPHA * stride + q] = 1.0 / sqrt(-M.gi[0][0]);
    tab[G_IALPHA * stride + q] = sqrt(-M.gi[0][0]);
    tab[G_IGDET * stride + q] = pole ? 0.0 : 1.0 / M.gdet;
}

__global__ void k_geometry(GeomArgs A) {
    const long n2d = A.table_stride;
    const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long)A.n1p * A.n2p) return;
    const int i = (int)(q % A.n1p) - NG;
    const int j = (int)(q / A.n1p) - NG;
    const double x1c = A.x1min + (i + 0.5) * A.dx1, x2c = A.x2min + (j + 0.5) * A.dx2;
    const double x1f = A.x1min + i * A.dx1, x2f = A.x2min + j * A.dx2;
    FullMetric M;
    metric_at(A.metric, A.a, x1c, x2c, M);
    store_metric(A.centre, n2d, q, M, false);
    // Christoffel symbols at the centre
    double dg[3][4][4];  // d/dx1, d/dx2 (index 1, 2); index 0 unused
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) dg[0][m][n] = dg[1][m][n] = dg[2][m][n] = 0.0;
    if (A.metric != HAMR_METRIC_MINKOWSKI) {
        for (int s = 1; s <= 2; s++) {
            const double e1 = (s == 1) ? CONN_H : 0.0, e2 = (s == 2) ? CONN_H : 0.0;
            FullMetric p2, p1, m1, m2;
            metric_at(A.metric, A.a, x1c + 2.0 * e1, x2c + 2.0 * e2, p2);
            metric_at(A.metric, A.a, x1c + e1, x2c + e2, p1);
            metric_at(A.metric, A.a, x1c - e1, x2c - e2, m1);
            metric_at(A.metric, A.a, x1c - 2.0 * e1, x2c - 2.0 * e2, m2);
            for (int m = 0; m < 4; m++)
                for (int n = 0; n < 4; n++)
                    dg[s][m][n] = (8.0 * (p1.g[m][n] - m1.g[m][n]) - (p2.g[m][n] - m2.g[m][n])) / (12.0 * CONN_H);
        }
    }
    // Gamma^l_{mn} = 1/2 g^{lk} (d_m g_{kn} + d_n g_{km} - d_k g_{mn})
    for (int l = 0; l < 4; l++)
        for (int m = 0; m < 4; m++)
            for (int n = m; n < 4; n++) {
                double s = 0.0;
                for (int k = 0; k < 4; k++) {
                    const double dm = (m == 1 || m == 2) ? dg[m][k][n] : 0.0;
                    const double dn = (n == 1 || n == 2) ? dg[n][k][m] : 0.0;
                    const double dk = (k == 1 || k == 2) ? dg[k][m][n] : 0.0;
                    s += M.gi[l][k] * (dm + dn - dk);
                }
                A.centre[(C_CONN + l * 10 + sym(m, n)) * n2d + q] = 0.5 * s;
            }
    {
        const int pm[7] = {0, 0, 0, 1, 1, 2, 3}, pn[7] = {0, 1, 3, 1, 3, 2, 3};
        for (int s = 1; s <= 2; s++)
            for (int p = 0; p < 7; p++)
                A.centre[(C_DG + (s - 1) * 7 + p) * n2d + q] = (pm[p] == pn[p] ? 0.5 : 1.0) * dg[s][pm[p]][pn[p]];
    }
    const double r = (A.metric != HAMR_METRIC_MINKOWSKI) ? exp(x1c) : 1.0;
    A.centre[C_RHOFLR * n2d + q] = 1.0e-7 / (r * r);
    A.centre[C_UFLR * n2d + q] = 1.0e-9 * pow(r, -10.0 / 3.0);

    metric_at(A.metric, A.a, x1f, x2c, M);
    store_metric(A.face1, n2d, q, M, false);
    metric_at(A.metric, A.a, x1c, x2f, M);
    const bool pole = (A.pole_lo && j == 0) || (A.pole_hi && j == A.n2);
    store_metric(A.face2, n2d, q, M, pole);
}

}  // namespace

__global__ void k_table_f32(const double* __restrict__ src, float* __restrict__ dst, long n) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = (float)src[t];
}

cudaError_t launch_table_f32(const double* src, float* dst, int nplanes, long stride, cudaStream_t s) {
    const long n = (long)nplanes * stride;
    k_table_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_geometry(const GeomArgs& A, cudaStream_t s) {
    const long n2d = (long)A.n1p * A.n2p;  // threads: one per (i, j) point
    const int bs = 128;
    k_geometry<<<(unsigned)((n2d + bs - 1) / bs), bs, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace hamr
