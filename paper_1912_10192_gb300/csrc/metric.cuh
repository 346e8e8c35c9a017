// metric.cuh -- the Kerr metric in Kerr-Schild coordinates carried to the
// internal coordinates x1 = log r, x2 = theta, x3 = phi (Liska et al. 2019,
// Sec. 2.2), evaluated analytically on the device; flat space in Cartesian
// coordinates as option 1, in the same spherical coordinates as option 2.
#pragma once
#include "grmhd.cuh"

namespace hamr {

struct FullMetric {
    double g[4][4];
    double gi[4][4];
    double gdet;
};

__device__ inline double mirror_theta(double th) {
    const double pi = 3.14159265358979323846;
    if (th < 0.0) return -th;
    if (th > pi) return 2.0 * pi - th;
    return th;
}

__device__ inline void metric_at(int metric, double a, double x1, double x2, FullMetric& M) {
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) M.g[m][n] = M.gi[m][n] = 0.0;
    if (metric == 1) {
        M.g[0][0] = M.gi[0][0] = -1.0;
        for (int i = 1; i < 4; i++) M.g[i][i] = M.gi[i][i] = 1.0;
        M.gdet = 1.0;
        return;
    }
    // metric 2: flat space in the same coordinates (mass 0, no spin)
    const double mass = (metric == 2) ? 0.0 : 1.0;
    if (metric == 2) a = 0.0;
    const double r = exp(x1);
    const double th = mirror_theta(x2);
    double sth, cth;
    sincos(th, &sth, &cth);
    const double s2 = sth * sth;
    const double r2 = r * r;
    const double sig = r2 + a * a * cth * cth;
    const double z = 2.0 * mass * r / sig;  // 2Mr / Sigma
    M.g[0][0] = z - 1.0;
    M.g[0][1] = M.g[1][0] = z * r;
    M.g[0][3] = M.g[3][0] = -z * a * s2;
    M.g[1][1] = (1.0 + z) * r2;
    M.g[1][3] = M.g[3][1] = -(1.0 + z) * a * s2 * r;
    M.g[2][2] = sig;
    M.g[3][3] = s2 * (sig + (1.0 + z) * a * a * s2);
    M.gi[0][0] = -(1.0 + z);
    M.gi[0][1] = M.gi[1][0] = z / r;
    M.gi[1][1] = (r2 - 2.0 * mass * r + a * a) / (sig * r2);
    M.gi[1][3] = M.gi[3][1] = a / (sig * r);
    M.gi[2][2] = 1.0 / sig;
    M.gi[3][3] = 1.0 / (sig * s2);
    M.gdet = r * sig * sth;
}


// the sparse table form of a full metric
__device__ inline void to_sparse(const FullMetric& M, Metric<double>& m) {
    m.g00 = M.g[0][0];
    m.g01 = M.g[0][1];
    m.g03 = M.g[0][3];
    m.g11 = M.g[1][1];
    m.g13 = M.g[1][3];
    m.g22 = M.g[2][2];
    m.g33 = M.g[3][3];
    m.c00 = M.gi[0][0];
    m.c01 = M.gi[0][1];
    m.c11 = M.gi[1][1];
    m.c13 = M.gi[1][3];
    m.c22 = M.gi[2][2];
    m.c33 = M.gi[3][3];
    m.gdet = M.gdet;
    m.alpha = 1.0 / sqrt(-M.gi[0][0]);
    m.ialpha = sqrt(-M.gi[0][0]);
    m.igdet = (M.gdet != 0.0) ? 1.0 / M.gdet : 0.0;
}

}  // namespace hamr
