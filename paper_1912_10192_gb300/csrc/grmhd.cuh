// grmhd.cuh -- device-side ideal GRMHD physics of the block update.
//
// Liska et al., arXiv 1912.10192, Sec. 2. Everything here is per point and
// runs in registers; the kernels in step.cu and c2p.cu compose it.
//
// Metric layout. In Kerr-Schild coordinates (t, log r, theta, phi) the
// metric entries g_{t theta}, g_{r theta}, g_{theta phi} and, for the
// inverse, additionally g^{t phi} vanish identically (and so in flat
// Cartesian space). The tables therefore store 7 covariant and 6
// contravariant entries, and every contraction below skips the entries that
// are structurally zero.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hamr {

constexpr int NG = 3;
enum { RHO = 0, UU, U1, U2, U3, B1, B2, B3, NPRIM };
enum { C_RHO = 0, C_EN, C_S1, C_S2, C_S3, C_ENT, NCONS };
constexpr int NFLUX = 8;  // 6 cell-conserved slots + the two B^i with i != dir

// geometry table components (SoA over the padded (i, j) plane)
enum {
    G_00 = 0, G_01, G_03, G_11, G_13, G_22, G_33,  // covariant
    GI_00, GI_01, GI_11, GI_13, GI_22, GI_33,      // contravariant
    G_DET, G_ALPHA, NGEOM
};
// centre tables append: Christoffel symbols (40 = 4 upper x 10 symmetric lower)
// and the r-dependent floor values
constexpr int C_CONN = NGEOM;
constexpr int C_RHOFLR = NGEOM + 40;
constexpr int C_UFLR = NGEOM + 41;
constexpr int NGEOM_C = NGEOM + 42;

// status bits of a cell (OR over the two stages of a step)
enum : uint8_t { ST_ENTROPY = 1, ST_FAIL = 2, ST_FLOOR = 4 };

// index of the symmetric pair (m <= n) in 0..9
__host__ __device__ constexpr int sym(int m, int n) {
    return (m <= n) ? (m * 4 - (m * (m - 1)) / 2 + (n - m)) : (n * 4 - (n * (n - 1)) / 2 + (m - n));
}

template <typename T>
struct Metric {
    T g00, g01, g03, g11, g13, g22, g33;
    T c00, c01, c11, c13, c22, c33;
    T gdet, alpha;
};

template <typename T>
__device__ __forceinline__ void load_metric(const double* __restrict__ tab, long stride, long q, Metric<T>& m) {
    m.g00 = (T)tab[G_00 * stride + q];
    m.g01 = (T)tab[G_01 * stride + q];
    m.g03 = (T)tab[G_03 * stride + q];
    m.g11 = (T)tab[G_11 * stride + q];
    m.g13 = (T)tab[G_13 * stride + q];
    m.g22 = (T)tab[G_22 * stride + q];
    m.g33 = (T)tab[G_33 * stride + q];
    m.c00 = (T)tab[GI_00 * stride + q];
    m.c01 = (T)tab[GI_01 * stride + q];
    m.c11 = (T)tab[GI_11 * stride + q];
    m.c13 = (T)tab[GI_13 * stride + q];
    m.c22 = (T)tab[GI_22 * stride + q];
    m.c33 = (T)tab[GI_33 * stride + q];
    m.gdet = (T)tab[G_DET * stride + q];
    m.alpha = (T)tab[G_ALPHA * stride + q];
}

template <typename T>
__device__ __forceinline__ void lower4(const Metric<T>& m, const T v[4], T o[4]) {
    o[0] = m.g00 * v[0] + m.g01 * v[1] + m.g03 * v[3];
    o[1] = m.g01 * v[0] + m.g11 * v[1] + m.g13 * v[3];
    o[2] = m.g22 * v[2];
    o[3] = m.g03 * v[0] + m.g13 * v[1] + m.g33 * v[3];
}

template <typename T>
__device__ __forceinline__ T gcon0(const Metric<T>& m, int i) {  // g^{t i}
    return (i == 1) ? m.c01 : T(0);
}
template <typename T>
__device__ __forceinline__ T gcondd(const Metric<T>& m, int i) {  // g^{i i}
    return (i == 1) ? m.c11 : ((i == 2) ? m.c22 : m.c33);
}

template <typename T>
struct Fluid {
    T ucon[4], ucov[4], bcon[4], bcov[4];
    T bsq;
};

// u^mu from utilde^i (Lorentz factor wrt the normal observer
// Gamma = sqrt(1 + g_ij ut^i ut^j), u^t = Gamma/alpha, u^i = ut^i - Gamma alpha g^{ti});
// b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t (Sec. 2.3).
template <typename T>
__device__ __forceinline__ void fluid_state(const T pr[NPRIM], const Metric<T>& m, Fluid<T>& s) {
    const T q1 = pr[U1], q2 = pr[U2], q3 = pr[U3];
    T qsq = m.g11 * q1 * q1 + m.g22 * q2 * q2 + m.g33 * q3 * q3 + T(2) * m.g13 * q1 * q3;
    T gamma = sqrt(T(1) + qsq);
    s.ucon[0] = gamma / m.alpha;
    s.ucon[1] = q1 - gamma * m.alpha * m.c01;
    s.ucon[2] = q2;
    s.ucon[3] = q3;
    lower4(m, s.ucon, s.ucov);
    T bt = pr[B1] * s.ucov[1] + pr[B2] * s.ucov[2] + pr[B3] * s.ucov[3];
    T iut = m.alpha / gamma;
    s.bcon[0] = bt;
    s.bcon[1] = (pr[B1] + bt * s.ucon[1]) * iut;
    s.bcon[2] = (pr[B2] + bt * s.ucon[2]) * iut;
    s.bcon[3] = (pr[B3] + bt * s.ucon[3]) * iut;
    lower4(m, s.bcon, s.bcov);
    s.bsq = s.bcon[0] * s.bcov[0] + s.bcon[1] * s.bcov[1] + s.bcon[2] * s.bcov[2] + s.bcon[3] * s.bcov[3];
}

// Row `dir` of the conserved/flux vector (dir = 0: U, else F^dir), without sqrt(-g):
//   rho u^d, T^d_t + rho u^d, T^d_i, kappa rho u^d, and the B^i flux
//   b^i u^d - b^d u^i for the two i != dir (dir = 0: B^1, B^2 are not needed).
// T^mu_nu = (rho + u + p + b^2) u^mu u_nu + delta (p + b^2/2) - b^mu b_nu.
template <typename T>
__device__ __forceinline__ void flux_row(const T pr[NPRIM], const Fluid<T>& s, int d, int bdir, T gam, T kappa,
                                         T out[NFLUX]) {
    const T p = (gam - T(1)) * pr[UU];
    const T eta = pr[RHO] + pr[UU] + p + s.bsq;
    const T ptot = p + T(0.5) * s.bsq;
    const T eud = eta * s.ucon[d];
    const T bd = s.bcon[d];
    const T mass = pr[RHO] * s.ucon[d];
    out[0] = mass;
    out[1] = eud * s.ucov[0] - bd * s.bcov[0] + ((d == 0) ? ptot : T(0)) + mass;
    out[2] = eud * s.ucov[1] - bd * s.bcov[1] + ((d == 1) ? ptot : T(0));
    out[3] = eud * s.ucov[2] - bd * s.bcov[2] + ((d == 2) ? ptot : T(0));
    out[4] = eud * s.ucov[3] - bd * s.bcov[3] + ((d == 3) ? ptot : T(0));
    out[5] = kappa * mass;
    // transverse B slots of a bdir-face: i = first and second of {1,2,3} \ {bdir}
    const int i1 = (bdir == 1) ? 2 : 1;
    const int i2 = (bdir == 3) ? 2 : 3;
    out[6] = s.bcon[i1] * s.ucon[d] - bd * s.ucon[i1];
    out[7] = s.bcon[i2] * s.ucon[d] - bd * s.ucon[i2];
}

// entropy tracer kappa = p / rho^gam
template <typename T>
__device__ __forceinline__ T entropy_kappa(const T pr[NPRIM], T gam) {
    return (gam - T(1)) * pr[UU] / pow(pr[RHO], gam);
}

// fastest magnetosonic characteristic speeds along dir (Sec. 2.1): roots of
// A v^2 - 2 B v + C = 0 with c^2 = vA^2 + cs^2 (1 - vA^2).
template <typename T>
__device__ __forceinline__ void wave_speeds(const T pr[NPRIM], const Fluid<T>& s, const Metric<T>& m, int dir, T gam,
                                            T& vp, T& vm) {
    const T p = (gam - T(1)) * pr[UU];
    const T w = pr[RHO] + pr[UU] + p;
    const T cs2 = gam * p / w;
    const T va2 = s.bsq / (s.bsq + w);
    const T c2 = va2 + cs2 * (T(1) - va2);
    const T ut = s.ucon[0], ud = s.ucon[dir];
    const T A = ut * ut - c2 * (ut * ut + m.c00);
    const T B = ut * ud - c2 * (ut * ud + gcon0(m, dir));
    const T C = ud * ud - c2 * (ud * ud + gcondd(m, dir));
    T disc = B * B - A * C;
    disc = disc > T(0) ? disc : T(0);
    const T sd = sqrt(disc);
    const T iA = T(1) / A;
    vp = (B + sd) * iA;
    vm = (B - sd) * iA;
}

// ---- reconstruction (Sec. 2.1) ----

// monotonised central slope (Colella & Woodward 1984)
template <typename T>
__device__ __forceinline__ T mc_slope(T qm, T q0, T qp) {
    const T dl = q0 - qm, dr = qp - q0;
    if (dl * dr <= T(0)) return T(0);
    const T dc = T(0.5) * (qp - qm);
    T lim = fmin(T(2) * fabs(dl), T(2) * fabs(dr));
    T mag = fmin(fabs(dc), lim);
    return dc > T(0) ? mag : -mag;
}

template <typename T>
__device__ __forceinline__ T minmod_slope(T qm, T q0, T qp) {
    const T dl = q0 - qm, dr = qp - q0;
    if (dl * dr <= T(0)) return T(0);
    return fabs(dl) < fabs(dr) ? dl : dr;
}

// PPM edge values of the centre cell of the 5-point stencil q[0..4]:
// interface values from monotonised slopes, then the parabola constraints.
template <typename T>
__device__ __forceinline__ void ppm_cell(const T q[5], T& aL, T& aR) {
    const T s1 = mc_slope(q[0], q[1], q[2]);
    const T s2 = mc_slope(q[1], q[2], q[3]);
    const T s3 = mc_slope(q[2], q[3], q[4]);
    const T sixth = T(1.0 / 6.0);
    T l = T(0.5) * (q[1] + q[2]) - (s2 - s1) * sixth;
    T r = T(0.5) * (q[2] + q[3]) - (s3 - s2) * sixth;
    const T c = q[2];
    if ((r - c) * (c - l) <= T(0)) {
        l = c;
        r = c;
    } else {
        const T da = r - l;
        const T a6 = T(6) * (c - T(0.5) * (l + r));
        if (da * a6 > da * da)
            l = T(3) * c - T(2) * r;
        else if (-(da * da) > da * a6)
            r = T(3) * c - T(2) * l;
    }
    aL = l;
    aR = r;
}

}  // namespace hamr
