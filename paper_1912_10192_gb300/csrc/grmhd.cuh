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

#include <type_traits>

#include "cvt.cuh"

namespace hamr {

constexpr int NG = 3;
enum { RHO = 0, UU, U1, U2, U3, B1, B2, B3, NPRIM };
enum { C_RHO = 0, C_EN, C_S1, C_S2, C_S3, C_ENT, NCONS };
constexpr int NFLUX = 8;  // 6 cell-conserved slots + the two B^i with i != dir

// geometry table components (SoA over the padded (i, j) plane)
enum {
    G_00 = 0, G_01, G_03, G_11, G_13, G_22, G_33,  // covariant
    GI_00, GI_01, GI_11, GI_13, GI_22, GI_33,      // contravariant
    G_DET, G_ALPHA, G_IALPHA, G_IGDET, NGEOM  // G_IALPHA: 1 / alpha; G_IGDET: 1 / sqrt(-g) (0 on the axis)
};
// centre tables append: Christoffel symbols (40 = 4 upper x 10 symmetric lower),
// the r-dependent floor values and the metric derivatives d_s g_{mn} (s = 1, 2; the
// 7 structurally non-zero (m, n) in the order of the covariant entries above), each
// times 1/2 on the diagonal and 1 off it: the weights of the symmetric contraction
// (1/2) T^{mn} d_s g_{mn} over m <= n
constexpr int C_CONN = NGEOM;
constexpr int C_RHOFLR = NGEOM + 40;
constexpr int C_UFLR = NGEOM + 41;
constexpr int C_DG = NGEOM + 42;
constexpr int NGEOM_C = NGEOM + 56;

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
    T gdet, alpha, ialpha, igdet;
};

template <typename T, typename TT>
__device__ __forceinline__ void load_metric(const TT* __restrict__ tab, long stride, long q, Metric<T>& m) {
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
    m.ialpha = (T)tab[G_IALPHA * stride + q];
    m.igdet = (T)tab[G_IGDET * stride + q];
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
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// The spatial covariant components need no lowering of u^mu: with u^mu = Gamma n^mu + (0, utilde^i)
// and n_i = 0, u_i = g_ij utilde^j; then g_ij utilde^i utilde^j = utilde^i u_i, and
// u_t = Gamma n_t + g_tj utilde^j = -alpha Gamma + g_t1 utilde^1 + g_t3 utilde^3.
template <typename T>
__device__ __forceinline__ void fluid_state(const T pr[NPRIM], const Metric<T>& m, Fluid<T>& s) {
    const T q1 = pr[U1], q2 = pr[U2], q3 = pr[U3];
    s.ucov[1] = m.g11 * q1 + m.g13 * q3;
    s.ucov[2] = m.g22 * q2;
    s.ucov[3] = m.g13 * q1 + m.g33 * q3;
    const T qsq = q1 * s.ucov[1] + q2 * s.ucov[2] + q3 * s.ucov[3];
    const T g2 = T(1) + qsq;
    const T ig = rsq(g2);  // 1 / Gamma
    const T gamma = g2 * ig;
    s.ucon[0] = gamma * m.ialpha;
    s.ucon[1] = q1 - gamma * m.alpha * m.c01;
    s.ucon[2] = q2;
    s.ucon[3] = q3;
    s.ucov[0] = m.g01 * q1 + m.g03 * q3 - m.alpha * gamma;
    T bt = pr[B1] * s.ucov[1] + pr[B2] * s.ucov[2] + pr[B3] * s.ucov[3];
    T iut = m.alpha * ig;
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

// x^y for finite x > 0 (FP64) as exp(y ln x):
//   ln x = e ln2 + ln m from x = 2^e m, m in [1/sqrt2, sqrt2), with
//   ln m = 2 atanh(t), t = (m - 1)/(m + 1), |t| <= 0.1716, by the odd power
//   series of atanh to t^23 (truncation < 1e-17);
//   exp(z) = 2^k exp(r), k = rint(z / ln2), |r| <= ln2/2, exp(r) by its Taylor
//   series to degree 14 (truncation < 3e-18).
// Relative error ~1e-14 (the rounding of z ~ y e ln2 dominates); other x take pow().
__device__ __forceinline__ double pow_pos(double x, double y) {
    const int hi = __double2hiint(x);
    const int bexp = (hi >> 20) & 0x7FF;
    if (x <= 0.0 || bexp == 0 || bexp == 0x7FF) return pow(x, y);  // zero, subnormal, inf, nan
    int e = bexp - 1023;
    double m = __hiloint2double((hi & 0x000FFFFF) | 0x3FF00000, __double2loint(x));  // [1, 2)
    if (m > 1.4142135623730951) {
        m *= 0.5;
        e += 1;
    }
    const double t = (m - 1.0) / (m + 1.0);
    const double t2 = t * t;
    double a = 1.0 / 23.0;
    a = fma(a, t2, 1.0 / 21.0);
    a = fma(a, t2, 1.0 / 19.0);
    a = fma(a, t2, 1.0 / 17.0);
    a = fma(a, t2, 1.0 / 15.0);
    a = fma(a, t2, 1.0 / 13.0);
    a = fma(a, t2, 1.0 / 11.0);
    a = fma(a, t2, 1.0 / 9.0);
    a = fma(a, t2, 1.0 / 7.0);
    a = fma(a, t2, 1.0 / 5.0);
    a = fma(a, t2, 1.0 / 3.0);
    a = fma(a, t2, 1.0);
    const double ln2 = 0.6931471805599453;
    const double z = y * fma((double)e, ln2, 2.0 * t * a);
    if (!(fabs(z) < 700.0)) return pow(x, y);
    const double k = rint(z * 1.4426950408889634);
    const double r = fma(-k, ln2, z);
    double b = 1.0 / 87178291200.0;  // 1/14!
    b = fma(b, r, 1.0 / 6227020800.0);
    b = fma(b, r, 1.0 / 479001600.0);
    b = fma(b, r, 1.0 / 39916800.0);
    b = fma(b, r, 1.0 / 3628800.0);
    b = fma(b, r, 1.0 / 362880.0);
    b = fma(b, r, 1.0 / 40320.0);
    b = fma(b, r, 1.0 / 5040.0);
    b = fma(b, r, 1.0 / 720.0);
    b = fma(b, r, 1.0 / 120.0);
    b = fma(b, r, 1.0 / 24.0);
    b = fma(b, r, 1.0 / 6.0);
    b = fma(b, r, 0.5);
    b = fma(b, r, 1.0);
    b = fma(b, r, 1.0);
    return b * __hiloint2double(((int)k + 1023) << 20, 0);
}
__device__ __forceinline__ float pow_pos(float x, float y) { return powf(x, y); }

// entropy tracer kappa = p / rho^gam
template <typename T>
__device__ __forceinline__ T entropy_kappa(const T pr[NPRIM], T gam) {
    return (gam - T(1)) * pr[UU] * pow_pos(pr[RHO], -gam);
}

// Bit patterns of FP64/FP32 values: sign tests, magnitude comparisons and
// maxima on the integer pipe (FP64 comparisons take the FP64 pipe).
template <typename T>
struct FBits;
template <>
struct FBits<double> {
    using I = long long;
    static constexpr I MAG = 0x7FFFFFFFFFFFFFFFll;
    static __device__ __forceinline__ I of(double x) { return __double_as_longlong(x); }
    static __device__ __forceinline__ double from(I i) { return __longlong_as_double(i); }
};
template <>
struct FBits<float> {
    using I = int;
    static constexpr I MAG = 0x7FFFFFFF;
    static __device__ __forceinline__ I of(float x) { return __float_as_int(x); }
    static __device__ __forceinline__ float from(I i) { return __int_as_float(i); }
};

// a non-NaN value as a signed integer of the same order (+0 and -0 both 0)
template <typename T>
__device__ __forceinline__ typename FBits<T>::I ordered_int(typename FBits<T>::I b) {
    const typename FBits<T>::I m = b & FBits<T>::MAG;
    return (b < 0) ? -m : m;
}

// max(a, b) of non-NaN values by their ordered bit patterns (ties give a); FP32 takes fmaxf, one
// instruction on the FP32 pipes
template <typename T>
__device__ __forceinline__ T max_i(T a, T b) {
    if constexpr (std::is_same<T, float>::value)
        return fmaxf(a, b);
    else
        return ordered_int<T>(FBits<T>::of(a)) >= ordered_int<T>(FBits<T>::of(b)) ? a : b;
}

// fastest magnetosonic characteristic speeds along dir (Sec. 2.1): roots of
// A v^2 - 2 B v + C = 0 with c^2 = vA^2 + cs^2 (1 - vA^2), vA^2 = b^2/(b^2 + w),
// cs^2 = gam p / w, i.e. c^2 = (b^2 + gam p)/(b^2 + w). The quadratic is taken
// times b^2 + w (same roots, no division for c^2): with num = b^2 + gam p and
// (b^2 + w)(1 - c^2) = w - gam p,
//   A = u^t u^t (w - gam p) - num g^{tt}, B = u^t u^d (w - gam p) - num g^{td},
//   C = u^d u^d (w - gam p) - num g^{dd}; v = (B +- sd)/A, sd = sqrt(max(0, B^2 - A C)).
// sqrt(max(x, 0)). FP64: x rsqrt(x) for x > 0 (the sign test on the integer pipe), which
// takes 6 FP64-pipe instructions where a correctly rounded sqrt takes 8 (counted with ncu on
// GB300), within 3e-16 of it; FP32 keeps sqrtf (not the FP64 pipe).
__device__ __forceinline__ double root_pos(double x) {
    return FBits<double>::of(x) > 0 ? x * rsqrt(x) : 0.0;
}
__device__ __forceinline__ float root_pos(float x) {
    return FBits<float>::of(x) > 0 ? sqrtf(x) : 0.0f;
}

template <typename T>
__device__ __forceinline__ void wave_quadratic(const T pr[NPRIM], const Fluid<T>& s, const Metric<T>& m, int dir,
                                               T gam, T& A, T& B, T& sd) {
    const T p = (gam - T(1)) * pr[UU];
    const T gp = gam * p;
    const T num = s.bsq + gp;
    const T dn = pr[RHO] + pr[UU] + p - gp;
    const T ut = s.ucon[0], ud = s.ucon[dir];
    A = ut * ut * dn - num * m.c00;
    B = ut * ud * dn - num * gcon0(m, dir);
    const T C = ud * ud * dn - num * gcondd(m, dir);
    const T disc = B * B - A * C;
    sd = root_pos(disc);
}

template <typename T>
__device__ __forceinline__ void wave_speeds(const T pr[NPRIM], const Fluid<T>& s, const Metric<T>& m, int dir, T gam,
                                            T& vp, T& vm) {
    T A, B, sd;
    wave_quadratic(pr, s, m, dir, gam, A, B, sd);
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

// The same limiters with their sign tests and magnitude comparisons done on the
// bit patterns (FBits above). dl dr <= 0 becomes "opposite signs or a zero";
// they differ from the products only where dl dr underflows.

// a b <= 0 (opposite signs or a zero)
template <typename T>
__device__ __forceinline__ bool nonpos_product(T a, T b) {
    using B = FBits<T>;
    const typename B::I ia = B::of(a), ib = B::of(b);
    return ((ia ^ ib) < 0) || (ia & B::MAG) == 0 || (ib & B::MAG) == 0;
}

// from the differences dl = q0 - qm, dr = qp - q0 and dlr = qp - qm
template <typename T>
__device__ __forceinline__ T mc_slope_d(T dl, T dr, T dlr) {
    if constexpr (std::is_same<T, float>::value) {
        // FP32: the FP32 pipes take the comparisons and products in one instruction each (the
        // bit-pattern forms pay off only where they replace FP64-pipe work)
        const float mag = fminf(fabsf(0.5f * dlr), 2.0f * fminf(fabsf(dl), fabsf(dr)));
        return (dl * dr > 0.0f) ? copysignf(mag, dlr) : 0.0f;
    } else {
        // FP64: the sign test, the magnitude comparisons, the halving and the doubling on the
        // integer pipe, bit-identical to the FP64 products for finite values: |x|/2 is one exponent
        // step down, or for |x| < 2^-1021 (the magnitude bits below 2^53, subnormal result) the bits
        // shifted right with the dropped bit rounded to even; 2|x| is one exponent step up, or for a
        // subnormal x (bits below 2^52) the bits shifted left
        using B = FBits<T>;
        using I = typename B::I;
        if (nonpos_product(dl, dr)) return T(0);
        const I al = B::of(dl) & B::MAG, ar = B::of(dr) & B::MAG;
        const I bl = B::of(dlr);
        const I ml = bl & B::MAG;
        const I ac = (ml >= (I(1) << 53)) ? ml - (I(1) << 52) : (ml >> 1) + (ml & (ml >> 1) & 1);  // |dlr|/2
        const I mn = al < ar ? al : ar;
        const I alim = (mn < (I(1) << 52)) ? (mn << 1) : mn + (I(1) << 52);                       // 2 min
        return B::from((ac < alim ? ac : alim) | (bl & ~B::MAG));
    }
}

template <typename T>
__device__ __forceinline__ T mc_slope_i(T qm, T q0, T qp) {
    return mc_slope_d(q0 - qm, qp - q0, qp - qm);
}

template <typename T>
__device__ __forceinline__ T minmod_slope_i(T qm, T q0, T qp) {
    using B = FBits<T>;
    const T dl = q0 - qm, dr = qp - q0;
    if (nonpos_product(dl, dr)) return T(0);
    return (B::of(dl) & B::MAG) < (B::of(dr) & B::MAG) ? dl : dr;
}

// the PPM interface value between cells with values qa, qb and slopes sa, sb
template <typename T>
__device__ __forceinline__ T ppm_face(T qa, T qb, T sa, T sb) {
    return T(0.5) * (qa + qb) - (sb - sa) * T(1.0 / 6.0);
}
// the same with d = qb - qa given: qa + d/2 - (sb - sa)/6
template <typename T>
__device__ __forceinline__ T ppm_face_d(T qa, T d, T sa, T sb) {
    return fma(T(0.5), d, qa) - (sb - sa) * T(1.0 / 6.0);
}

// the two parabola constraints of a cell with value c and edge values l, r.
// Every decision is a comparison of values, taken on the integer pipe:
// (r - c)(c - l) <= 0 is "c not strictly between l and r" (a rounded difference
// has the exact sign; as with nonpos_product, products that underflow aside);
// with da = r - l != 0 and s its sign, da a6 > da^2 is s a6 > |da| and
// -da^2 > da a6 is s a6 < -|da|. Near a tie the product form may take the
// other branch, which there gives the same edge value (the constraints are
// continuous across their switching surfaces).
template <typename T>
__device__ __forceinline__ void ppm_limit(T c, T& l, T& r) {
    using B = FBits<T>;
    using I = typename B::I;
    if constexpr (std::is_same<T, float>::value) {  // FP32: the product form on the FP32 pipes
        if ((r - c) * (c - l) <= 0.0f) {
            l = c;
            r = c;
            return;
        }
        const float da = r - l;
        const float a6 = 6.0f * (c - 0.5f * (l + r));
        const float daa6 = da * a6, da2 = da * da;
        if (daa6 > da2)
            l = 3.0f * c - 2.0f * r;
        else if (-da2 > daa6)
            r = 3.0f * c - 2.0f * l;
        return;
    }
    const I oc = ordered_int<T>(B::of(c)), ol = ordered_int<T>(B::of(l)), orr = ordered_int<T>(B::of(r));
    if (!((orr > oc && oc > ol) || (orr < oc && oc < ol))) {
        l = c;
        r = c;
    } else {
        const T da = r - l;
        const T a6 = T(6) * (c - T(0.5) * (l + r));
        const I bda = B::of(da);
        const I mda = bda & B::MAG;                                   // |da| (ordered, > 0)
        const I sa6 = ordered_int<T>(B::of(a6) ^ (bda & ~B::MAG));   // s a6 (ordered)
        if (sa6 > mda)
            l = T(3) * c - T(2) * r;
        else if (sa6 < -mda)
            r = T(3) * c - T(2) * l;
    }
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
