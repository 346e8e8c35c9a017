// c2p.cuh -- conserved-to-primitive inversion (Liska et al. 2019, Sec. 2.6).
//
// Primary: 2-D Newton-Raphson on W = w Gamma^2 and v^2 = 1 - 1/Gamma^2 for
// the two scalar equations of the energy and the projected momentum in the
// normal-observer frame (the formulation of Noble et al. 2006). Backup when
// it fails: the entropy equation replaces the energy one, p = kappa rho^gam
// with kappa = U_kappa / U_rho, and a 1-D Newton in W solves the projected
// momentum equation (Noble et al. 2009). A state where both fail keeps its
// guess.
//
// Stopping rule: |dW|/W + |dv^2| < 1e-10 (quadratic convergence leaves the
// accepted iterate at round-off), at most 30 iterations; v^2 is kept
// in [0, 1 - 1/50^2].
#pragma once
#include "../../include/hamr.h"
#include "grmhd.cuh"

namespace hamr {

constexpr double C2P_TOL = 1.0e-10;
constexpr int C2P_NMAX = 30;
constexpr double C2P_VSQMAX = 1.0 - 1.0 / (50.0 * 50.0);

enum { INV_OK = 0, INV_ENTROPY = 1, INV_FAIL = 2 };

// The normal-frame scalars of a conserved state (Sec. 2.6, Noble et al. 2006).
struct C2PScalars {
    double D, Qdotn, Qtsq, Bsq, QdotB, QB2;
    double Qc1, Qc2, Qc3, Bn1, Bn2, Bn3;
};

// U: sqrt(-g) (rho u^t, T^t_t + rho u^t, T^t_i, kappa rho u^t); Bc: centre B^i.
__device__ __forceinline__ void c2p_scalars(const double U[NCONS], const double Bc[3], const Metric<double>& m,
                                            C2PScalars& S) {
    const double al = m.alpha;
    const double aig = al * m.igdet;  // alpha / sqrt(-g), formed once
    S.D = U[C_RHO] * aig;
    // Q_mu = alpha T^t_mu, raised with the sparse inverse metric
    const double Q0 = (U[C_EN] - U[C_RHO]) * aig;
    const double Q1 = U[C_S1] * aig;
    const double Q2 = U[C_S2] * aig;
    const double Q3 = U[C_S3] * aig;
    const double Qc0 = m.c00 * Q0 + m.c01 * Q1;
    S.Qc1 = m.c01 * Q0 + m.c11 * Q1 + m.c13 * Q3;
    S.Qc2 = m.c22 * Q2;
    S.Qc3 = m.c13 * Q1 + m.c33 * Q3;
    S.Bn1 = al * Bc[0];
    S.Bn2 = al * Bc[1];
    S.Bn3 = al * Bc[2];
    S.Qdotn = -al * Qc0;
    S.Qtsq = Q0 * Qc0 + Q1 * S.Qc1 + Q2 * S.Qc2 + Q3 * S.Qc3 + S.Qdotn * S.Qdotn;
    S.Bsq = m.g11 * S.Bn1 * S.Bn1 + m.g22 * S.Bn2 * S.Bn2 + m.g33 * S.Bn3 * S.Bn3 + 2.0 * m.g13 * S.Bn1 * S.Bn3;
    S.QdotB = Q1 * S.Bn1 + Q2 * S.Bn2 + Q3 * S.Bn3;
    S.QB2 = S.QdotB * S.QdotB;
}

// 2-D Newton on (W, v^2) from the given start; true when it met the
// stopping rule. `it` returns the iterations taken.
__device__ __forceinline__ bool newton_wv(const C2PScalars& S, double gfac, double& W, double& vsq, int& it) {
    const double D = S.D, Bsq = S.Bsq, QB2 = S.QB2, Qdotn = S.Qdotn, Qtsq = S.Qtsq;
    bool ok = false;
    for (it = 1; it <= C2P_NMAX; it++) {
        const double omv = 1.0 - vsq;
        const double rs = rsqrt(omv);
        const double sq = omv * rs;
        const double W2 = W * W, W3 = W2 * W;
        const double BW = Bsq + W;
        const double p = gfac * (W * omv - D * sq);
        // the residuals f1, f2 times W^2 and the Jacobian's first column (d/dW) times W^3, so that no
        // 1/W is formed: with det' = det W^3 the Newton step is dW = W (j12 f2' - j22 f1') / det',
        // dv = (j21' f1' - j11' f2') / (W^2 det'), both from the one reciprocal of W^2 det'
        const double f1 = (-0.5 * Bsq * (1.0 + vsq) - W + p - Qdotn) * W2 + 0.5 * QB2;
        const double f2 = (vsq * BW * BW - Qtsq) * W2 - QB2 * (Bsq + 2.0 * W);
        const double j11 = (gfac * omv - 1.0) * W3 - QB2;
        const double j12 = -0.5 * Bsq + gfac * (0.5 * D * rs - W);
        const double j21 = 2.0 * BW * (vsq * W3 + QB2);
        const double j22 = BW * BW;
        const double r = 1.0 / ((j11 * j22 - j12 * j21) * W2);
        const double dW = (j12 * f2 - j22 * f1) * W3 * r;
        const double dv = (j21 * f1 - j11 * f2) * r;
        const double Wn = W + dW;
        const double vn = fmin(fmax(vsq + dv, 0.0), C2P_VSQMAX);
        if (!(Wn > 0.0)) break;
        const double err = fabs(Wn - W) + fabs(vn - vsq) * Wn;
        W = Wn;
        vsq = vn;
        if (err < C2P_TOL * Wn) {
            ok = true;
            break;
        }
    }
    if (it > C2P_NMAX) it = C2P_NMAX;
    return ok;
}

// Mixed precision (the FP32-flux form only): FP32 Newton iterations first, on
// the two equations scaled by k = 2^-e, e the binary exponent of the start's W
// (an exact scaling; every term then O(1): f1 ~ W, f2 ~ W^2, so D, B^2, Q.n
// scale by k, Qt^2 by k^2, (Q.B)^2 by k^3), until a step is below 1e-5 W (at
// most 8). Then one refinement step in the manner of mixed-precision iterative
// refinement: the FP64 residuals at the FP32 root, solved with the FP32
// Jacobian there; it shrinks the root's error (~1e-7 W) by the Jacobian's
// relative error times its condition, to the FP64 level. It is accepted when
// the step is below 1e-5 W and that bound times the Jacobian's cancellation
// (|j11 j22| + |j12 j21|) / |det| stays below 1e-3 W (the remaining error of
// order 1e-10 W, the FP64 rule's); otherwise FP64 Newton iterations run from
// the refined point, stopping at the usual rule. When the FP32 stage does not
// converge the FP64 iteration runs from the original start alone. `it` counts
// the iterations of both precisions (the refinement as one).
__device__ __forceinline__ bool newton_wv_mixed(const C2PScalars& S, double gfac, double& W, double& vsq, int& it) {
    // the scalars rounded to FP32 first and scaled there (their magnitudes stay far inside FP32's
    // range for admissible states; a start outside the normal FP32 range takes the FP64 iteration)
    const float Wf = narrow(W);
    const unsigned eb = (__float_as_uint(Wf) >> 23) & 0xffu;  // biased exponent of the start
    if (!(Wf > 0.0f) || eb == 0u || eb >= 254u) {
        const bool ok = newton_wv(S, gfac, W, vsq, it);
        return ok;
    }
    const float k = __uint_as_float((254u - eb) << 23);  // 2^(127 - eb): w = W k in [1, 2)
    const float k2 = k * k;
    const float D = narrow(S.D) * k, Bsq = narrow(S.Bsq) * k, Qdotn = narrow(S.Qdotn) * k;
    const float Qtsq = narrow(S.Qtsq) * k2, QB2 = narrow(S.QB2) * (k2 * k);
    const float gf = narrow(gfac), vmax = (float)C2P_VSQMAX;
    float w = Wf * k, v = narrow(vsq);
    bool ok32 = false;
    int it32 = 0;
    for (it32 = 1; it32 <= 8; it32++) {
        const float omv = 1.0f - v;
        const float rs = rsqrtf(omv);
        const float sq = omv * rs;
        const float iw = 1.0f / w;
        const float iw2 = iw * iw;
        const float bw = Bsq + w;
        const float p = gf * (w * omv - D * sq);
        const float f1 = -0.5f * Bsq * (1.0f + v) + 0.5f * QB2 * iw2 - w + p - Qdotn;
        const float f2 = v * bw * bw - QB2 * (Bsq + 2.0f * w) * iw2 - Qtsq;
        const float j11 = -QB2 * iw2 * iw - 1.0f + gf * omv;
        const float j12 = -0.5f * Bsq + gf * (0.5f * D * rs - w);
        const float j21 = 2.0f * bw * (v + QB2 * iw2 * iw);
        const float j22 = bw * bw;
        const float idet = 1.0f / (j11 * j22 - j12 * j21);
        const float wn = w + (j12 * f2 - j22 * f1) * idet;
        const float vn = fminf(fmaxf(v + (j21 * f1 - j11 * f2) * idet, 0.0f), vmax);
        if (!(wn > 0.0f) || !(wn < 1e30f)) break;
        const float err = fabsf(wn - w) + fabsf(vn - v) * wn;
        w = wn;
        v = vn;
        if (err < 1e-5f * wn) {
            ok32 = true;
            break;
        }
    }
    if (it32 > 8) it32 = 8;
    if (!ok32) {  // the FP64 iteration from the original start
        const bool ok = newton_wv(S, gfac, W, vsq, it);
        it += it32;
        return ok;
    }
    const double D64 = S.D, Bsq64 = S.Bsq, QB264 = S.QB2, Qdotn64 = S.Qdotn, Qtsq64 = S.Qtsq;
    // the FP32 root in FP64 (W = w / k exactly) and the exact powers 1/k, k^3, k^4 in FP64
    const int ed = (int)eb - 127;  // 1/k = 2^ed
    const double ik = __hiloint2double((1023 + ed) << 20, 0);
    const double k3 = __hiloint2double((1023 - 3 * ed) << 20, 0), k4 = __hiloint2double((1023 - 4 * ed) << 20, 0);
    double Wd = widen(w) * ik, vd = widen(v);
    int it64 = 0;
    {
        // FP64 residuals of newton_wv's form (times W^2) at the root
        const double omv = 1.0 - vd;
        const double sq = omv * rsqrt(omv);
        const double W2 = Wd * Wd;
        const double BW = Bsq64 + Wd;
        const double p = gfac * (Wd * omv - D64 * sq);
        const double f1 = (-0.5 * Bsq64 * (1.0 + vd) - Wd + p - Qdotn64) * W2 + 0.5 * QB264;
        const double f2 = (vd * BW * BW - Qtsq64) * W2 - QB264 * (Bsq64 + 2.0 * Wd);
        // in the FP32 stage's scaled form: k f1 / W^2 = k^3 f1 / w^2, k^2 f2 / W^2 = k^4 f2 / w^2
        const float iw = 1.0f / w, iw2 = iw * iw;
        const float r1 = narrow(f1 * k3) * iw2, r2 = narrow(f2 * k4) * iw2;
        // the FP32 Jacobian at the root
        const float om = 1.0f - v;
        const float rs = rsqrtf(om);
        const float bw = Bsq + w;
        const float j11 = -QB2 * iw2 * iw - 1.0f + gf * om;
        const float j12 = -0.5f * Bsq + gf * (0.5f * D * rs - w);
        const float j21 = 2.0f * bw * (v + QB2 * iw2 * iw);
        const float j22 = bw * bw;
        const float det = j11 * j22 - j12 * j21;
        const float idet = 1.0f / det;
        const float dw = (j12 * r2 - j22 * r1) * idet, dv = (j21 * r1 - j11 * r2) * idet;
        const float step = fabsf(dw) + fabsf(dv) * w;
        const float cancel = (fabsf(j11 * j22) + fabsf(j12 * j21)) * fabsf(idet);
        const double Wn = Wd + widen(dw) * ik;
        const double vn = fmin(fmax(vd + widen(dv), 0.0), C2P_VSQMAX);
        if (Wn > 0.0 && step < 1e-5f * w && step * cancel < 1e-3f * w) {
            it = it32 + 1;
            W = Wn;
            vsq = vn;
            return true;
        }
        if (Wn > 0.0) {
            Wd = Wn;
            vd = vn;
        }
    }
    bool ok = false;
    for (it64 = 1; it64 <= C2P_NMAX; it64++) {
        const double omv = 1.0 - vd;
        const double rs = rsqrt(omv);
        const double sq = omv * rs;
        const double W2 = Wd * Wd, W3 = W2 * Wd;
        const double BW = Bsq64 + Wd;
        const double p = gfac * (Wd * omv - D64 * sq);
        // scaled as in newton_wv: one reciprocal per iteration
        const double f1 = (-0.5 * Bsq64 * (1.0 + vd) - Wd + p - Qdotn64) * W2 + 0.5 * QB264;
        const double f2 = (vd * BW * BW - Qtsq64) * W2 - QB264 * (Bsq64 + 2.0 * Wd);
        const double j11 = (gfac * omv - 1.0) * W3 - QB264;
        const double j12 = -0.5 * Bsq64 + gfac * (0.5 * D64 * rs - Wd);
        const double j21 = 2.0 * BW * (vd * W3 + QB264);
        const double j22 = BW * BW;
        const double r = 1.0 / ((j11 * j22 - j12 * j21) * W2);
        const double Wn = Wd + (j12 * f2 - j22 * f1) * W3 * r;
        const double vn = fmin(fmax(vd + (j21 * f1 - j11 * f2) * r, 0.0), C2P_VSQMAX);
        if (!(Wn > 0.0)) break;
        const double err = fabs(Wn - Wd) + fabs(vn - vd) * Wn;
        Wd = Wn;
        vd = vn;
        if (err < C2P_TOL * Wn) {
            ok = true;
            break;
        }
    }
    if (it64 > C2P_NMAX) it64 = C2P_NMAX;
    it = it32 + 1 + it64;
    W = Wd;
    vsq = vd;
    return ok;
}

// Aitken-accelerated inversion (Sec. 2.6 names it beside Newton; Newman &
// Hamlin 2014). With E = -Q.n, S^2 = Qt^2, T = Q.B the two equations give, for
// a trial pressure p, a cubic in phi = W + B^2: phi^3 - a phi^2 + d = 0,
// a = E + p + B^2/2, d = (S^2 B^2 - T^2)/2. Its largest root (closed form
// (a/3)(1 + 2 cos(acos(1 - 27 d / (2 a^3)) / 3))), v^2 from the momentum
// equation and the ideal-gas pressure of (W, v^2) map p to the next p.
// Returns false when W <= 0 or the pressure is not finite.
__device__ __forceinline__ bool nh_map(const C2PScalars& S, double gfac, double p, double& W, double& vsq,
                                       double& pn) {
    const double B2 = S.Bsq;
    const double a = -S.Qdotn + p + 0.5 * B2;
    const double d = fmax(0.5 * (S.Qtsq * B2 - S.QB2), 0.0);
    if (!(a > 0.0)) return false;
    const double x = fmin(fmax(1.0 - 27.0 * d / (2.0 * a * a * a), -1.0), 1.0);
    const double phi = a / 3.0 * (1.0 + 2.0 * cos(acos(x) / 3.0));
    const double w = phi - B2;
    if (!(w > 0.0)) return false;
    const double v = fmin(fmax((S.Qtsq * w * w + S.QB2 * (2.0 * w + B2)) / (w * w * phi * phi), 0.0), C2P_VSQMAX);
    W = w;
    vsq = v;
    pn = gfac * (w * (1.0 - v) - S.D * sqrt(1.0 - v));
    return isfinite(pn);
}

// Steffensen's form of the Aitken delta-squared acceleration of p -> map(p):
// two evaluations from p0 give p1, p2, and the next cycle starts from
// p0 - (p1 - p0)^2 / (p2 - 2 p1 + p0) (from p2 when that is not a valid
// pressure). Pressures stay >= max(0, (27 d / 4)^(1/3) - E - B^2/2), where
// the cubic has its root. An extrapolation step below C2P_TOL W ends the
// iteration, and one more evaluation gives (W, v^2). `it` counts evaluations.
__device__ __forceinline__ bool aitken_wv(const C2PScalars& S, double gfac, double p, double& W, double& vsq,
                                          int& it) {
    const double d = fmax(0.5 * (S.Qtsq * S.Bsq - S.QB2), 0.0);
    const double pmin = fmax(cbrt(6.75 * d) + S.Qdotn - 0.5 * S.Bsq, 0.0);
    if (!(p >= pmin)) p = pmin;
    it = 0;
    for (int cycle = 1; cycle <= C2P_NMAX; cycle++) {
        double W1, v1, p1, W2, v2, p2;
        it++;
        if (!nh_map(S, gfac, p, W1, v1, p1)) return false;
        p1 = fmax(p1, pmin);
        it++;
        if (!nh_map(S, gfac, p1, W2, v2, p2)) return false;
        p2 = fmax(p2, pmin);
        const double den = p2 - 2.0 * p1 + p;
        double pa = p2;
        if (den != 0.0) {
            const double e = p - (p1 - p) * (p1 - p) / den;
            if (e >= pmin && isfinite(e)) pa = e;
        }
        const double step = fabs(pa - p);
        p = pa;
        if (step < C2P_TOL * W2) {
            it++;
            double pn;
            return nh_map(S, gfac, p, W, vsq, pn);
        }
    }
    return false;
}

// rho and u_g of a converged (W, v^2) (u_g = p / (gam - 1) = (W (1 - v^2) - D sqrt(1 - v^2)) / gam);
// false unless both are positive. rs: 1/sqrt(1 - v^2), the Lorentz factor, for the velocity.
__device__ __forceinline__ bool energy_result(const C2PScalars& S, double igam, double W, double vsq, double& rho,
                                              double& u, double& rs) {
    const double omv = 1.0 - vsq;
    rs = rsqrt(omv);
    const double sq = omv * rs;
    rho = S.D * sq;
    u = (W * omv - S.D * sq) * igam;
    return (rho > 0.0) && (u > 0.0);
}

// The inversion in three pieces (invert() below composes them):
// c2p_prepare (scalars and the start from the guess primitives), any number of
// energy-equation attempts from given starts, c2p_finish (entropy backup when
// no attempt succeeded, then the primitives).
struct C2PWork {
    C2PScalars S;
    double W0, vsq0;  // the start from the guess primitives
    double p0;        // ... and its pressure (the Aitken inversion's start)
    int method;       // HAMR_INV_NEWTON or HAMR_INV_AITKEN
    int mixed;        // Newton: FP32 iterations first (newton_wv_mixed)
    double igam, gfac;  // 1/gam and (gam - 1)/gam, from one division per inversion
    double W, vsq, rho, u;
    double rs;        // 1/sqrt(1 - v^2) of an energy result
    bool ok;
    int its;          // Newton iterations of every energy attempt
};

// start32 (mixed form, optional): the start (W, v^2) already formed in FP32 from the guess primitives;
// igam, gfac (optional, > 0): 1/gam and (gam - 1)/gam formed once by the caller (else here, per state)
__device__ __forceinline__ void c2p_prepare(const double U[NCONS], const double Bc[3], const Metric<double>& m,
                                            double gam, const double pr[NPRIM], C2PWork& w,
                                            int method = HAMR_INV_NEWTON, int mixed = 0,
                                            const float* start32 = nullptr, double igam = 0.0, double gfac = 0.0) {
    c2p_scalars(U, Bc, m, w.S);
    if (igam > 0.0) {
        w.igam = igam;
        w.gfac = gfac;
    } else {
        w.igam = 1.0 / gam;
        w.gfac = (gam - 1.0) * w.igam;
    }
    w.method = method;
    w.mixed = mixed;
    w.p0 = (method == HAMR_INV_AITKEN) ? (gam - 1.0) * pr[UU] : 0.0;
    if (mixed && start32) {
        w.W0 = widen(start32[0]);
        w.vsq0 = widen(fminf(start32[1], (float)C2P_VSQMAX));
    } else if (mixed) {
        // the start only seeds the FP32 iterations (and, where they fail, the FP64 ones): in FP32
        const float q1 = narrow(pr[U1]), q2 = narrow(pr[U2]), q3 = narrow(pr[U3]);
        const float qsq = narrow(m.g11) * q1 * q1 + narrow(m.g22) * q2 * q2 + narrow(m.g33) * q3 * q3 +
                          2.0f * narrow(m.g13) * q1 * q3;
        const float gsq = 1.0f + qsq;
        w.W0 = widen((narrow(pr[RHO]) + narrow(gam) * narrow(pr[UU])) * gsq);
        w.vsq0 = widen(fminf(qsq / gsq, (float)C2P_VSQMAX));
    } else {
        const double q1 = pr[U1], q2 = pr[U2], q3 = pr[U3];
        const double qsq = m.g11 * q1 * q1 + m.g22 * q2 * q2 + m.g33 * q3 * q3 + 2.0 * m.g13 * q1 * q3;
        const double gsq = 1.0 + qsq;
        w.W0 = (pr[RHO] + gam * pr[UU]) * gsq;
        w.vsq0 = fmin(qsq * (1.0 / gsq), C2P_VSQMAX);
    }
    w.W = w.W0;
    w.vsq = 0.0;
    w.rho = w.u = 0.0;
    w.ok = false;
    w.its = 0;
}

// one energy-equation attempt from the pressure p (Aitken inversion)
__device__ __forceinline__ void c2p_attempt_p(C2PWork& w, double gam, double p) {
    if (w.ok) return;
    (void)gam;
    int it = 0;
    double W = 0.0, vsq = 0.0;
    bool ok = aitken_wv(w.S, w.gfac, p, W, vsq, it);
    w.its += it;
    if (ok) {
        w.W = W;
        w.vsq = vsq;
        ok = energy_result(w.S, w.igam, W, vsq, w.rho, w.u, w.rs);
    }
    w.ok = ok;
}

// one energy-equation attempt from (W, v^2); no-op once an attempt succeeded.
// The Aitken inversion starts from the pressure of (W, v^2).
__device__ __forceinline__ void c2p_attempt(C2PWork& w, double gam, double W, double vsq) {
    if (w.ok || !(W > 0.0)) return;
    const double gfac = w.gfac;
    vsq = fmin(fmax(vsq, 0.0), C2P_VSQMAX);
    if (w.method == HAMR_INV_AITKEN) {
        c2p_attempt_p(w, gam, gfac * (W * (1.0 - vsq) - w.S.D * sqrt(1.0 - vsq)));
        return;
    }
    int it = 0;
    bool ok = w.mixed ? newton_wv_mixed(w.S, gfac, W, vsq, it) : newton_wv(w.S, gfac, W, vsq, it);
    w.its += it;
    w.W = W;
    w.vsq = vsq;
    if (ok) ok = energy_result(w.S, w.igam, W, vsq, w.rho, w.u, w.rs);
    w.ok = ok;
}

// the attempt from the guess primitives: (W, v^2) for Newton, their pressure for Aitken
__device__ __forceinline__ void c2p_attempt_plain(C2PWork& w, double gam) {
    if (w.method == HAMR_INV_AITKEN)
        c2p_attempt_p(w, gam, w.p0);
    else
        c2p_attempt(w, gam, w.W0, w.vsq0);
}

// pr: out the result (slots 0..4) unless INV_FAIL (then untouched)
__device__ __forceinline__ int c2p_finish(C2PWork& w, const double U[NCONS], const Metric<double>& m, double gam,
                                          double pr[NPRIM]) {
    const C2PScalars& S = w.S;
    const double D = S.D, Bsq = S.Bsq, QB2 = S.QB2, Qtsq = S.Qtsq;
    double W = w.W, vsq = w.vsq, rho = w.rho, u = w.u;
    int status = INV_OK;
    if (!w.ok) {
        const double kappa = U[C_ENT] / U[C_RHO];
        const double gr = gam / (gam - 1.0);
        W = w.W0;
        bool eok = false;
        for (int k = 1; k <= C2P_NMAX; k++) {
            const double W2 = W * W;
            const double BW = Bsq + W;
            const double num = Qtsq * W2 + QB2 * (Bsq + 2.0 * W);
            const double den = W2 * BW * BW;
            const double iden = 1.0 / den;
            double vs = num * iden;
            double dvs = (2.0 * (Qtsq * W + QB2) - num * 2.0 * W * BW * (Bsq + 2.0 * W) * iden) * iden;
            if (vs > C2P_VSQMAX) {
                vs = C2P_VSQMAX;
                dvs = 0.0;
            }
            const double s1 = 1.0 - vs;
            const double sq = sqrt(s1);
            const double rh = D * sq;
            const double p = kappa * pow(rh, gam);
            const double f = W * s1 - rh - gr * p;
            const double drh = -0.5 * D / sq * dvs;
            const double df = s1 - W * dvs - drh * (1.0 + gr * gam * p / rh);
            const double Wn = W - f / df;
            if (!(Wn > 0.0)) break;
            const double err = fabs(Wn - W);
            W = Wn;
            if (err < C2P_TOL * Wn) {
                eok = true;
                break;
            }
        }
        if (eok) {
            const double W2 = W * W;
            const double BW = Bsq + W;
            vsq = fmin((Qtsq * W2 + QB2 * (Bsq + 2.0 * W)) / (W2 * BW * BW), C2P_VSQMAX);
            const double sq = sqrt(1.0 - vsq);
            rho = D * sq;
            u = kappa * pow(rho, gam) / (gam - 1.0);
            eok = (rho > 0.0) && (u > 0.0) && (vsq >= 0.0);
        }
        if (!eok) return INV_FAIL;
        status = INV_ENTROPY;
    }
    // utilde^i = Gamma/(W + B^2) (Qt^i + (Q.B) Bn^i / W), Qt^i = Q^i - alpha g^{ti} (Q.n);
    // 1/(W + B^2) and 1/W from one reciprocal of W (W + B^2)
    const double gamma = (status == INV_OK) ? w.rs : rsqrt(1.0 - vsq);
    const double WB = W + Bsq;
    const double r = 1.0 / (W * WB);
    const double pre = gamma * W * r;
    const double qbw = S.QdotB * WB * r;
    pr[U1] = pre * (S.Qc1 - m.alpha * m.c01 * S.Qdotn + qbw * S.Bn1);
    pr[U2] = pre * (S.Qc2 + qbw * S.Bn2);
    pr[U3] = pre * (S.Qc3 + qbw * S.Bn3);
    pr[RHO] = rho;
    pr[UU] = u;
    w.W = W;
    w.vsq = vsq;
    return status;
}

// pr: in the guess (slots 0..4), out the result (slots 0..4) unless INV_FAIL.
// guess2 (optional): a first start (W, v^2) tried before the one of pr; the
// start from pr is then the fallback. `iters` counts the energy-inversion
// Newton iterations of every start tried.
__device__ __forceinline__ int invert(const double U[NCONS], const double Bc[3], const Metric<double>& m, double gam,
                                      double pr[NPRIM], int* iters, bool entropy_only,
                                      const double* guess2 = nullptr, int method = HAMR_INV_NEWTON) {
    C2PWork w;
    c2p_prepare(U, Bc, m, gam, pr, w, method);
    if (!entropy_only) {
        if (guess2) c2p_attempt(w, gam, guess2[0], guess2[1]);
        c2p_attempt_plain(w, gam);
    }
    if (iters) *iters = w.its;
    return c2p_finish(w, U, m, gam, pr);
}

}  // namespace hamr
