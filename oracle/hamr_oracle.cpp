/* hamr_oracle.cpp -- plain, slow, single-threaded FP64 CPU oracle of the
 * H-AMR GRMHD block update (Liska et al., arXiv 1912.10192, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY. It defines what the CUDA path must compute and is
 * used by tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg.
 * It shares no code with paper_1912_10192_gb300/csrc and neither side
 * includes or links the other.
 *
 * Every function follows the paper's equations in the paper's order; readings
 * of passages the paper leaves silent or prints garbled are marked "Reading:".
 *
 *   geometry         Sec. 2.2 "Coordinate System and Metric"
 *   primitives       Sec. 2.3 (b^t, b^i, utilde^i relations; T, F*, kappa)
 *   conserved/flux   Sec. 2.4-2.5 (U, F^j, sqrt(-g) absorbed)
 *   reconstruction   Sec. 2.1 (PPM of primitives; MINMOD/MC as options)
 *   Riemann solver   Sec. 2.1 (HLLE with the approximate fast speed; LLF option)
 *   EMF / CT         Sec. 2.5 (4-flux EMF average, staggered face-B update,
 *                    face-to-centre B average)
 *   source           Sec. 2.5 (sqrt(-g) T^k_l Gamma^l_{nu k})
 *   inversion        Sec. 2.6 (2-D Newton on (W, v^2); entropy backup)
 *   floors           Sec. 2.7 (b^2/rho<50, b^2/u<750, rho>1e-7/r^2, u>1e-9/r^(10/3))
 *   time step        Sec. 2.1 (midpoint predictor/corrector; C0 / sum 1/dt^i)
 */
#include "ora_real.h"
#include "hamr_oracle.h"

#include <cmath>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <vector>

#ifdef ORA_COUNT_FLOPS
extern "C" {
unsigned long long ora_flop_ctr[5] = {0, 0, 0, 0, 0};
}
#endif

/* phase attribution of the counted operations (counting build only):
 * 0 reconstruction, 1 face fluxes, 2 EMFs, 3 CT, 4 cell update + inversion
 * + floors, 5 CFL rate. Elements: the five counter classes. */
static unsigned long long ora_phase_ctr[6][5];
[[maybe_unused]] static unsigned long long ora_phase_mark[5];
static void phase_begin() {
#ifdef ORA_COUNT_FLOPS
    for (int m = 0; m < 5; m++) ora_phase_mark[m] = ora_flop_ctr[m];
#endif
}
static void phase_end(int ph) {
#ifdef ORA_COUNT_FLOPS
    for (int m = 0; m < 5; m++) ora_phase_ctr[ph][m] += ora_flop_ctr[m] - ora_phase_mark[m];
#else
    (void)ph;
#endif
}

namespace {

const int NG = 3;                                   /* ghost layers */
enum { RHO = 0, UU, U1, U2, U3, B1, B2, B3, NPR };  /* primitive slots */
enum { CRHO = 0, CEN, CS1, CS2, CS3, CENT, NCONS }; /* cell conserved slots */
const int NFX = 8; /* face-flux slots: 0..5 as NCONS, 6/7 = the two B^i with i != dir */

/* Reading (Sec. 2.2): the paper takes Christoffel symbols "by finite
 * differences of the metric in internal coordinates" without the stencil;
 * we use 4th-order central differences with this step in x1 and x2. */
const double CONN_H = 1.0e-3;

/* Reading (Sec. 2.6): Newton stopping rule and limits, not given in the paper. */
const double C2P_TOL = 1.0e-10;
const int C2P_NMAX = 30;
const double GAMMA_MAX = 50.0;

/* ------------------------------------------------------------------ */
/* geometry (Sec. 2.2)                                                  */
/* ------------------------------------------------------------------ */

struct Geom {
    real gcov[4][4];
    real gcon[4][4];
    real gdet;  /* sqrt(-g) in internal coordinates */
    real alpha; /* lapse 1/sqrt(-g^{00}) */
    int pole;   /* 1: an x2 face on the polar axis (sqrt(-g) = 0) */
};

/* Reflect theta into [0, pi]: ghost cells beyond the pole take the geometry
 * of the mirrored point (transmissive polar boundary, Sec. 3.3.1). */
static double mirror_theta(double th) {
    const double pi = 3.14159265358979323846;
    if (th < 0.0) return -th;
    if (th > pi) return 2.0 * pi - th;
    return th;
}

/* Kerr metric in Kerr-Schild coordinates (M = 1), transformed to internal
 * coordinates x1 = log r, x2 = theta, x3 = phi. The Jacobian of x1 = log r is
 * dr/dx1 = r, applied analytically: every covariant r index gets a factor r,
 * every contravariant one a factor 1/r. */
static void metric_point(const ora_desc& d, double x1, double x2, double gcov[4][4],
                         double gcon[4][4], double* gdet) {
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) gcov[m][n] = gcon[m][n] = 0.0;
    if (d.metric == ORA_METRIC_MINKOWSKI) {
        gcov[0][0] = gcon[0][0] = -1.0;
        for (int i = 1; i < 4; i++) gcov[i][i] = gcon[i][i] = 1.0;
        *gdet = 1.0;
        return;
    }
    /* flat spherical coordinates: the same form with mass 0 and no spin */
    const double mass = (d.metric == ORA_METRIC_SPHERICAL) ? 0.0 : 1.0;
    const double a = (d.metric == ORA_METRIC_SPHERICAL) ? 0.0 : d.a;
    const double r = std::exp(x1);
    const double th = mirror_theta(x2);
    const double sth = std::sin(th), cth = std::cos(th);
    const double s2 = sth * sth;
    const double sig = r * r + a * a * cth * cth;
    const double del = r * r - 2.0 * mass * r + a * a;
    const double z = 2.0 * mass * r / sig;
    /* covariant KS: g_tt, g_tr, g_tphi, g_rr, g_rphi, g_thth, g_phph */
    gcov[0][0] = -(1.0 - z);
    gcov[0][1] = gcov[1][0] = z * r;
    gcov[0][3] = gcov[3][0] = -z * a * s2;
    gcov[1][1] = (1.0 + z) * r * r;
    gcov[1][3] = gcov[3][1] = -a * s2 * (1.0 + z) * r;
    gcov[2][2] = sig;
    gcov[3][3] = s2 * (sig + a * a * s2 * (1.0 + z));
    /* contravariant KS */
    gcon[0][0] = -(1.0 + z);
    gcon[0][1] = gcon[1][0] = z / r;
    gcon[1][1] = del / sig / (r * r);
    gcon[1][3] = gcon[3][1] = a / sig / r;
    gcon[2][2] = 1.0 / sig;
    gcon[3][3] = 1.0 / (sig * s2);
    *gdet = r * sig * sth;
}

static void geom_point(const ora_desc& d, double x1, double x2, Geom& G) {
    double gc[4][4], gn[4][4], gd;
    metric_point(d, x1, x2, gc, gn, &gd);
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            G.gcov[m][n] = gc[m][n];
            G.gcon[m][n] = gn[m][n];
        }
    G.gdet = gd;
    G.alpha = 1.0 / std::sqrt(-gn[0][0]);
    G.pole = 0;
}

/* Gamma^l_{mn} = 1/2 g^{lk} (d_m g_{kn} + d_n g_{km} - d_k g_{mn}); only
 * d/dx1 and d/dx2 are non-zero (stationary, axisymmetric metric). */
static void conn_point(const ora_desc& d, double x1, double x2, double conn[4][4][4]) {
    double dg[4][4][4];
    for (int s = 0; s < 4; s++)
        for (int m = 0; m < 4; m++)
            for (int n = 0; n < 4; n++) dg[s][m][n] = 0.0;
    double gc[4][4], gn[4][4], gd;
    if (d.metric != ORA_METRIC_MINKOWSKI) {
        const double h = CONN_H;
        for (int s = 1; s <= 2; s++) {
            double gp2[4][4], gp1[4][4], gm1[4][4], gm2[4][4];
            double ex1 = (s == 1) ? h : 0.0, ex2 = (s == 2) ? h : 0.0;
            metric_point(d, x1 + 2 * ex1, x2 + 2 * ex2, gp2, gn, &gd);
            metric_point(d, x1 + ex1, x2 + ex2, gp1, gn, &gd);
            metric_point(d, x1 - ex1, x2 - ex2, gm1, gn, &gd);
            metric_point(d, x1 - 2 * ex1, x2 - 2 * ex2, gm2, gn, &gd);
            for (int m = 0; m < 4; m++)
                for (int n = 0; n < 4; n++)
                    dg[s][m][n] = (-gp2[m][n] + 8.0 * gp1[m][n] - 8.0 * gm1[m][n] + gm2[m][n]) / (12.0 * h);
        }
    }
    metric_point(d, x1, x2, gc, gn, &gd);
    for (int l = 0; l < 4; l++)
        for (int m = 0; m < 4; m++)
            for (int n = 0; n < 4; n++) {
                double s = 0.0;
                for (int k = 0; k < 4; k++) s += gn[l][k] * (dg[m][k][n] + dg[n][k][m] - dg[k][m][n]);
                conn[l][m][n] = 0.5 * s;
            }
}

/* ------------------------------------------------------------------ */
/* primitives -> 4-vectors (Sec. 2.3)                                   */
/* ------------------------------------------------------------------ */

struct State {
    real ucon[4], ucov[4], bcon[4], bcov[4];
    real bsq;
};

static void lower(const real v[4], const Geom& G, real out[4]) {
    for (int m = 0; m < 4; m++) {
        real s = 0.0;
        for (int n = 0; n < 4; n++) s += G.gcov[m][n] * v[n];
        out[m] = s;
    }
}

/* u^mu from utilde^i: Lorentz factor wrt the normal observer
 * Gamma = sqrt(1 + g_ij ut^i ut^j); u^t = Gamma/alpha;
 * u^i = ut^i - Gamma alpha g^{ti}.
 * Reading: the paper writes utilde^i = u^i + beta^i Gamma/alpha with
 * "beta^i = g^{0i}"; the shift that makes utilde^i = gamma^i_mu u^mu hold is
 * beta^i = alpha^2 g^{0i}, which is what is used here.
 * b^t = B^i u_i, b^i = (B^i + b^t u^i)/u^t. */
static void get_state(const real* pr, const Geom& G, State& s) {
    real qsq = 0.0;
    for (int i = 1; i < 4; i++)
        for (int j = 1; j < 4; j++) qsq += G.gcov[i][j] * pr[U1 + i - 1] * pr[U1 + j - 1];
    real gamma = sqrt(1.0 + qsq);
    s.ucon[0] = gamma / G.alpha;
    for (int i = 1; i < 4; i++) s.ucon[i] = pr[U1 + i - 1] - gamma * G.alpha * G.gcon[0][i];
    lower(s.ucon, G, s.ucov);
    real bt = 0.0;
    for (int i = 1; i < 4; i++) bt += pr[B1 + i - 1] * s.ucov[i];
    s.bcon[0] = bt;
    for (int i = 1; i < 4; i++) s.bcon[i] = (pr[B1 + i - 1] + bt * s.ucon[i]) / s.ucon[0];
    lower(s.bcon, G, s.bcov);
    real bsq = 0.0;
    for (int m = 0; m < 4; m++) bsq += s.bcon[m] * s.bcov[m];
    s.bsq = bsq;
}

/* T^mu_nu of ideal MHD.
 * Reading: the printed T^mu_nu omits the b^2 u^mu u_nu term; the stress
 * tensor of the paper's own F*^{mu nu} = b^mu u^nu - b^nu u^mu contains it, so
 * T^mu_nu = (rho + u + p + b^2) u^mu u_nu + delta^mu_nu (p + b^2/2) - b^mu b_nu. */
static real tmunu(const real* pr, const State& s, int mu, int nu, double gam) {
    real p = (gam - 1.0) * pr[UU];
    real eta = pr[RHO] + pr[UU] + p + s.bsq;
    real t = eta * s.ucon[mu] * s.ucov[nu] - s.bcon[mu] * s.bcov[nu];
    if (mu == nu) t = t + (p + 0.5 * s.bsq);
    return t;
}

/* U (dir = 0) or F^dir (dir = 1..3), not yet multiplied by sqrt(-g):
 *   [rho u^dir, T^dir_t + rho u^dir, T^dir_i, kappa rho u^dir, B-flux^1..3].
 * Reading: the energy entry is T^dir_t + rho u^dir for U and F alike (the
 * paper evolves div(T^mu_t + rho u^mu)); the printed "+ rho u^t" in F is taken
 * as a slip.
 * Reading: the flux of B^i in direction j is F*^{ij} = b^i u^j - b^j u^i, the
 * sign that makes U_B = B^i = F*^{it} obey div F* = 0; the printed
 * "b^j u^i - b^i u^j" has the opposite sign. (For dir = 0 this gives B^i.) */
/* kap: the entropy tracer kappa to use (the face value reconstructed from the
 * cells' kappa, see stage_fluxes); NULL: kappa = p / rho^gam of pr */
static void prim_to_uf(const real* pr, const State& s, int dir, double gam, real out[9], const real* kap = nullptr) {
    real mass = pr[RHO] * s.ucon[dir];
    out[0] = mass;
    out[1] = tmunu(pr, s, dir, 0, gam) + mass;
    for (int i = 1; i < 4; i++) out[1 + i] = tmunu(pr, s, dir, i, gam);
    real p = (gam - 1.0) * pr[UU];
    real kappa = kap ? *kap : p / pow(pr[RHO], gam);
    out[5] = kappa * mass;
    for (int i = 1; i < 4; i++) out[5 + i] = s.bcon[i] * s.ucon[dir] - s.bcon[dir] * s.ucon[i];
}

/* Fastest characteristic speeds dx^dir/dt of the magnetosonic wave.
 * Reading (Sec. 2.1 "approximation for the fast-wave speed"): the fluid-frame
 * speed c^2 = vA^2 + cs^2 (1 - vA^2), cs^2 = gam p / w, vA^2 = b^2/(b^2 + w),
 * w = rho + u + p, put into the dispersion relation of a sound wave,
 * (k.u)^2 = c^2 (k.k + (k.u)^2) with k_mu = (-v, delta^dir_mu):
 *   A v^2 - 2 B v + C = 0,
 *   A = (u^t)^2 - c^2 ((u^t)^2 + g^tt), B = u^t u^d - c^2 (u^t u^d + g^td),
 *   C = (u^d)^2 - c^2 ((u^d)^2 + g^dd). */
static void vchar(const real* pr, const State& s, const Geom& G, int dir, double gam, real* vp,
                  real* vm) {
    real p = (gam - 1.0) * pr[UU];
    real w = pr[RHO] + pr[UU] + p;
    real cs2 = gam * p / w;
    real va2 = s.bsq / (s.bsq + w);
    real cms2 = va2 + cs2 * (1.0 - va2);
    real ut = s.ucon[0], ud = s.ucon[dir];
    real A = ut * ut - cms2 * (ut * ut + G.gcon[0][0]);
    real B = ut * ud - cms2 * (ut * ud + G.gcon[0][dir]);
    real C = ud * ud - cms2 * (ud * ud + G.gcon[dir][dir]);
    real disc = B * B - A * C;
    if (disc < 0.0) disc = 0.0;
    real sd = sqrt(disc);
    *vp = (B + sd) / A;
    *vm = (B - sd) / A;
}

/* ------------------------------------------------------------------ */
/* reconstruction (Sec. 2.1)                                            */
/* ------------------------------------------------------------------ */

/* Monotonised central slope (Colella-Woodward 1984 form):
 * sign(dc) min(|dc|, 2|dl|, 2|dr|) when dl, dr have the same sign, else 0. */
static real slope_mc(real qm, real q0, real qp) {
    real dl = q0 - qm, dr = qp - q0;
    if (dl * dr <= 0.0) return 0.0;
    real dc = 0.5 * (qp - qm);
    real m = fabs(dc);
    if (2.0 * fabs(dl) < m) m = 2.0 * fabs(dl);
    if (2.0 * fabs(dr) < m) m = 2.0 * fabs(dr);
    return (dc > 0.0) ? m : -m;
}

static real slope_minmod(real qm, real q0, real qp) {
    real dl = q0 - qm, dr = qp - q0;
    if (dl * dr <= 0.0) return 0.0;
    return (fabs(dl) < fabs(dr)) ? dl : dr;
}

/* Left/right edge values of every cell of a 1-D line q[0..n-1].
 * PPM (Reading: Colella & Woodward 1984 on a uniform mesh, no flattener, no
 * steepener, as the paper's shock tubes): interface values
 * a_{c+1/2} = (q_c + q_{c+1})/2 - (dq_{c+1} - dq_c)/6 with monotonised slopes,
 * then the per-cell parabola constraints. Valid for c = 2..n-3.
 * MC / MINMOD: piecewise linear, valid for c = 1..n-2. */
/* Shock flattening coefficient of every cell of a line (Colella & Woodward 1984,
 * their flattening of the interface values near strong shocks), from the
 * internal energy u (p = (gam - 1) u) and the velocity primitive w along the
 * line. Reading: a cell sits in a shock when the pressure jumps across it by
 * more than 0.33 of the smaller neighbour, |p(c+1) - p(c-1)| >
 * 0.33 min(p(c+1), p(c-1)), and the flow converges there, w(c-1) > w(c+1);
 * then f = 10 (|dp1| / |dp2| - 3/4) clamped to [0, 1], dp1 = p(c+1) - p(c-1),
 * dp2 = p(c+2) - p(c-2) (a sharp jump gives |dp1| = |dp2|, f = 1; a linear
 * ramp |dp2| = 2 |dp1|, f = 0). Reading: the ratio is taken in magnitude and
 * dp2 = 0 counts as an infinitely sharp jump (f = 1). On a monotone profile
 * this is the signed ratio; at a narrow pressure peak (two shocks leaving a
 * collision) p(c+2) - p(c-2) vanishes up to rounding, and the signed ratio
 * would jump between plus and minus infinity on the rounding noise. The coefficient stays with its cell: Colella & Woodward
 * also take the larger coefficient of the upwind neighbour, whose stencil
 * would reach past three ghost layers. Gas pressure only (no magnetic term).
 * Valid for c = 2..n-3; f = 0 elsewhere. */
static void flatten_line(int n, real gam, const real* u, const real* w, real* f) {
    for (int c = 0; c < n; c++) f[c] = 0.0;
    for (int c = 2; c <= n - 3; c++) {
        real pm = (gam - 1.0) * u[c - 1], pp = (gam - 1.0) * u[c + 1];
        real dp1 = pp - pm;
        real dp2 = (gam - 1.0) * (u[c + 2] - u[c - 2]);
        real pmin = pm < pp ? pm : pp;
        real a1 = fabs(dp1), a2 = fabs(dp2);
        if (a1 > 0.33 * pmin && w[c - 1] > w[c + 1]) {
            if (a2 == 0.0) {
                f[c] = 1.0;
            } else {
                real x = 10.0 * (a1 / a2 - 0.75);
                f[c] = x < 0.0 ? real(0.0) : (x > 1.0 ? real(1.0) : x);
            }
        }
    }
}

/* flat: optional per-cell flattening coefficients f in [0, 1] (Colella & Woodward 1984): the
 * interface values become f q + (1 - f) a before the parabola constraints */
static void recon_line_impl(int recon, int n, const real* q, real* al, real* ar, const real* flat = nullptr) {
    if (recon == ORA_RECON_PPM) {
        std::vector<real> dq(n, real(0.0)), ah(n, real(0.0));
        for (int c = 1; c <= n - 2; c++) dq[c] = slope_mc(q[c - 1], q[c], q[c + 1]);
        for (int c = 1; c <= n - 3; c++) ah[c] = 0.5 * (q[c] + q[c + 1]) - (dq[c + 1] - dq[c]) / 6.0;
        for (int c = 2; c <= n - 3; c++) {
            real aL = ah[c - 1], aR = ah[c], q0 = q[c];
            if (flat) {
                aL = flat[c] * q0 + (1.0 - flat[c]) * aL;
                aR = flat[c] * q0 + (1.0 - flat[c]) * aR;
            }
            if ((aR - q0) * (q0 - aL) <= 0.0) {
                aL = q0;
                aR = q0;
            } else {
                real da = aR - aL;
                real a6 = 6.0 * (q0 - 0.5 * (aL + aR));
                if (da * a6 > da * da)
                    aL = 3.0 * q0 - 2.0 * aR;
                else if (-(da * da) > da * a6)
                    aR = 3.0 * q0 - 2.0 * aL;
            }
            al[c] = aL;
            ar[c] = aR;
        }
    } else {
        for (int c = 1; c <= n - 2; c++) {
            real dq = (recon == ORA_RECON_MC) ? slope_mc(q[c - 1], q[c], q[c + 1])
                                              : slope_minmod(q[c - 1], q[c], q[c + 1]);
            al[c] = q[c] - 0.5 * dq;
            ar[c] = q[c] + 0.5 * dq;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Riemann solver (Sec. 2.1)                                            */
/* ------------------------------------------------------------------ */

static int bslot(int dir, int i) { /* flux slot 6/7 of B^i for a dir-face, i != dir */
    int t1 = (dir == 1) ? 2 : 1;
    return (i == t1) ? 6 : 7;
}

/* HLLE flux through a dir-face, multiplied by the face sqrt(-g):
 *   F = (cmin F_R + cmax F_L - cmax cmin (U_R - U_L)) / (cmax + cmin),
 *   cmax = max(0, v+_L, v+_R), cmin = max(0, -v-_L, -v-_R).
 * Reading: when cmax + cmin = 0, F = (F_L + F_R)/2.
 * LLF: c = max(cmax, cmin), F = (F_L + F_R - c (U_R - U_L))/2. */
/* kap (optional): the entropy tracer kappa on the left and right of the face */
static void face_flux(const ora_desc& d, const real* pl, const real* pr, const Geom& G, int dir,
                      real F[NFX], const real* kap = nullptr) {
    if (G.pole) {
        for (int m = 0; m < NFX; m++) F[m] = 0.0;
        return;
    }
    State sl, sr;
    get_state(pl, G, sl);
    get_state(pr, G, sr);
    real Ul[9], Ur[9], Fl[9], Fr[9];
    prim_to_uf(pl, sl, 0, d.gam, Ul, kap);
    prim_to_uf(pl, sl, dir, d.gam, Fl, kap);
    prim_to_uf(pr, sr, 0, d.gam, Ur, kap ? kap + 1 : nullptr);
    prim_to_uf(pr, sr, dir, d.gam, Fr, kap ? kap + 1 : nullptr);
    real vpl, vml, vpr, vmr;
    vchar(pl, sl, G, dir, d.gam, &vpl, &vml);
    vchar(pr, sr, G, dir, d.gam, &vpr, &vmr);
    real cmax = fmax(0.0, fmax(vpl, vpr));
    real cmin = fmax(0.0, fmax(-vml, -vmr));
    int src[NFX] = {0, 1, 2, 3, 4, 5, 0, 0};
    for (int i = 1, k = 6; i < 4; i++)
        if (i != dir) src[k++] = 5 + i;
    for (int m = 0; m < NFX; m++) {
        int c = src[m];
        real f;
        if (d.riemann == ORA_FLUX_LLF) {
            real cm = fmax(cmax, cmin);
            f = 0.5 * (Fl[c] + Fr[c] - cm * (Ur[c] - Ul[c]));
        } else if (cmax + cmin > 0.0) {
            f = (cmin * Fr[c] + cmax * Fl[c] - cmax * cmin * (Ur[c] - Ul[c])) / (cmax + cmin);
        } else {
            f = 0.5 * (Fl[c] + Fr[c]);
        }
        F[m] = f * G.gdet;
    }
}

/* ------------------------------------------------------------------ */
/* source (Sec. 2.5): Qbar_nu = sqrt(-g) T^k_l Gamma^l_{nu k}           */
/* ------------------------------------------------------------------ */

/* Reading: the paper prints the momentum component; the energy component
 * (nu = t) follows from the same covariant divergence, and mass, entropy and
 * B have no source. */
static void source_terms(const ora_desc& d, const real* pr, const State& s, const Geom& G,
                         const double conn[4][4][4], real Q[NCONS]) {
    real T[4][4];
    for (int k = 0; k < 4; k++)
        for (int l = 0; l < 4; l++) T[k][l] = tmunu(pr, s, k, l, d.gam);
    real q[4];
    for (int nu = 0; nu < 4; nu++) {
        real sum = 0.0;
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++) sum += T[k][l] * real(conn[l][nu][k]);
        q[nu] = sum * G.gdet;
    }
    Q[CRHO] = 0.0;
    Q[CEN] = q[0];
    Q[CS1] = q[1];
    Q[CS2] = q[2];
    Q[CS3] = q[3];
    Q[CENT] = 0.0;
}

/* ------------------------------------------------------------------ */
/* conserved -> primitive inversion (Sec. 2.6)                          */
/* ------------------------------------------------------------------ */

enum { C2P_OK = 0, C2P_ENTROPY = 1, C2P_FAIL = 2, C2P_FLOOR = 4 };

/* Inverts U (sqrt(-g) weighted: rho u^t, T^t_t + rho u^t, T^t_i, kappa rho u^t)
 * with the cell-centred B^i, for rho, u, utilde^i.
 *
 * Normal-observer scalars (n_mu = (-alpha, 0, 0, 0), sqrt(gamma) = sqrt(-g)/alpha):
 *   D = rho Gamma, Q_mu = -n_nu T^nu_mu = alpha T^t_mu, Bn^i = alpha B^i,
 *   Q.n = -alpha Q^t, Qt^2 = Q_mu Q^mu + (Q.n)^2, B^2 = g_ij Bn^i Bn^j, Q.B.
 * Unknowns W = w Gamma^2 (w = rho + u + p) and v^2 = 1 - 1/Gamma^2:
 *   E1: Q.n = -B^2 (1 + v^2)/2 + (Q.B)^2 / (2 W^2) - W + p
 *   E2: Qt^2 = v^2 (B^2 + W)^2 - (Q.B)^2 (B^2 + 2W) / W^2
 *   p  = (gam-1)/gam [ W (1 - v^2) - D sqrt(1 - v^2) ]
 * solved by 2-D Newton-Raphson with the analytic Jacobian (energy inversion);
 * if that fails, the entropy inversion takes p = kappa rho^gam with
 * kappa = U_kappa / U_rho and solves E2 together with
 * W (1 - v^2) = rho + gam/(gam-1) p, rho = D sqrt(1 - v^2) by 1-D Newton in W.
 * Recovery: rho = D/Gamma, u = p/(gam-1),
 *   utilde^i = Gamma/(W + B^2) (Qt^i + (Q.B) Bn^i / W),
 *   Qt^i = (g^{i nu} + n^i n^nu) Q_nu (spatial projection of Q).
 * Reading: tolerance |dW|/W + |dv^2| < 1e-10 (with quadratic convergence the
 * accepted iterate is then at round-off), at most 30 iterations,
 * v^2 kept in [0, 1 - 1/50^2]; a failed state keeps its guess. */
/* The pressure map of Newman & Hamlin (2014), the Aitken-accelerated
 * inversion the paper names beside Newton (Sec. 2.6). With E = -Q.n,
 * S^2 = Qt^2, T = Q.B, E1 and E2 above combine, for a trial pressure p, into
 * a cubic in phi = W + B^2:
 *   phi^3 - a phi^2 + d = 0,  a = E + p + B^2/2,  d = (S^2 B^2 - T^2)/2 >= 0
 * (E1 rewritten with B.v = T/W and v^2 from E2). Its largest root is
 * phi = (a/3)(1 + 2 cos(acos(1 - 27 d / (2 a^3)) / 3)); then W = phi - B^2,
 * v^2 from E2 solved for v^2, and the ideal-gas pressure of (W, v^2) is the
 * image of p. A real root >= 2a/3 needs a^3 >= 27 d / 4: the argument of
 * acos is clamped to [-1, 1] (the caller keeps p above that bound).
 * Returns false when W <= 0 or a value is not finite. */
static bool nh_map(real E, real S2, real T2, real B2, real D, double gfac, double vsqmax, real p, real* W, real* vsq,
                   real* pn) {
    real a = E + p + 0.5 * B2;
    real d = 0.5 * (S2 * B2 - T2);
    if (d < 0.0) d = 0.0;
    if (!(a > 0.0)) return false;
    real x = 1.0 - 27.0 * d / (2.0 * a * a * a);
    if (x < -1.0) x = -1.0;
    if (x > 1.0) x = 1.0;
    real phi = a / 3.0 * (1.0 + 2.0 * cos(acos(x) / 3.0));
    real w = phi - B2;
    if (!(w > 0.0)) return false;
    real v = (S2 * w * w + T2 * (2.0 * w + B2)) / (w * w * phi * phi);
    if (v < 0.0) v = 0.0;
    if (v > vsqmax) v = vsqmax;
    real sq = sqrt(1.0 - v);
    *W = w;
    *vsq = v;
    *pn = gfac * (w * (1.0 - v) - D * sq);
    return isfinite(*pn);
}

/* Energy inversion by the Newman & Hamlin fixed point p -> map(p), accelerated
 * by Aitken's delta-squared extrapolation in Steffensen's form: from p0 two
 * map evaluations give p1, p2, and the cycle restarts from
 * p0 - (p1 - p0)^2 / (p2 - 2 p1 + p0) (from p2 when the denominator is 0 or
 * the extrapolation is not a valid pressure). Pressures are kept >= the
 * bound of the cubic, max(0, (27 d / 4)^(1/3) - E - B^2/2).
 * Reading (stopping rule): an Aitken step smaller than 1e-10 W ends the
 * iteration; one more evaluation at the extrapolated pressure gives (W, v^2)
 * (the extrapolation error is then of second order in that step, as for
 * Newton's last step). At most 30 cycles; iterations counted as map
 * evaluations. Returns 1 when converged. */
static int aitken_energy(real E, real S2, real T2, real B2, real D, double gfac, double vsqmax, real p0, real* W,
                         real* vsq, int* evals) {
    real d = 0.5 * (S2 * B2 - T2);
    if (d < 0.0) d = 0.0;
    real pmin = cbrt(6.75 * d) - E - 0.5 * B2;
    if (pmin < 0.0) pmin = 0.0;
    real p = p0;
    if (!(p >= pmin)) p = pmin;
    int n = 0;
    for (int cycle = 1; cycle <= C2P_NMAX; cycle++) {
        real W1, v1, p1, W2, v2, p2;
        n++;
        if (!nh_map(E, S2, T2, B2, D, gfac, vsqmax, p, &W1, &v1, &p1)) break;
        if (p1 < pmin) p1 = pmin;
        n++;
        if (!nh_map(E, S2, T2, B2, D, gfac, vsqmax, p1, &W2, &v2, &p2)) break;
        if (p2 < pmin) p2 = pmin;
        real den = p2 - 2.0 * p1 + p;
        real pa = p2;
        if (den != 0.0) {
            real e = p - (p1 - p) * (p1 - p) / den;
            if (e >= pmin && isfinite(e)) pa = e;
        }
        real step = fabs(pa - p);
        p = pa;
        if (step < C2P_TOL * W2) {
            n++;
            real pn;
            if (!nh_map(E, S2, T2, B2, D, gfac, vsqmax, p, W, vsq, &pn)) break;
            *evals = n;
            return 1;
        }
    }
    *evals = n;
    return 0;
}

static int con2prim(const ora_desc& d, const real Ucons[NCONS], const real Bc[3], const Geom& G,
                    real* pr, int* iters, int entropy_only = 0) {
    const double gam = d.gam;
    const double gfac = (gam - 1.0) / gam;
    const double vsqmax = 1.0 - 1.0 / (GAMMA_MAX * GAMMA_MAX);
    real alpha = G.alpha, gdet = G.gdet;
    real D = Ucons[CRHO] * alpha / gdet;
    real Qcov[4];
    Qcov[0] = alpha * (Ucons[CEN] - Ucons[CRHO]) / gdet;
    Qcov[1] = alpha * Ucons[CS1] / gdet;
    Qcov[2] = alpha * Ucons[CS2] / gdet;
    Qcov[3] = alpha * Ucons[CS3] / gdet;
    real Qcon[4];
    for (int m = 0; m < 4; m++) {
        real s = 0.0;
        for (int n = 0; n < 4; n++) s += G.gcon[m][n] * Qcov[n];
        Qcon[m] = s;
    }
    real Bn[4] = {0.0, alpha * Bc[0], alpha * Bc[1], alpha * Bc[2]};
    real Qdotn = -alpha * Qcon[0];
    real Qsq = 0.0;
    for (int m = 0; m < 4; m++) Qsq += Qcov[m] * Qcon[m];
    real Qtsq = Qsq + Qdotn * Qdotn;
    real Bsq = 0.0;
    for (int i = 1; i < 4; i++)
        for (int j = 1; j < 4; j++) Bsq += G.gcov[i][j] * Bn[i] * Bn[j];
    real QdotB = 0.0;
    for (int i = 1; i < 4; i++) QdotB += Qcov[i] * Bn[i];
    real QdotBsq = QdotB * QdotB;

    /* initial guess from the guess primitives */
    real qsq = 0.0;
    for (int i = 1; i < 4; i++)
        for (int j = 1; j < 4; j++) qsq += G.gcov[i][j] * pr[U1 + i - 1] * pr[U1 + j - 1];
    real gsq = 1.0 + qsq;
    real vsq = qsq / gsq;
    if (vsq > vsqmax) vsq = vsqmax;
    real W = (pr[RHO] + gam * pr[UU]) * gsq;
    real W0 = W;

    int ok = 0, it = 0;
    if (d.inversion == ORA_INV_AITKEN) {
        /* the start: the pressure of the guess primitives */
        if (!entropy_only)
            ok = aitken_energy(-Qdotn, Qtsq, QdotBsq, Bsq, D, gfac, vsqmax, (gam - 1.0) * pr[UU], &W, &vsq, &it);
    } else {
        for (it = 1; it <= (entropy_only ? 0 : C2P_NMAX); it++) {
            real sq = sqrt(1.0 - vsq);
            real p = gfac * (W * (1.0 - vsq) - D * sq);
            real W2 = W * W;
            real BW = Bsq + W;
            real f1 = -0.5 * Bsq * (1.0 + vsq) + QdotBsq / (2.0 * W2) - W + p - Qdotn;
            real f2 = vsq * BW * BW - QdotBsq * (Bsq + 2.0 * W) / W2 - Qtsq;
            real dpdW = gfac * (1.0 - vsq);
            real dpdv = gfac * (-W + 0.5 * D / sq);
            real j11 = -QdotBsq / (W2 * W) - 1.0 + dpdW;
            real j12 = -0.5 * Bsq + dpdv;
            real j21 = 2.0 * vsq * BW + 2.0 * QdotBsq * BW / (W2 * W);
            real j22 = BW * BW;
            real det = j11 * j22 - j12 * j21;
            real dW = -(j22 * f1 - j12 * f2) / det;
            real dv = -(j11 * f2 - j21 * f1) / det;
            real Wn = W + dW;
            real vn = vsq + dv;
            if (vn < 0.0) vn = 0.0;
            if (vn > vsqmax) vn = vsqmax;
            if (!(Wn > 0.0)) break;
            real err = fabs(Wn - W) / Wn + fabs(vn - vsq);
            W = Wn;
            vsq = vn;
            if (err < C2P_TOL) {
                ok = 1;
                break;
            }
        }
        if (it > C2P_NMAX) it = C2P_NMAX;
    }
    if (entropy_only) it = 0;
    *iters = it;
    real rho = 0.0, u = 0.0;
    if (ok) {
        real sq = sqrt(1.0 - vsq);
        real p = gfac * (W * (1.0 - vsq) - D * sq);
        rho = D * sq;
        u = p / (gam - 1.0);
        if (!(rho > 0.0) || !(u > 0.0)) ok = 0;
    }
    int status = C2P_OK;
    if (!ok) {
        /* entropy inversion */
        real kappa = Ucons[CENT] / Ucons[CRHO];
        const double gr = gam / (gam - 1.0);
        W = W0;
        int eok = 0;
        for (int k = 1; k <= C2P_NMAX; k++) {
            real W2 = W * W;
            real BW = Bsq + W;
            real num = Qtsq * W2 + QdotBsq * (Bsq + 2.0 * W);
            real den = W2 * BW * BW;
            real vs = num / den;
            real dnum = 2.0 * Qtsq * W + 2.0 * QdotBsq;
            real dden = 2.0 * W * BW * (Bsq + 2.0 * W);
            real dvs = (dnum * den - num * dden) / (den * den);
            if (vs > vsqmax) {
                vs = vsqmax;
                dvs = 0.0;
            }
            real s1 = 1.0 - vs;
            real sq = sqrt(s1);
            real rh = D * sq;
            real p = kappa * pow(rh, gam);
            real f = W * s1 - rh - gr * p;
            real drh = -0.5 * D / sq * dvs;
            real dp = gam * p / rh * drh;
            real df = s1 - W * dvs - drh - gr * dp;
            real Wn = W - f / df;
            if (!(Wn > 0.0)) break;
            real err = fabs(Wn - W) / Wn;
            W = Wn;
            if (err < C2P_TOL) {
                eok = 1;
                vsq = vs;
                break;
            }
        }
        if (eok) {
            /* final consistent v^2(W) */
            real W2 = W * W;
            real BW = Bsq + W;
            vsq = (Qtsq * W2 + QdotBsq * (Bsq + 2.0 * W)) / (W2 * BW * BW);
            if (vsq > vsqmax) vsq = vsqmax;
            real sq = sqrt(1.0 - vsq);
            rho = D * sq;
            u = kappa * pow(rho, gam) / (gam - 1.0);
            if (!(rho > 0.0) || !(u > 0.0) || !(vsq >= 0.0)) eok = 0;
        }
        if (!eok) return C2P_FAIL; /* keep the guess */
        status = C2P_ENTROPY;
    }
    real gamma = 1.0 / sqrt(1.0 - vsq);
    real pre = gamma / (W + Bsq);
    for (int i = 1; i < 4; i++) {
        real Qt = Qcon[i] - alpha * G.gcon[0][i] * Qdotn;
        pr[U1 + i - 1] = pre * (Qt + QdotB * Bn[i] / W);
    }
    pr[RHO] = rho;
    pr[UU] = u;
    return status;
}

/* Floors in the drift frame (Sec. 2.7: the paper injects the floor material
 * in the drift frame, after Ressler et al. 2017). Reading: the material the
 * floors add, drho = rho_f - rho and du = u_f - u (each >= 0), moves with the
 * drift velocity of the field lines, the part of the fluid's normal-frame
 * velocity across B, v_d = v - (v.Bn / Bn^2) Bn (which is E x B / B^2 for the
 * ideal-MHD E = -v x B; v_d = v where B = 0). Its stress-energy (no field) is
 * added to the current state's in conserved form, sqrt(-g)(rho u^t,
 * T^t_mu + rho u^t), the entropy slot keeps the current kappa, and the sum is
 * inverted with the same B, starting from the floored rho and u at the drift
 * velocity (the fluid's own velocity is a poor start where a fast flow along B
 * is slowed by much). So the
 * material brings no momentum along B: a flow along the field slows down as
 * mass is added instead of keeping its Lorentz factor (the runaway of
 * fluid-frame injection), and the motion across B is the field's. The
 * fluid-frame floor is applied to the result (mixing changes the Lorentz
 * factor, so rho and u can land slightly below the floors) and replaces the
 * whole step where the inversion fails. */
static bool drift_floor(const ora_desc& d, real* pr, const State& s, const Geom& G, real rf, real uf) {
    const double gam = d.gam;
    real drho = rf - pr[RHO], du = uf - pr[UU];
    if (drho < 0.0) drho = 0.0;
    if (du < 0.0) du = 0.0;
    real qsq = 0.0;
    for (int i = 1; i < 4; i++)
        for (int j = 1; j < 4; j++) qsq += G.gcov[i][j] * pr[U1 + i - 1] * pr[U1 + j - 1];
    real gamma = sqrt(1.0 + qsq);
    real v[4] = {0.0, pr[U1] / gamma, pr[U2] / gamma, pr[U3] / gamma};
    real Bn[4] = {0.0, G.alpha * pr[B1], G.alpha * pr[B2], G.alpha * pr[B3]};
    real bn2 = 0.0, vB = 0.0;
    for (int i = 1; i < 4; i++)
        for (int j = 1; j < 4; j++) {
            bn2 += G.gcov[i][j] * Bn[i] * Bn[j];
            vB += G.gcov[i][j] * v[i] * Bn[j];
        }
    real f = (bn2 > 0.0) ? vB / bn2 : real(0.0);
    real vd[4];
    for (int i = 1; i < 4; i++) vd[i] = v[i] - f * Bn[i];
    real vd2 = 0.0;
    for (int i = 1; i < 4; i++)
        for (int j = 1; j < 4; j++) vd2 += G.gcov[i][j] * vd[i] * vd[j];
    real gd = 1.0 / sqrt(1.0 - vd2);
    real pa[NPR] = {drho, du, gd * vd[1], gd * vd[2], gd * vd[3], 0.0, 0.0, 0.0};
    State sa;
    get_state(pa, G, sa);
    real uo[9], ua[9];
    prim_to_uf(pr, s, 0, gam, uo);
    prim_to_uf(pa, sa, 0, gam, ua);
    real U[NCONS];
    for (int m = 0; m < 5; m++) U[m] = G.gdet * (uo[m] + ua[m]);
    U[CENT] = G.gdet * uo[5] / uo[0] * (uo[0] + ua[0]);
    real q[NPR];
    for (int m = 0; m < NPR; m++) q[m] = pr[m];
    if (q[RHO] < rf) q[RHO] = rf;
    if (q[UU] < uf) q[UU] = uf;
    for (int i = 0; i < 3; i++) q[U1 + i] = pa[U1 + i]; /* start at the drift velocity */
    real Bc[3] = {pr[B1], pr[B2], pr[B3]};
    int its = 0;
    if (con2prim(d, U, Bc, G, q, &its) == C2P_FAIL) return false;
    if (q[RHO] < rf) q[RHO] = rf;
    if (q[UU] < uf) q[UU] = uf;
    for (int m = 0; m < 5; m++) pr[m] = q[m];
    return true;
}

/* Floors (Sec. 2.7): rho >= max(1e-7/r^2, b^2/50), u >= max(1e-9/r^(10/3), b^2/750),
 * b^2 of the state before the floors. ORA_FLOOR_FLUID raises rho and u and keeps
 * utilde^i (fluid-frame injection); ORA_FLOOR_DRIFT adds the material in the
 * drift frame (drift_floor above). */
static int apply_floors(const ora_desc& d, real* pr, const Geom& G, double r) {
    State s;
    get_state(pr, G, s);
    real rhoflr = 1.0e-7 / (r * r);
    real uflr = 1.0e-9 * std::pow(r, -10.0 / 3.0);
    real rb = s.bsq / 50.0, ub = s.bsq / 750.0;
    if (rb > rhoflr) rhoflr = rb;
    if (ub > uflr) uflr = ub;
    if (!(pr[RHO] < rhoflr) && !(pr[UU] < uflr)) return 0;
    if (d.floor_frame == ORA_FLOOR_DRIFT && drift_floor(d, pr, s, G, rhoflr, uflr)) return 1;
    if (pr[RHO] < rhoflr) pr[RHO] = rhoflr;
    if (pr[UU] < uflr) pr[UU] = uflr;
    return 1;
}

} /* namespace */

/* ------------------------------------------------------------------ */
/* grid                                                                  */
/* ------------------------------------------------------------------ */

struct ora_grid {
    ora_desc d;
    int n1p, n2p, n3p;
    long ncell;
    std::vector<double> prim, bface;
    std::vector<Geom> gc, gf1, gf2; /* (i,j) tables over the padded 2-D extent */
    std::vector<double> conn;       /* 64 per (i,j) centre */
    std::vector<double> rc;         /* r at centres */
    std::vector<int> status;        /* per cell: OR of the inversion/floor bits of the last step */
    long long stats[4];
    int smr_l2, smr_l3;             /* internal SMR in a block tree: log2 of the coarsest polar block's
                                       x2 and x3 cell widths over this block's (0 on a single block) */
};

namespace {

inline long cidx(const ora_grid* g, int i, int j, int k) {
    return ((long)(k + NG) * g->n2p + (j + NG)) * g->n1p + (i + NG);
}
inline long gidx(const ora_grid* g, int i, int j) { return (long)(j + NG) * g->n1p + (i + NG); }

void build_geometry(ora_grid* g) {
    const ora_desc& d = g->d;
    long n2d = (long)g->n1p * g->n2p;
    g->gc.resize(n2d);
    g->gf1.resize(n2d);
    g->gf2.resize(n2d);
    g->conn.resize(n2d * 64);
    g->rc.resize(n2d);
    for (int j = -NG; j < d.n2 + NG; j++)
        for (int i = -NG; i < d.n1 + NG; i++) {
            long q = gidx(g, i, j);
            double x1c = d.x1min + (i + 0.5) * d.dx1, x2c = d.x2min + (j + 0.5) * d.dx2;
            double x1f = d.x1min + i * d.dx1, x2f = d.x2min + j * d.dx2;
            geom_point(d, x1c, x2c, g->gc[q]);
            geom_point(d, x1f, x2c, g->gf1[q]);
            geom_point(d, x1c, x2f, g->gf2[q]);
            if ((d.bc[2] == ORA_BC_POLAR && j == 0) || (d.bc[3] == ORA_BC_POLAR && j == d.n2)) {
                g->gf2[q].pole = 1;
                g->gf2[q].gdet = 0.0;
            }
            double cn[4][4][4];
            conn_point(d, x1c, x2c, cn);
            std::memcpy(&g->conn[q * 64], cn, sizeof(cn));
            g->rc[q] = (d.metric != ORA_METRIC_MINKOWSKI) ? std::exp(x1c) : 1.0;
        }
}

/* Boundary conditions (Sec. 3.3 transmissive pole; radial outflow; periodic
 * phi). Reading: applied direction by direction in the order x3, x2, x1, each
 * pass over the full padded extent of the other two directions, so corner
 * ghosts take the composition of the three maps.
 * Polar: ghost cell (j = -1-m, k) takes interior (j = m, k + n3/2) with
 * utilde^2 and B^2 negated (the theta basis vector flips across the axis);
 * ghost x2-faces likewise (Bbar^2 negated); faces on the axis hold 0.
 * Outflow: copy the last interior cell (faces: the last interior face);
 * OUTFLOW_NOINFLOW also clamps utilde^1 so that nothing flows in.
 * Periodic: copy from the other end (face n equals face 0). */
int bc_cell_src(int bc, int n, int gi) {
    if (bc == ORA_BC_PERIODIC) return gi < 0 ? gi + n : gi - n;
    if (bc == ORA_BC_POLAR) return gi < 0 ? -1 - gi : 2 * n - 1 - gi;
    return gi < 0 ? 0 : n - 1;
}
int bc_face_src(int bc, int n, int gf) {
    if (bc == ORA_BC_PERIODIC) return gf < 0 ? gf + n : gf - n;
    if (bc == ORA_BC_POLAR) return gf < 0 ? -gf : 2 * n - gf;
    return gf < 0 ? 0 : n;
}

void apply_bc(ora_grid* g, double* P, double* Bf) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    const int nn[4] = {0, d.n1, d.n2, d.n3};
    for (int e = 3; e >= 1; e--) {
        const int ta = (e == 1) ? 2 : 1, tb = (e == 3) ? 2 : 3;
        for (int side = 0; side < 2; side++) {
            const int bc = d.bc[2 * (e - 1) + side];
            const bool polar = (bc == ORA_BC_POLAR);
            for (int b = -NG; b < nn[tb] + NG; b++)
                for (int a = -NG; a < nn[ta] + NG; a++) {
                    int src_ab[4] = {0, 0, 0, 0};
                    src_ab[ta] = a;
                    src_ab[tb] = b;
                    if (polar) { /* phi shift by pi across the axis (e == 2) */
                        src_ab[3] = ((src_ab[3] + d.n3 / 2) % d.n3 + d.n3) % d.n3;
                    }
                    for (int m = 0; m < NG; m++) {
                        /* cells and the cell-like face arrays (d != e) */
                        int gi = (side == 0) ? -1 - m : nn[e] + m;
                        int si = bc_cell_src(bc, nn[e], gi);
                        int dd[4] = {0, 0, 0, 0}, ss[4] = {0, src_ab[1], src_ab[2], src_ab[3]};
                        dd[ta] = a;
                        dd[tb] = b;
                        dd[e] = gi;
                        ss[e] = si;
                        long dst = cidx(g, dd[1], dd[2], dd[3]), src = cidx(g, ss[1], ss[2], ss[3]);
                        for (int v = 0; v < NPR; v++) P[v * nc + dst] = P[v * nc + src];
                        if (polar) {
                            P[U2 * nc + dst] = -P[U2 * nc + dst];
                            P[B2 * nc + dst] = -P[B2 * nc + dst];
                        }
                        if (bc == ORA_BC_OUTFLOW_NOINFLOW && e == 1) {
                            if (side == 1 && P[U1 * nc + dst] < 0.0) P[U1 * nc + dst] = 0.0;
                            if (side == 0 && P[U1 * nc + dst] > 0.0) P[U1 * nc + dst] = 0.0;
                        }
                        for (int f = 1; f <= 3; f++)
                            if (f != e) Bf[(f - 1) * nc + dst] = Bf[(f - 1) * nc + src];
                        /* the face array of direction e: ghost faces -1..-3, n+1..n+2;
                         * periodic also copies face 0 onto face n */
                        int gf = (side == 0) ? -1 - m : nn[e] + (bc == ORA_BC_PERIODIC ? 0 : 1) + m;
                        if (gf >= nn[e] + NG) continue;
                        int sf = bc_face_src(bc, nn[e], gf);
                        dd[e] = gf;
                        ss[e] = sf;
                        dst = cidx(g, dd[1], dd[2], dd[3]);
                        src = cidx(g, ss[1], ss[2], ss[3]);
                        Bf[(e - 1) * nc + dst] = polar ? -Bf[(e - 1) * nc + src] : Bf[(e - 1) * nc + src];
                    }
                    if (polar) { /* the axis face itself */
                        int dd[4] = {0, 0, 0, 0};
                        dd[ta] = a;
                        dd[tb] = b;
                        dd[e] = (side == 0) ? 0 : nn[e];
                        Bf[(e - 1) * nc + cidx(g, dd[1], dd[2], dd[3])] = 0.0;
                    }
                }
        }
    }
}

/* centre B^i = (Bbar^i_lo + Bbar^i_hi) / 2 / sqrt(-g)_centre (Sec. 2.5) */
void centre_b(ora_grid* g, const double* Bf, int i, int j, int k, real Bc[3]) {
    const long nc = g->ncell;
    real gd = g->gc[gidx(g, i, j)].gdet;
    Bc[0] = 0.5 * (real(Bf[0 * nc + cidx(g, i, j, k)]) + real(Bf[0 * nc + cidx(g, i + 1, j, k)])) / gd;
    Bc[1] = 0.5 * (real(Bf[1 * nc + cidx(g, i, j, k)]) + real(Bf[1 * nc + cidx(g, i, j + 1, k)])) / gd;
    Bc[2] = 0.5 * (real(Bf[2 * nc + cidx(g, i, j, k)]) + real(Bf[2 * nc + cidx(g, i, j, k + 1)])) / gd;
}

void load_prim(const ora_grid* g, const double* P, long c, real* pr) {
    for (int v = 0; v < NPR; v++) pr[v] = P[v * g->ncell + c];
}

/* A stage of the midpoint scheme (Sec. 2.1, 2.5) in its four phases:
 *   stage_fluxes: edge values and face fluxes from (Pf, Bff) [ghosts filled];
 *   stage_emf:    edge EMFs from the face fluxes;
 *   stage_ct:     Bf_out = Bf_base + dts * curl E;
 *   stage_update: U = U(P_base) + dts (-div F + Q(Pf)); P_out = con2prim(U,
 *                 centre B of Bf_out) with guess Pf; floors. */
typedef std::vector<double> Fluxes[4];

void stage_fluxes(ora_grid* g, const double* Pf, const double* Bff, Fluxes& F) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    const int nn[4] = {0, d.n1, d.n2, d.n3};
    for (int dir = 1; dir <= 3; dir++) F[dir].assign((size_t)NFX * nc, 0.0);

    /* the entropy tracer kappa = p / rho^gam of every cell, ghosts included: the
     * face fluxes take reconstructed values of it, like the primitives (reading:
     * the paper leaves the face value of kappa open; this takes one power per
     * cell, not one per face side) */
    phase_begin();
    std::vector<real> kcell((size_t)nc);
    for (long c = 0; c < nc; c++) kcell[c] = (d.gam - 1.0) * real(Pf[UU * nc + c]) / pow(real(Pf[RHO * nc + c]), d.gam);
    phase_end(0);

    /* fluxes: dir-faces over the interior faces, one transverse ghost layer */
    for (int dir = 1; dir <= 3; dir++) {
        int lo[4], hi[4]; /* inclusive face/cell ranges */
        for (int e = 1; e <= 3; e++) {
            lo[e] = (e == dir) ? 0 : -1;
            hi[e] = (e == dir) ? nn[e] : nn[e];
        }
        int L = nn[dir] + 2 * NG;
        std::vector<real> q(L), al(L), ar(L);
        std::vector<real> PL((size_t)NPR * L), PR((size_t)NPR * L), KL(L), KR(L);
        /* loop over lines along dir */
        int ta = (dir == 1) ? 2 : 1, tb = (dir == 3) ? 2 : 3;
        std::vector<real> flat(L, real(0.0));
        for (int b = lo[tb]; b <= hi[tb]; b++)
            for (int a = lo[ta]; a <= hi[ta]; a++) {
                phase_begin();
                if (d.flatten && d.recon == ORA_RECON_PPM) {
                    std::vector<real> uu(L), ww(L);
                    for (int c = 0; c < L; c++) {
                        int ii[4];
                        ii[dir] = c - NG;
                        ii[ta] = a;
                        ii[tb] = b;
                        const size_t ci = cidx(g, ii[1], ii[2], ii[3]);
                        uu[c] = Pf[UU * nc + ci];
                        ww[c] = Pf[(U1 + dir - 1) * nc + ci];
                    }
                    flatten_line(L, d.gam, uu.data(), ww.data(), flat.data());
                }
                for (int v = 0; v < NPR; v++) {
                    if (v == B1 + dir - 1) continue;
                    for (int c = 0; c < L; c++) {
                        int ii[4];
                        ii[dir] = c - NG;
                        ii[ta] = a;
                        ii[tb] = b;
                        q[c] = Pf[v * nc + cidx(g, ii[1], ii[2], ii[3])];
                    }
                    recon_line_impl(d.recon, L, q.data(), al.data(), ar.data(),
                                    (d.flatten && d.recon == ORA_RECON_PPM) ? flat.data() : nullptr);
                    for (int c = 0; c < L; c++) {
                        PL[(size_t)v * L + c] = al[c];
                        PR[(size_t)v * L + c] = ar[c];
                    }
                }
                for (int c = 0; c < L; c++) {  /* the cells' kappa along the line */
                    int ii[4];
                    ii[dir] = c - NG;
                    ii[ta] = a;
                    ii[tb] = b;
                    q[c] = kcell[cidx(g, ii[1], ii[2], ii[3])];
                }
                recon_line_impl(d.recon, L, q.data(), KL.data(), KR.data(),
                                (d.flatten && d.recon == ORA_RECON_PPM) ? flat.data() : nullptr);
                phase_end(0);
                phase_begin();
                for (int f = lo[dir]; f <= hi[dir]; f++) {
                    int ii[4];
                    ii[dir] = f;
                    ii[ta] = a;
                    ii[tb] = b;
                    long fi = cidx(g, ii[1], ii[2], ii[3]);
                    const Geom& G = (dir == 1)   ? g->gf1[gidx(g, ii[1], ii[2])]
                                    : (dir == 2) ? g->gf2[gidx(g, ii[1], ii[2])]
                                                 : g->gc[gidx(g, ii[1], ii[2])];
                    real pl[NPR], pr[NPR];
                    int cl = f - 1 + NG, cr = f + NG; /* line positions of the two cells */
                    for (int v = 0; v < NPR; v++) {
                        if (v == B1 + dir - 1) continue;
                        pl[v] = PR[(size_t)v * L + cl]; /* right edge of the left cell */
                        pr[v] = PL[(size_t)v * L + cr]; /* left edge of the right cell */
                    }
                    real fx[NFX];
                    if (G.pole) {
                        for (int m = 0; m < NFX; m++) fx[m] = 0.0;
                    } else {
                        real bn = real(Bff[(dir - 1) * nc + fi]) / G.gdet;
                        pl[B1 + dir - 1] = bn;
                        pr[B1 + dir - 1] = bn;
                        const real kap[2] = {KR[cl], KL[cr]};
                        face_flux(d, pl, pr, G, dir, fx, kap);
                    }
                    for (int m = 0; m < NFX; m++) F[dir][(size_t)m * nc + fi] = tod(fx[m]);
                }
                phase_end(1);
            }
    }
}

/* EMFs at edges (Sec. 2.5, the 4-flux average). Reading: E1 and E3 on the
 * polar axis are 0, which keeps Bbar^2 = 0 on axis faces and div B intact.
 * E holds three fields E1, E2, E3 (edge (i, j-1/2, k-1/2) etc. at index (i,j,k)).
 *
 * Upwinded EMFs (the paper's usual setting, the figure caption of Sec. 2.5
 * and the text after the EMF equations: Gardiner & Stone 2005). For an
 * edge between directions p and q, with e_p the EMF value a p-face carries
 * (its B-flux entry with the EMF's sign), e_q likewise, and E_c the EMF of
 * the cell-centred state (sqrt(-g)(b^m u^n - b^n u^m) for the edge's
 * component), the average of the four faces gets two corrections:
 *   E = 1/4 [sum of the 4 face values]
 *     + 1/4 [D_q(q-3/4) - D_q(q-1/4)] + 1/4 [D_p(p-3/4) - D_p(p-1/4)],
 *   D_q(q-1/4) = E_c(c, q) - e_q(c, q-1/2),  D_q(q-3/4) = e_q(c, q-1/2) - E_c(c, q-1)
 * (half-cell differences toward the edge along q) taken in the cell column
 * c = p-1 or p upwind of the mass flux through the p-face next to it (the
 * average of both when that flux is zero); D_p likewise along p, upwind of
 * the mass flux through the q-faces. */
namespace {
/* E_c of the three edge components at every cell of the padded block from the stage state */
void cell_emfs(ora_grid* g, const double* P, std::vector<double>& Ec) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    Ec.assign((size_t)3 * nc, 0.0);
    for (int k = -1; k <= d.n3; k++)
        for (int j = -1; j <= d.n2; j++)
            for (int i = -1; i <= d.n1; i++) {
                long c = cidx(g, i, j, k);
                const Geom& G = g->gc[gidx(g, i, j)];
                real pr[NPR];
                load_prim(g, P, c, pr);
                State s;
                get_state(pr, G, s);
                /* E1 ~ b^2 u^3 - b^3 u^2, E2 ~ b^3 u^1 - b^1 u^3, E3 ~ b^1 u^2 - b^2 u^1, times sqrt(-g) */
                Ec[c] = tod((s.bcon[2] * s.ucon[3] - s.bcon[3] * s.ucon[2]) * G.gdet);
                Ec[nc + c] = tod((s.bcon[3] * s.ucon[1] - s.bcon[1] * s.ucon[3]) * G.gdet);
                Ec[2 * nc + c] = tod((s.bcon[1] * s.ucon[2] - s.bcon[2] * s.ucon[1]) * G.gdet);
            }
}

/* upwind choice of two half-cell differences by the sign of a mass flux */
real upwind(real mass_flux, real lower, real upper) {
    if (mass_flux > 0.0) return lower;
    if (mass_flux < 0.0) return upper;
    return 0.5 * (lower + upper);
}
}  // namespace

void stage_emf(ora_grid* g, const Fluxes& F, const double* Pf, std::vector<double>& E) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
    phase_begin();
    E.assign((size_t)3 * nc, 0.0);
    double* E1 = E.data();
    double* E2 = E.data() + nc;
    double* E3 = E.data() + 2 * nc;
    auto FX = [&](int dir, int slot, int i, int j, int k) -> real {
        return real(F[dir][(size_t)slot * nc + cidx(g, i, j, k)]);
    };
    const int s3B2 = bslot(3, 2), s2B3 = bslot(2, 3), s1B3 = bslot(1, 3), s3B1 = bslot(3, 1),
              s2B1 = bslot(2, 1), s1B2 = bslot(1, 2);
    std::vector<double> Ec;
    const bool up = (d.emf == ORA_EMF_UPWIND);
    if (up) cell_emfs(g, Pf, Ec);
    /* the Gardiner-Stone corrections of one edge: component a (0..2) with face directions p, q;
     * ep(dp, dq) / eq(dp, dq): the p- / q-face values at offsets from the edge's cell (i, j, k),
     * mass fluxes likewise; ec(dp, dq) the cell-centred EMF */
    auto gs = [&](int a, int p, int q, int i, int j, int k, auto ep, auto eq) -> real {
        int I[4] = {0, i, j, k};
        auto at = [&](int dp, int dq) {  /* cell index offset along p and q */
            int J[4] = {0, I[1], I[2], I[3]};
            J[p] += dp;
            J[q] += dq;
            return cidx(g, J[1], J[2], J[3]);
        };
        auto ec = [&](int dp, int dq) { return real(Ec[(size_t)a * nc + at(dp, dq)]); };
        auto mp = [&](int dp, int dq) { return real(F[p][at(dp, dq)]); }; /* mass flux through a p-face */
        auto mq = [&](int dp, int dq) { return real(F[q][at(dp, dq)]); };
        /* along q, column c = p-1 (dp = -1) or p (dp = 0), upwind of the p-face mass flux */
        real dq_lo = upwind(mp(0, -1), eq(-1, 0) - ec(-1, -1), eq(0, 0) - ec(0, -1)); /* D_q(q-3/4) */
        real dq_hi = upwind(mp(0, 0), ec(-1, 0) - eq(-1, 0), ec(0, 0) - eq(0, 0));   /* D_q(q-1/4) */
        real dp_lo = upwind(mq(-1, 0), ep(0, -1) - ec(-1, -1), ep(0, 0) - ec(-1, 0)); /* D_p(p-3/4) */
        real dp_hi = upwind(mq(0, 0), ec(0, -1) - ep(0, -1), ec(0, 0) - ep(0, 0));   /* D_p(p-1/4) */
        return 0.25 * (dq_lo - dq_hi) + 0.25 * (dp_lo - dp_hi);
    };
    for (int k = 0; k <= n3; k++)
        for (int j = 0; j <= n2; j++)
            for (int i = 0; i <= n1; i++) {
                long e = cidx(g, i, j, k);
                bool axis = (d.bc[2] == ORA_BC_POLAR && j == 0) || (d.bc[3] == ORA_BC_POLAR && j == n2);
                if (i < n1) {
                    real v = 0.25 * (FX(3, s3B2, i, j, k) + FX(3, s3B2, i, j - 1, k) - FX(2, s2B3, i, j, k - 1) -
                                     FX(2, s2B3, i, j, k));
                    if (up) /* p = x2 faces (value -F2(B3)), q = x3 faces (value F3(B2)) */
                        v = v + gs(0, 2, 3, i, j, k,
                                   [&](int dp, int dq) { return -FX(2, s2B3, i, j + dp, k + dq); },
                                   [&](int dp, int dq) { return FX(3, s3B2, i, j + dp, k + dq); });
                    E1[e] = axis ? 0.0 : tod(v);
                }
                if (j < n2) {
                    real v = 0.25 * (FX(1, s1B3, i, j, k - 1) + FX(1, s1B3, i, j, k) - FX(3, s3B1, i, j, k) -
                                     FX(3, s3B1, i - 1, j, k));
                    if (up) /* p = x1 faces (value F1(B3)), q = x3 faces (value -F3(B1)) */
                        v = v + gs(1, 1, 3, i, j, k,
                                   [&](int dp, int dq) { return FX(1, s1B3, i + dp, j, k + dq); },
                                   [&](int dp, int dq) { return -FX(3, s3B1, i + dp, j, k + dq); });
                    E2[e] = tod(v);
                }
                if (k < n3) {
                    real v = 0.25 * (FX(2, s2B1, i - 1, j, k) + FX(2, s2B1, i, j, k) - FX(1, s1B2, i, j, k) -
                                     FX(1, s1B2, i, j - 1, k));
                    if (up) /* p = x1 faces (value -F1(B2)), q = x2 faces (value F2(B1)) */
                        v = v + gs(2, 1, 2, i, j, k,
                                   [&](int dp, int dq) { return -FX(1, s1B2, i + dp, j + dq, k); },
                                   [&](int dp, int dq) { return FX(2, s2B1, i + dp, j + dq, k); });
                    E3[e] = axis ? 0.0 : tod(v);
                }
            }

    phase_end(2);
}

/* staggered face update (Sec. 2.5, the three CT equations) */
void stage_ct(ora_grid* g, const std::vector<double>& E, const double* Bfb, double dts, double* Bfout) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
    const double* E1 = E.data();
    const double* E2 = E.data() + nc;
    const double* E3 = E.data() + 2 * nc;
    phase_begin();
    for (int v = 0; v < 3; v++)
        for (long c = 0; c < nc; c++) Bfout[v * nc + c] = Bfb[v * nc + c];
    for (int k = 0; k <= n3; k++)
        for (int j = 0; j <= n2; j++)
            for (int i = 0; i <= n1; i++) {
                long c = cidx(g, i, j, k);
                if (j < n2 && k < n3) {
                    real r = (real(E2[cidx(g, i, j, k + 1)]) - real(E2[c])) / d.dx3 -
                             (real(E3[cidx(g, i, j + 1, k)]) - real(E3[c])) / d.dx2;
                    Bfout[0 * nc + c] = tod(real(Bfb[0 * nc + c]) + dts * r);
                }
                if (i < n1 && k < n3) {
                    bool axis = (d.bc[2] == ORA_BC_POLAR && j == 0) || (d.bc[3] == ORA_BC_POLAR && j == n2);
                    real r = (real(E3[cidx(g, i + 1, j, k)]) - real(E3[c])) / d.dx1 -
                             (real(E1[cidx(g, i, j, k + 1)]) - real(E1[c])) / d.dx3;
                    Bfout[1 * nc + c] = axis ? 0.0 : tod(real(Bfb[1 * nc + c]) + dts * r);
                }
                if (i < n1 && j < n2) {
                    real r = (real(E1[cidx(g, i, j + 1, k)]) - real(E1[c])) / d.dx2 -
                             (real(E2[cidx(g, i + 1, j, k)]) - real(E2[c])) / d.dx1;
                    Bfout[2 * nc + c] = tod(real(Bfb[2 * nc + c]) + dts * r);
                }
            }

    phase_end(3);
}

/* cell update, inversion, floors */
/* Internal SMR (Sec. 3.3.2: phi-averaging within polar blocks; the paper
 * averages "the fluxes and conserved quantities"). Reading: with n_max
 * levels, a row of cells at distance jp (in cells) from a polar face is
 * grouped into cells 2^n wide in phi, n the largest level in 1..n_max with
 * jp < 2^(n_max - n) (rows farther out: no grouping). A group acts as one
 * cell. Its field changes as a wide cell's: the EMFs (the fluxes of the
 * induction equation) are averaged before the face update (smr_emf), so
 * the change of every x1- and x2-face of a group is its group mean and the
 * change of its inner x3-faces is linear between its outer ones, and div B
 * stays at round-off under CT. Its fluid state: after the cell update the
 * group's conserved variables are averaged and inverted once (start: the
 * mean of the cells' primitives, field: the mean of their centre fields),
 * and every cell of the group takes the result (its own centre field
 * kept). The CFL rate uses the group's width in x3. Returns the group width
 * of row j (1: none).
 *
 * In a block tree the rows and widths are those of the coarsest polar
 * blocks (reading: the paper counts cells from the pole without saying at
 * which resolution). A polar block whose x2 cells are 2^l2 times finer and x3
 * cells 2^l3 times finer than theirs groups its row j as their row
 * j / 2^l2, with 2^l3 times as many of its own cells, so the groups of blocks
 * that meet at a face cover the same phi ranges and the EMFs that blocks
 * exchange (edge synchronisation, refluxing) are averaged alike on both
 * sides. */
int smr_width(const ora_grid* g, int j) {
    const ora_desc& d = g->d;
    if (d.smr <= 0) return 1;
    int jp = 1 << 30;
    if (d.bc[2] == ORA_BC_POLAR) jp = j;
    if (d.bc[3] == ORA_BC_POLAR) jp = std::min(jp, d.n2 - 1 - j);
    const int jb = jp >> g->smr_l2;
    for (int n = d.smr; n >= 1; n--)
        if (jb < (1 << (d.smr - n))) return (1 << n) << g->smr_l3;
    return 1;
}

/* sum of w = 2^n values as a balanced binary tree: w equal values sum to
 * exactly w times the value, so a group mean of equal values is that value */
double pair_sum(const double* a, int w) { return (w == 1) ? a[0] : pair_sum(a, w / 2) + pair_sum(a + w / 2, w / 2); }

/* group width of the EMF line at x2-edge je: that of the adjacent row
 * closer to the pole (the wider one) */
int smr_line_width(const ora_grid* g, int je) {
    int w = 1;
    if (je >= 1) w = std::max(w, smr_width(g, je - 1));
    if (je < g->d.n2) w = std::max(w, smr_width(g, je));
    return w;
}

/* the EMFs of grouped rows as a wide cell's (smr_width): along each x2-line
 * of edges with group width W, the x3-edge EMFs E3 take their group mean
 * and the x1-edge EMFs E1 inside a group are linear between the group's two
 * outer ones; inside each grouped row the x2-edge EMFs E2 are linear
 * between the group's outer ones. Then the CT changes of a group's x1- and
 * x2-faces are uniform and those of its inner x3-faces linear. */
void smr_emf(ora_grid* g, std::vector<double>& E) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    double* E1 = E.data();
    double* E2 = E.data() + nc;
    double* E3 = E.data() + 2 * nc;
    std::vector<double> a;
    for (int je = 0; je <= d.n2; je++) {
        const int W = smr_line_width(g, je);
        if (W == 1) continue;
        a.resize(W);
        for (int k0 = 0; k0 < d.n3; k0 += W) {
            for (int i = 0; i <= d.n1; i++) {
                for (int m = 0; m < W; m++) a[m] = E3[cidx(g, i, je, k0 + m)];
                const double s3 = pair_sum(a.data(), W);
                for (int m = 0; m < W; m++) E3[cidx(g, i, je, k0 + m)] = s3 / W;
            }
            for (int i = 0; i < d.n1; i++) {
                const double e0 = E1[cidx(g, i, je, k0)], ew = E1[cidx(g, i, je, k0 + W)];
                for (int m = 1; m < W; m++) E1[cidx(g, i, je, k0 + m)] = e0 + (ew - e0) * m / W;
            }
        }
    }
    for (int j = 0; j < d.n2; j++) {
        const int w = smr_width(g, j);
        if (w == 1) continue;
        for (int k0 = 0; k0 < d.n3; k0 += w)
            for (int i = 0; i <= d.n1; i++) {
                const double e0 = E2[cidx(g, i, j, k0)], ew = E2[cidx(g, i, j, k0 + w)];
                for (int m = 1; m < w; m++) E2[cidx(g, i, j, k0 + m)] = e0 + (ew - e0) * m / w;
            }
    }
}

void stage_update(ora_grid* g, const Fluxes& F, const double* Pb, const double* Pf, const double* Bfout, double dts,
                  double* Pout) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    const int n1 = d.n1, n2 = d.n2, n3 = d.n3;
    const double dx[4] = {0.0, d.dx1, d.dx2, d.dx3};
    std::vector<double> Usmr(d.smr > 0 ? (size_t)NCONS * nc : 0);
    phase_begin();
    for (int k = 0; k < n3; k++)
        for (int j = 0; j < n2; j++)
            for (int i = 0; i < n1; i++) {
                long c = cidx(g, i, j, k);
                long q2 = gidx(g, i, j);
                const Geom& G = g->gc[q2];
                real pb[NPR], pf[NPR];
                load_prim(g, Pb, c, pb);
                load_prim(g, Pf, c, pf);
                State sb, sf;
                get_state(pb, G, sb);
                get_state(pf, G, sf);
                real u9[9];
                prim_to_uf(pb, sb, 0, d.gam, u9);
                real Q[NCONS];
                double cn[4][4][4];
                std::memcpy(cn, &g->conn[q2 * 64], sizeof(cn));
                source_terms(d, pf, sf, G, cn, Q);
                real U[NCONS];
                long c1 = cidx(g, i + 1, j, k), c2 = cidx(g, i, j + 1, k), c3 = cidx(g, i, j, k + 1);
                for (int m = 0; m < NCONS; m++) {
                    real div = (real(F[1][(size_t)m * nc + c1]) - real(F[1][(size_t)m * nc + c])) / dx[1] +
                               (real(F[2][(size_t)m * nc + c2]) - real(F[2][(size_t)m * nc + c])) / dx[2] +
                               (real(F[3][(size_t)m * nc + c3]) - real(F[3][(size_t)m * nc + c])) / dx[3];
                    U[m] = u9[m] * G.gdet + dts * (Q[m] - div);
                }
                if (smr_width(g, j) > 1) { /* inverted with its group below */
                    for (int m = 0; m < NCONS; m++) Usmr[(size_t)m * nc + c] = tod(U[m]);
                    continue;
                }
                real Bc[3];
                centre_b(g, Bfout, i, j, k, Bc);
                real pr[NPR];
                for (int v = 0; v < NPR; v++) pr[v] = pf[v];
                pr[B1] = Bc[0];
                pr[B2] = Bc[1];
                pr[B3] = Bc[2];
                int its = 0;
                int st = con2prim(d, U, Bc, G, pr, &its);
                if (st == C2P_FAIL) {
                    for (int v = 0; v < 5; v++) pr[v] = pf[v];
                }
                g->stats[st == C2P_OK ? 0 : (st == C2P_ENTROPY ? 1 : 2)]++;
                g->status[c] |= st;
                if (d.floors && apply_floors(d, pr, G, g->rc[q2])) {
                    g->stats[3]++;
                    g->status[c] |= C2P_FLOOR;
                }
                for (int v = 0; v < NPR; v++) Pout[v * nc + c] = tod(pr[v]);
            }
    /* internal SMR groups: one inversion of the group's mean state */
    for (int j = 0; j < n2; j++) {
        const int w = smr_width(g, j);
        if (w == 1) continue;
        for (int k0 = 0; k0 < n3; k0 += w)
            for (int i = 0; i < n1; i++) {
                const long q2 = gidx(g, i, j);
                const Geom& G = g->gc[q2];
                real U[NCONS], Bc[3] = {0.0, 0.0, 0.0}, pr[NPR];
                for (int m = 0; m < NCONS; m++) U[m] = 0.0;
                for (int v = 0; v < NPR; v++) pr[v] = 0.0;
                for (int q = 0; q < w; q++) {
                    const long c = cidx(g, i, j, k0 + q);
                    for (int m = 0; m < NCONS; m++) U[m] += Usmr[(size_t)m * nc + c];
                    real b[3];
                    centre_b(g, Bfout, i, j, k0 + q, b);
                    for (int e = 0; e < 3; e++) Bc[e] += b[e];
                    for (int v = 0; v < 5; v++) pr[v] += Pf[v * nc + c];
                }
                for (int m = 0; m < NCONS; m++) U[m] /= w;
                for (int e = 0; e < 3; e++) Bc[e] /= w;
                for (int v = 0; v < 5; v++) pr[v] /= w;
                real pf[5];
                for (int v = 0; v < 5; v++) pf[v] = pr[v];
                pr[B1] = Bc[0];
                pr[B2] = Bc[1];
                pr[B3] = Bc[2];
                int its = 0;
                int st = con2prim(d, U, Bc, G, pr, &its);
                if (st == C2P_FAIL)
                    for (int v = 0; v < 5; v++) pr[v] = pf[v];
                int fl = (d.floors && apply_floors(d, pr, G, g->rc[q2])) ? 1 : 0;
                for (int q = 0; q < w; q++) {
                    const long c = cidx(g, i, j, k0 + q);
                    g->stats[st == C2P_OK ? 0 : (st == C2P_ENTROPY ? 1 : 2)]++;
                    g->status[c] |= st;
                    if (fl) {
                        g->stats[3]++;
                        g->status[c] |= C2P_FLOOR;
                    }
                    real b[3];
                    centre_b(g, Bfout, i, j, k0 + q, b);
                    for (int v = 0; v < 5; v++) Pout[v * nc + c] = tod(pr[v]);
                    for (int e = 0; e < 3; e++) Pout[(B1 + e) * nc + c] = tod(b[e]);
                }
            }
    }
    phase_end(4);
}

void stage(ora_grid* g, const double* Pf, const double* Bff, const double* Pb, const double* Bfb, double dts,
           double* Pout, double* Bfout) {
    Fluxes F;
    std::vector<double> E;
    stage_fluxes(g, Pf, Bff, F);
    stage_emf(g, F, Pf, E);
    if (g->d.smr > 0) smr_emf(g, E);
    stage_ct(g, E, Bfb, dts, Bfout);
    stage_update(g, F, Pb, Pf, Bfout, dts, Pout);
}

/* CFL time step (Sec. 2.1): per cell 1/dt = sum_i v_f^i / dx^i with
 * v_f^i = max(|v+|, |v-|) at the cell centre; dt = C0 / max over cells.
 * Reading: speeds are taken at cell centres from the current primitives. */
double grid_dt(ora_grid* g) {
    const ora_desc& d = g->d;
    const double dx[4] = {0.0, d.dx1, d.dx2, d.dx3};
    real invmax = 0.0;
    phase_begin();
    for (int k = 0; k < d.n3; k++)
        for (int j = 0; j < d.n2; j++)
            for (int i = 0; i < d.n1; i++) {
                const Geom& G = g->gc[gidx(g, i, j)];
                real pr[NPR];
                load_prim(g, g->prim.data(), cidx(g, i, j, k), pr);
                State s;
                get_state(pr, G, s);
                real inv = 0.0;
                for (int dir = 1; dir <= 3; dir++) {
                    real vp, vm;
                    vchar(pr, s, G, dir, d.gam, &vp, &vm);
                    real vf = fmax(fabs(vp), fabs(vm));
                    inv += vf / (dir == 3 ? dx[3] * smr_width(g, j) : dx[dir]);
                }
                if (inv > invmax) invmax = inv;
            }
    phase_end(5);
    return tod(d.cour / invmax);
}

} /* namespace */

/* ------------------------------------------------------------------ */
/* C interface                                                           */
/* ------------------------------------------------------------------ */

extern "C" {

void ora_geom(const ora_desc* d, double x1, double x2, double* gcov16, double* gcon16, double* gdet,
              double* alpha) {
    Geom G;
    geom_point(*d, x1, x2, G);
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            gcov16[4 * m + n] = tod(G.gcov[m][n]);
            gcon16[4 * m + n] = tod(G.gcon[m][n]);
        }
    *gdet = tod(G.gdet);
    *alpha = tod(G.alpha);
}

void ora_conn(const ora_desc* d, double x1, double x2, double* conn64) {
    double cn[4][4][4];
    conn_point(*d, x1, x2, cn);
    std::memcpy(conn64, cn, sizeof(cn));
}

void ora_state(const ora_desc* d, const double* pr8, double x1, double x2, double* ucon4, double* ucov4,
               double* bcon4, double* bcov4, double* bsq) {
    Geom G;
    geom_point(*d, x1, x2, G);
    real pr[NPR];
    for (int v = 0; v < NPR; v++) pr[v] = pr8[v];
    State s;
    get_state(pr, G, s);
    for (int m = 0; m < 4; m++) {
        ucon4[m] = tod(s.ucon[m]);
        ucov4[m] = tod(s.ucov[m]);
        bcon4[m] = tod(s.bcon[m]);
        bcov4[m] = tod(s.bcov[m]);
    }
    *bsq = tod(s.bsq);
}

void ora_p2uf(const ora_desc* d, const double* pr8, double x1, double x2, int dir, double* out9) {
    Geom G;
    geom_point(*d, x1, x2, G);
    real pr[NPR];
    for (int v = 0; v < NPR; v++) pr[v] = pr8[v];
    State s;
    get_state(pr, G, s);
    real o[9];
    prim_to_uf(pr, s, dir, d->gam, o);
    for (int m = 0; m < 9; m++) out9[m] = tod(o[m] * G.gdet);
}

void ora_vchar(const ora_desc* d, const double* pr8, double x1, double x2, int dir, double* vp, double* vm) {
    Geom G;
    geom_point(*d, x1, x2, G);
    real pr[NPR];
    for (int v = 0; v < NPR; v++) pr[v] = pr8[v];
    State s;
    get_state(pr, G, s);
    real a, b;
    vchar(pr, s, G, dir, d->gam, &a, &b);
    *vp = tod(a);
    *vm = tod(b);
}

void ora_face_flux(const ora_desc* d, const double* pl8, const double* pr8, double x1, double x2, int dir,
                   double* f8) {
    Geom G;
    geom_point(*d, x1, x2, G);
    real pl[NPR], pr[NPR], f[NFX];
    for (int v = 0; v < NPR; v++) {
        pl[v] = pl8[v];
        pr[v] = pr8[v];
    }
    face_flux(*d, pl, pr, G, dir, f);
    for (int m = 0; m < NFX; m++) f8[m] = tod(f[m]);
}

void ora_source(const ora_desc* d, const double* pr8, double x1, double x2, double* q6) {
    Geom G;
    geom_point(*d, x1, x2, G);
    double cn[4][4][4];
    conn_point(*d, x1, x2, cn);
    real pr[NPR];
    for (int v = 0; v < NPR; v++) pr[v] = pr8[v];
    State s;
    get_state(pr, G, s);
    real Q[NCONS];
    source_terms(*d, pr, s, G, cn, Q);
    for (int m = 0; m < NCONS; m++) q6[m] = tod(Q[m]);
}

void ora_recon_line(int recon, int n, const double* q, double* al, double* ar) {
    std::vector<real> qq(n), a(n, real(0.0)), b(n, real(0.0));
    for (int c = 0; c < n; c++) {
        qq[c] = q[c];
        a[c] = al[c];
        b[c] = ar[c];
    }
    recon_line_impl(recon, n, qq.data(), a.data(), b.data());
    for (int c = 0; c < n; c++) {
        al[c] = tod(a[c]);
        ar[c] = tod(b[c]);
    }
}

void ora_flatten_line(int n, double gam, const double* u, const double* w, double* f) {
    std::vector<real> uu(n), ww(n), ff(n);
    for (int c = 0; c < n; c++) {
        uu[c] = u[c];
        ww[c] = w[c];
    }
    flatten_line(n, gam, uu.data(), ww.data(), ff.data());
    for (int c = 0; c < n; c++) f[c] = tod(ff[c]);
}

void ora_recon_line_flat(int n, const double* q, const double* f, double* al, double* ar) {
    std::vector<real> qq(n), ff(n), a(n, real(0.0)), b(n, real(0.0));
    for (int c = 0; c < n; c++) {
        qq[c] = q[c];
        ff[c] = f[c];
        a[c] = al[c];
        b[c] = ar[c];
    }
    recon_line_impl(ORA_RECON_PPM, n, qq.data(), a.data(), b.data(), ff.data());
    for (int c = 0; c < n; c++) {
        al[c] = tod(a[c]);
        ar[c] = tod(b[c]);
    }
}

void ora_c2p_many(const ora_desc* d, long n, const double* U6, const double* Bc3, const double* x1,
                  const double* x2, double* pr8, int* status, int* iters, int entropy_only) {
    for (long s = 0; s < n; s++) {
        Geom G;
        geom_point(*d, x1[s], x2[s], G);
        real U[NCONS], Bc[3], pr[NPR];
        for (int m = 0; m < NCONS; m++) U[m] = U6[s * NCONS + m];
        for (int m = 0; m < 3; m++) Bc[m] = Bc3[s * 3 + m];
        for (int v = 0; v < NPR; v++) pr[v] = pr8[s * NPR + v];
        pr[B1] = Bc[0];
        pr[B2] = Bc[1];
        pr[B3] = Bc[2];
        int its = 0;
        int st = con2prim(*d, U, Bc, G, pr, &its, entropy_only);
        for (int v = 0; v < NPR; v++) pr8[s * NPR + v] = tod(pr[v]);
        status[s] = st;
        iters[s] = its;
    }
}

void ora_nh_map(double E, double S2, double T2, double B2, double D, double gam, double p, double* out3) {
    real W = 0.0, vsq = 0.0, pn = 0.0;
    const double vsqmax = 1.0 - 1.0 / (GAMMA_MAX * GAMMA_MAX);
    bool ok = nh_map(E, S2, T2, B2, D, (gam - 1.0) / gam, vsqmax, p, &W, &vsq, &pn);
    out3[0] = ok ? tod(W) : -1.0;
    out3[1] = tod(vsq);
    out3[2] = tod(pn);
}

void ora_floors_many(const ora_desc* d, long n, double* pr8, const double* x1, const double* x2, const double* r,
                     int* hit) {
    for (long s = 0; s < n; s++) {
        Geom G;
        geom_point(*d, x1[s], x2[s], G);
        real pr[NPR];
        for (int v = 0; v < NPR; v++) pr[v] = pr8[s * NPR + v];
        hit[s] = apply_floors(*d, pr, G, r[s]);
        for (int v = 0; v < NPR; v++) pr8[s * NPR + v] = tod(pr[v]);
    }
}

void ora_p2u_many(const ora_desc* d, long n, const double* pr8, const double* x1, const double* x2,
                  double* U6) {
    for (long s = 0; s < n; s++) {
        Geom G;
        geom_point(*d, x1[s], x2[s], G);
        real pr[NPR];
        for (int v = 0; v < NPR; v++) pr[v] = pr8[s * NPR + v];
        State st;
        get_state(pr, G, st);
        real o[9];
        prim_to_uf(pr, st, 0, d->gam, o);
        for (int m = 0; m < NCONS; m++) U6[s * NCONS + m] = tod(o[m] * G.gdet);
    }
}

/* ================================================================== */
/* Inputs and targets of the learned inversion guess.
 *
 * The network maps a conserved state (with its metric) to an initial guess
 * for the Newton inversion of Sec. 2.6. Its ten inputs are the scalars the
 * inversion works with, made dimensionless with D where they carry the
 * density scale (rho -> lambda rho, u -> lambda u, B -> sqrt(lambda) B
 * leaves W / D and v^2 unchanged), plus four metric invariants:
 *   f0 = ln D
 *   f1 = ln((-Q.n - D) / D)              energy beyond rest mass, per D
 *   f2 = ln(Qt^2 / D^2 + 1e-30)
 *   f3 = (Q.B)^2 / (Qt^2 B^2 + 1e-300)   cos^2 of the angle of Qt and B
 *   f4 = ln(U_kappa / U_rho) + (gam - 1) ln D = ln(kappa D^(gam - 1))
 *   f5 = ln(B^2 / D + 1e-30)
 *   f6 = alpha
 *   f7 = ln(beta_i beta^i + 1e-30),  beta^i = alpha^2 g^{ti}
 *   f8 = ln sqrt(gamma) = ln(sqrt(-g) / alpha)
 *   f9 = x1 (= ln r in Kerr-Schild)
 * (f1 is floored at ln 1e-30.) Targets: y0 = ln(W / D) = ln(h Gamma),
 * h = 1 + gam u / rho, and y1 = ln Gamma^2 = ln(1 + g_ij utilde^i utilde^j),
 * from which the guess is W = D e^y0, v^2 = 1 - e^-y1.
 * Reading: the paper has no learned guess; these definitions are this
 * project's. */
void ora_mlp_features(const ora_desc* d, long n, const double* U6, const double* Bc3, const double* x1,
                      const double* x2, double* f10) {
    for (long s = 0; s < n; s++) {
        Geom G;
        geom_point(*d, x1[s], x2[s], G);
        const double* U = U6 + s * NCONS;
        const double* Bc = Bc3 + s * 3;
        const double alpha = tod(G.alpha), gdet = tod(G.gdet);
        const double D = U[CRHO] * alpha / gdet;
        double Qcov[4] = {alpha * (U[CEN] - U[CRHO]) / gdet, alpha * U[CS1] / gdet, alpha * U[CS2] / gdet,
                          alpha * U[CS3] / gdet};
        double Qcon[4];
        for (int m = 0; m < 4; m++) {
            double t = 0.0;
            for (int k = 0; k < 4; k++) t += tod(G.gcon[m][k]) * Qcov[k];
            Qcon[m] = t;
        }
        const double Qdotn = -alpha * Qcon[0];
        double Qsq = 0.0;
        for (int m = 0; m < 4; m++) Qsq += Qcov[m] * Qcon[m];
        const double Qtsq = Qsq + Qdotn * Qdotn;
        const double Bn[4] = {0.0, alpha * Bc[0], alpha * Bc[1], alpha * Bc[2]};
        double Bsq = 0.0, QdotB = 0.0;
        for (int i = 1; i < 4; i++) {
            QdotB += Qcov[i] * Bn[i];
            for (int j = 1; j < 4; j++) Bsq += tod(G.gcov[i][j]) * Bn[i] * Bn[j];
        }
        double beta[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 1; i < 4; i++) beta[i] = alpha * alpha * tod(G.gcon[0][i]);
        double bsq = 0.0;
        for (int i = 1; i < 4; i++)
            for (int j = 1; j < 4; j++) bsq += tod(G.gcov[i][j]) * beta[i] * beta[j];
        double* f = f10 + s * 10;
        f[0] = std::log(D);
        f[1] = std::log(std::max(-Qdotn - D, 1e-30 * D) / D);
        f[2] = std::log(Qtsq / (D * D) + 1e-30);
        f[3] = QdotB * QdotB / (Qtsq * Bsq + 1e-300);
        f[4] = std::log(U[CENT] / U[CRHO]) + (d->gam - 1.0) * std::log(D);
        f[5] = std::log(Bsq / D + 1e-30);
        f[6] = alpha;
        f[7] = std::log(bsq + 1e-30);
        f[8] = std::log(gdet / alpha);
        f[9] = x1[s];
    }
}

void ora_mlp_targets(const ora_desc* d, long n, const double* pr8, const double* x1, const double* x2,
                     double* y2) {
    for (long s = 0; s < n; s++) {
        Geom G;
        geom_point(*d, x1[s], x2[s], G);
        const double* pr = pr8 + s * NPR;
        double qsq = 0.0;
        for (int i = 1; i < 4; i++)
            for (int j = 1; j < 4; j++) qsq += tod(G.gcov[i][j]) * pr[U1 + i - 1] * pr[U1 + j - 1];
        const double gamma = std::sqrt(1.0 + qsq);
        const double h = 1.0 + d->gam * pr[UU] / pr[RHO];
        y2[s * 2 + 0] = std::log(h * gamma);
        y2[s * 2 + 1] = std::log(1.0 + qsq);
    }
}

ora_grid* ora_grid_new(const ora_desc* d) {
    ora_grid* g = new ora_grid;
    g->d = *d;
    g->n1p = d->n1 + 2 * NG;
    g->n2p = d->n2 + 2 * NG;
    g->n3p = d->n3 + 2 * NG;
    g->ncell = (long)g->n1p * g->n2p * g->n3p;
    g->prim.assign((size_t)NPR * g->ncell, 0.0);
    g->bface.assign((size_t)3 * g->ncell, 0.0);
    g->status.assign(g->ncell, 0);
    for (int m = 0; m < 4; m++) g->stats[m] = 0;
    g->smr_l2 = g->smr_l3 = 0;
    build_geometry(g);
    return g;
}

void ora_grid_free(ora_grid* g) { delete g; }

void ora_grid_set(ora_grid* g, const double* prim, const double* bface) {
    std::memcpy(g->prim.data(), prim, sizeof(double) * NPR * g->ncell);
    std::memcpy(g->bface.data(), bface, sizeof(double) * 3 * g->ncell);
    const long nc = g->ncell;
    for (int k = 0; k < g->d.n3; k++)
        for (int j = 0; j < g->d.n2; j++)
            for (int i = 0; i < g->d.n1; i++) {
                real Bc[3];
                centre_b(g, g->bface.data(), i, j, k, Bc);
                long c = cidx(g, i, j, k);
                for (int m = 0; m < 3; m++) g->prim[(B1 + m) * nc + c] = tod(Bc[m]);
            }
    apply_bc(g, g->prim.data(), g->bface.data());
}

void ora_grid_get(const ora_grid* g, double* prim, double* bface) {
    std::memcpy(prim, g->prim.data(), sizeof(double) * NPR * g->ncell);
    std::memcpy(bface, g->bface.data(), sizeof(double) * 3 * g->ncell);
}

void ora_grid_bc(ora_grid* g) { apply_bc(g, g->prim.data(), g->bface.data()); }

double ora_grid_dt(ora_grid* g) { return grid_dt(g); }

/* One full midpoint step (Sec. 2.1): predictor to t + dt/2 with F(P^n),
 * corrector from U^n to t + dt with F(P^{n+1/2}); boundaries refreshed before
 * each stage. dt <= 0 takes the CFL step of the current state. */
double ora_grid_step(ora_grid* g, double dt) {
    for (int m = 0; m < 4; m++) g->stats[m] = 0;
    std::fill(g->status.begin(), g->status.end(), 0);
    apply_bc(g, g->prim.data(), g->bface.data());
    if (!(dt > 0.0)) dt = grid_dt(g);
    const size_t np = (size_t)NPR * g->ncell, nb = (size_t)3 * g->ncell;
    std::vector<double> Ph(g->prim), Bh(g->bface), Pn(np), Bn(nb);
    stage(g, g->prim.data(), g->bface.data(), g->prim.data(), g->bface.data(), 0.5 * dt, Ph.data(), Bh.data());
    apply_bc(g, Ph.data(), Bh.data());
    Pn = g->prim;
    Bn = g->bface;
    stage(g, Ph.data(), Bh.data(), g->prim.data(), g->bface.data(), dt, Pn.data(), Bn.data());
    g->prim.swap(Pn);
    g->bface.swap(Bn);
    apply_bc(g, g->prim.data(), g->bface.data());
    return dt;
}

void ora_grid_stats(const ora_grid* g, long long* counts4) {
    for (int m = 0; m < 4; m++) counts4[m] = g->stats[m];
}

/* per interior cell: OR over both stages of the last step of
 * 1 = entropy inversion used, 2 = both inversions failed, 4 = floor applied */
void ora_grid_status(const ora_grid* g, int* out) {
    const ora_desc& d = g->d;
    long o = 0;
    for (int k = 0; k < d.n3; k++)
        for (int j = 0; j < d.n2; j++)
            for (int i = 0; i < d.n1; i++) out[o++] = g->status[cidx(g, i, j, k)];
}

void ora_grid_fluxes(ora_grid* g, double* out) {
    apply_bc(g, g->prim.data(), g->bface.data());
    Fluxes F;
    stage_fluxes(g, g->prim.data(), g->bface.data(), F);
    const size_t n = (size_t)NFX * g->ncell;
    for (int dir = 1; dir <= 3; dir++) std::copy(F[dir].begin(), F[dir].end(), out + (dir - 1) * n);
}

/* discrete div B per interior cell: sum_d (Bbar^d_hi - Bbar^d_lo)/dx^d */
void ora_grid_divb(const ora_grid* g, double* divb) {
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    const double* B = g->bface.data();
    long o = 0;
    for (int k = 0; k < d.n3; k++)
        for (int j = 0; j < d.n2; j++)
            for (int i = 0; i < d.n1; i++) {
                long c = cidx(g, i, j, k);
                divb[o++] = (B[0 * nc + cidx(g, i + 1, j, k)] - B[0 * nc + c]) / d.dx1 +
                            (B[1 * nc + cidx(g, i, j + 1, k)] - B[1 * nc + c]) / d.dx2 +
                            (B[2 * nc + cidx(g, i, j, k + 1)] - B[2 * nc + c]) / d.dx3;
            }
}

void ora_flops_reset(void) {
#ifdef ORA_COUNT_FLOPS
    for (int m = 0; m < 5; m++) ora_flop_ctr[m] = 0;
#endif
    for (int p = 0; p < 6; p++)
        for (int m = 0; m < 5; m++) ora_phase_ctr[p][m] = 0;
}

void ora_flops_phase(unsigned long long* out30) {
    for (int p = 0; p < 6; p++)
        for (int m = 0; m < 5; m++) out30[p * 5 + m] = ora_phase_ctr[p][m];
}

void ora_flops_get(unsigned long long* out5) {
    for (int m = 0; m < 5; m++) out5[m] = 0;
#ifdef ORA_COUNT_FLOPS
    for (int m = 0; m < 5; m++) out5[m] = ora_flop_ctr[m];
#endif
}

} /* extern "C" */

/* ================================================================== */
/* Multi-block grids: static refinement (Sec. 3.2) and local adaptive   */
/* time stepping (Sec. 3.4)                                             */
/* ================================================================== */
/*
 * Ghost zones (Sec. 3.2): a ghost cell's centre is mapped across the
 * receiving block's physical boundaries (outflow: the nearest interior
 * cell; periodic: shifted by the period; polar: mirrored theta, phi + pi,
 * utilde^2 / B^2 / Bbar^2 negated), then looked up in the block that holds
 * it. The value is sampled from that block per dimension:
 *   same cell size   -> the cell itself,
 *   source finer     -> the average of the source cells it covers
 *                       (restriction),
 *   source coarser   -> the source cell plus delta * MINMOD slope along that
 *                       dimension (prolongation; delta = offset of the ghost
 *                       centre in units of the source cell).
 * Reading: a MINMOD slope whose stencil leaves the source block's interior
 * is 0. Ghost faces are sampled the same way without slopes; along their
 * normal they interpolate linearly between the source face planes.
 *
 * Time (Sec. 3.4): blocks of LAT level L step with 2^L dt_fine at the fine
 * substeps s with s mod 2^L = 0, coarsest level first. A ghost of block b
 * at stage time t samples a neighbour n of coarser level by linear
 * interpolation between n's state at the start of its step and its new
 * state; a neighbour of the same level at the same stage state (P or the
 * midpoint state); a neighbour of finer level at its current state.
 *
 * Synchronisation (Sec. 3.2, 3.4): blocks of the same level stepped together
 * share the flux of a face (the spatially coarser side takes the average of
 * the finer side's faces) and the EMF of an edge (every block takes the
 * EMF of the edge's dominant block: finest cell along the edge, then finest
 * across it, then lowest index). Across levels, at the end of each coarse
 * step the coarse block's face fluxes and edge EMFs are replaced by the time
 * integrals of the finer level's (refluxing), and its cells next to the
 * corrected faces are inverted again.
 */
namespace {

const double AMR_PI = 3.14159265358979323846;

struct FaceRec {  /* a coarse face refluxed from a finer-level block */
    int c;        /* coarse block */
    int d, side;  /* face direction, 0 = lower face of the block, 1 = upper */
    int i, j, k;  /* face index in c (lower-face convention) */
    int f;        /* fine block */
    std::vector<long> ff; /* fine face indices (padded cell index) */
    double own[NFX], acc[NFX];
};
struct EdgeRec { /* a coarse edge synchronised with the dominant edge of a finer level */
    int c, e;     /* block, edge direction */
    int i, j, k;  /* edge index in c */
    int f;        /* dominant block */
    std::vector<long> fe; /* its edge indices covering this edge */
    double own, acc;
};
struct SyncRec { /* same-level synchronisation: dst value := average of src values */
    int dst, d;
    long di;
    int src;
    std::vector<long> si;
};

struct AmrBlk {
    ora_grid* g;
    int lat;
    long s0;
    double lo[4], hi[4], h[4];
    std::vector<double> Pold, Bold, Ph, Bh;
    Fluxes F;
    std::vector<double> E;
};

}  // namespace

struct ora_amr {
    ora_desc phys;
    std::vector<AmrBlk> b;
    int Lmax;
    double dlo[4], dhi[4];
    bool per[4];
    long s;  /* substeps taken in the current period */
    std::vector<FaceRec> frec;
    std::vector<EdgeRec> erec;
    std::vector<SyncRec> fsync, esync;
    std::vector<std::vector<int>> touch; /* blocks whose boxes touch each block (lookup hints) */
    long long stats[4];
};

namespace {

bool amr_in(const AmrBlk& B, const double x[4], int pass) {
    for (int d = 1; d <= 3; d++) {
        double tol = 1e-9 * B.h[d];
        if (x[d] < B.lo[d] - tol) return false;
        if (pass == 0 ? !(x[d] < B.hi[d] - tol) : (x[d] > B.hi[d] + tol)) return false;
    }
    return true;
}

/* the block holding x: the half-open boxes first (a point on a shared plane
 * belongs to the block above it), then the closed ones (the domain's upper
 * boundary); `hint`'s touching blocks are tried before the full scan */
int amr_find(const ora_amr* m, const double x[4], int hint = -1) {
    for (int pass = 0; pass < 2; pass++) {
        if (hint >= 0) {
            if (amr_in(m->b[hint], x, pass)) return hint;
            for (int n : m->touch[hint])
                if (amr_in(m->b[n], x, pass)) return n;
        }
        for (int n = 0; n < (int)m->b.size(); n++)
            if (amr_in(m->b[n], x, pass)) return n;
    }
    return -1;
}

/* maps x (outside block b) across b's physical boundaries; fdir = normal
 * direction of a face point (0 for a cell centre) */
void amr_map(const ora_amr* m, int b, double x[4], int fdir, int* neg, int* clamp) {
    const AmrBlk& B = m->b[b];
    *neg = 0;
    *clamp = 0;
    for (int d = 1; d <= 3; d++) {
        const double q = 0.25 * B.h[d];
        int side = -1;
        if (x[d] < B.lo[d] - q) side = 0;
        if (x[d] > B.hi[d] + q) side = 1;
        if (side < 0) continue;
        const int bc = B.g->d.bc[2 * (d - 1) + side];
        if (bc == ORA_BC_OUTFLOW || bc == ORA_BC_OUTFLOW_NOINFLOW) {
            if (d == fdir)
                x[d] = side ? B.hi[d] : B.lo[d];
            else
                x[d] = side ? B.hi[d] - 0.5 * B.h[d] : B.lo[d] + 0.5 * B.h[d];
            if (bc == ORA_BC_OUTFLOW_NOINFLOW && d == 1) *clamp = side ? 1 : -1;
        } else if (bc == ORA_BC_PERIODIC) {
            x[d] += side ? -(m->dhi[d] - m->dlo[d]) : (m->dhi[d] - m->dlo[d]);
        } else if (bc == ORA_BC_POLAR) {
            x[2] = side ? 2.0 * AMR_PI - x[2] : -x[2];
            x[3] += AMR_PI;
            *neg = 1;
        }
    }
    if (m->per[3]) {
        const double L = m->dhi[3] - m->dlo[3];
        while (x[3] >= m->dhi[3] - 1e-12 * L) x[3] -= L;
        while (x[3] < m->dlo[3] - 1e-12 * L) x[3] += L;
    }
}

/* state of source n as seen by receiver b at stage sigma of substep s */
struct Src {
    const double *Pa, *Pb, *Ba, *Bb;
    double w;
    double P(long i) const { return Pb ? Pa[i] + w * (Pb[i] - Pa[i]) : Pa[i]; }
    double B(long i) const { return Bb ? Ba[i] + w * (Bb[i] - Ba[i]) : Ba[i]; }
};

Src amr_src(const ora_amr* m, int b, int n, int sigma, long s) {
    const AmrBlk& R = m->b[b];
    const AmrBlk& N = m->b[n];
    Src r;
    r.Pb = r.Bb = nullptr;
    r.w = 0.0;
    if (N.lat > R.lat) {
        r.Pa = N.Pold.data();
        r.Ba = N.Bold.data();
        r.Pb = N.g->prim.data();
        r.Bb = N.g->bface.data();
        r.w = ((double)(s - N.s0) + sigma * 0.5 * (double)(1L << R.lat)) / (double)(1L << N.lat);
    } else if (N.lat == R.lat && sigma == 1) {
        r.Pa = N.Ph.data();
        r.Ba = N.Bh.data();
    } else {
        /* a same-level source at the predictor, or a finer one at either
         * stage: its current state. A finer neighbour has not yet advanced
         * (coarse first), so at the receiver's midpoint this is a first-order
         * value; the receiver's fluxes through the shared face are replaced by
         * the finer side's at the end of its step (refluxing). Extrapolating
         * it linearly in time from its last two states instead amplified
         * step-to-step oscillations at coarse-fine faces in a magnetised torus
         * until the inversions failed. */
        r.Pa = N.g->prim.data();
        r.Ba = N.g->bface.data();
    }
    return r;
}

/* MINMOD: the argument of smaller magnitude where both have the same strict
 * sign, else 0 */
double minmod(double a, double b) {
    if (!((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0))) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* per-dimension footprint of a target cell of size ht centred at x in block N */
void footprint(const AmrBlk& N, const double x[4], const double ht[4], int i0[4], int cnt[4], double dl[4]) {
    for (int d = 1; d <= 3; d++) {
        const double hs = N.h[d];
        const double r = ht[d] / hs;
        dl[d] = 0.0;
        if (r > 1.5) {
            cnt[d] = (int)std::lround(r);
            i0[d] = (int)std::lround((x[d] - 0.5 * ht[d] - N.lo[d]) / hs);
        } else {
            cnt[d] = 1;
            i0[d] = (int)std::floor((x[d] - N.lo[d]) / hs);
            /* offset of the target centre in source cells, a multiple of 1/8 */
            if (r < 0.75) dl[d] = std::nearbyint(8.0 * (x[d] - (N.lo[d] + (i0[d] + 0.5) * hs)) / hs) / 8.0;
        }
    }
}

void amr_sample_cell(const ora_amr* m, int n, const Src& S, const double x[4], const double ht[4], double out[NPR]) {
    const AmrBlk& N = m->b[n];
    const ora_grid* g = N.g;
    const int nn[4] = {0, g->d.n1, g->d.n2, g->d.n3};
    int i0[4], cnt[4];
    double dl[4];
    footprint(N, x, ht, i0, cnt, dl);
    const long nc = g->ncell;
    const double inv = 1.0 / (double)(cnt[1] * cnt[2] * cnt[3]);
    for (int v = 0; v < NPR; v++) {
        double sum = 0.0;
        for (int c3 = 0; c3 < cnt[3]; c3++)
            for (int c2 = 0; c2 < cnt[2]; c2++)
                for (int c1 = 0; c1 < cnt[1]; c1++) {
                    int ii[4] = {0, i0[1] + c1, i0[2] + c2, i0[3] + c3};
                    long c = cidx(g, ii[1], ii[2], ii[3]);
                    const double q0 = S.P(v * nc + c);
                    double q = q0;
                    for (int d = 1; d <= 3; d++) {
                        if (dl[d] == 0.0) continue;
                        if (ii[d] - 1 < 0 || ii[d] + 1 >= nn[d]) continue;
                        int im[4] = {0, ii[1], ii[2], ii[3]}, ip[4] = {0, ii[1], ii[2], ii[3]};
                        im[d]--;
                        ip[d]++;
                        double qm = S.P(v * nc + cidx(g, im[1], im[2], im[3]));
                        double qp = S.P(v * nc + cidx(g, ip[1], ip[2], ip[3]));
                        q += dl[d] * minmod(q0 - qm, qp - q0);
                    }
                    sum += q;
                }
        out[v] = sum * inv;
    }
}

/* face value of direction fd at point x (x[fd] on a face plane) */
double amr_sample_face(const ora_amr* m, int n, const Src& S, const double x[4], const double ht[4], int fd) {
    const AmrBlk& N = m->b[n];
    const ora_grid* g = N.g;
    const long nc = g->ncell;
    int i0[4], cnt[4];
    double dl[4];
    double xc[4] = {0, x[1], x[2], x[3]};
    xc[fd] += 0.5 * ht[fd]; /* footprint along fd from the cell above the face */
    footprint(N, xc, ht, i0, cnt, dl);
    /* along the normal: the plane at x[fd], linearly between source planes */
    double pos = (x[fd] - N.lo[fd]) / N.h[fd];
    int p0 = (int)std::floor(pos + 1e-9);
    double fr = std::nearbyint(8.0 * (pos - p0)) / 8.0; /* a multiple of 1/8 */
    if (fr >= 1.0) {
        p0 += 1;
        fr = 0.0;
    }
    cnt[fd] = 1;
    const double inv = 1.0 / (double)(cnt[1] * cnt[2] * cnt[3]);
    double sum = 0.0;
    for (int c3 = 0; c3 < cnt[3]; c3++)
        for (int c2 = 0; c2 < cnt[2]; c2++)
            for (int c1 = 0; c1 < cnt[1]; c1++) {
                int ii[4] = {0, i0[1] + c1, i0[2] + c2, i0[3] + c3};
                ii[fd] = p0;
                double q = S.B((fd - 1) * nc + cidx(g, ii[1], ii[2], ii[3]));
                if (fr != 0.0) {
                    ii[fd] = p0 + 1;
                    double q1 = S.B((fd - 1) * nc + cidx(g, ii[1], ii[2], ii[3]));
                    q = q + fr * (q1 - q);
                }
                sum += q;
            }
    return sum * inv;
}

void amr_fill_block(ora_amr* m, int b, int sigma, double* P, double* Bf) {
    AmrBlk& R = m->b[b];
    ora_grid* g = R.g;
    const ora_desc& d = g->d;
    const int nn[4] = {0, d.n1, d.n2, d.n3};
    const long nc = g->ncell;
    for (int k = -NG; k < d.n3 + NG; k++)
        for (int j = -NG; j < d.n2 + NG; j++)
            for (int i = -NG; i < d.n1 + NG; i++) {
                const int ii[4] = {0, i, j, k};
                bool ghost = false;
                for (int e = 1; e <= 3; e++)
                    if (ii[e] < 0 || ii[e] >= nn[e]) ghost = true;
                const long c = cidx(g, i, j, k);
                if (ghost) {
                    double x[4] = {0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2],
                                   R.lo[3] + (k + 0.5) * R.h[3]};
                    int neg, clamp;
                    amr_map(m, b, x, 0, &neg, &clamp);
                    int n = amr_find(m, x, b);
                    if (n < 0) continue;
                    Src S = amr_src(m, b, n, sigma, m->s);
                    double out[NPR];
                    amr_sample_cell(m, n, S, x, R.h, out);
                    if (neg) {
                        out[U2] = -out[U2];
                        out[B2] = -out[B2];
                    }
                    if (clamp > 0 && out[U1] < 0.0) out[U1] = 0.0;
                    if (clamp < 0 && out[U1] > 0.0) out[U1] = 0.0;
                    for (int v = 0; v < NPR; v++) P[v * nc + c] = out[v];
                }
                for (int fd = 1; fd <= 3; fd++) {
                    bool owned = true;
                    for (int e = 1; e <= 3; e++) {
                        if (e == fd) {
                            if (ii[e] < 0 || ii[e] > nn[e]) owned = false;
                        } else if (ii[e] < 0 || ii[e] >= nn[e]) {
                            owned = false;
                        }
                    }
                    if (owned) continue;
                    double x[4] = {0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2],
                                   R.lo[3] + (k + 0.5) * R.h[3]};
                    x[fd] = R.lo[fd] + ii[fd] * R.h[fd];
                    int neg, clamp;
                    amr_map(m, b, x, fd, &neg, &clamp);
                    int n = amr_find(m, x, b);
                    if (n < 0) continue;
                    Src S = amr_src(m, b, n, sigma, m->s);
                    double v = amr_sample_face(m, n, S, x, R.h, fd);
                    Bf[(fd - 1) * nc + c] = (neg && fd == 2) ? -v : v;
                }
            }
}

/* blocks around an edge of direction e at the corner point p (p[e] = edge centre) */
void edge_blocks(const ora_amr* m, int b, const double p[4], int e, std::vector<int>& out) {
    const AmrBlk& B = m->b[b];
    int a1 = (e == 1) ? 2 : 1, a2 = (e == 3) ? 2 : 3;
    out.clear();
    for (int sa = -1; sa <= 1; sa += 2)
        for (int sb = -1; sb <= 1; sb += 2) {
            double x[4] = {0, p[1], p[2], p[3]};
            x[a1] += sa * 0.25 * B.h[a1];
            x[a2] += sb * 0.25 * B.h[a2];
            bool outside = false;
            for (int d = 1; d <= 3; d++) {
                if (m->per[d]) {
                    const double L = m->dhi[d] - m->dlo[d];
                    if (x[d] < m->dlo[d]) x[d] += L;
                    if (x[d] >= m->dhi[d]) x[d] -= L;
                } else if (x[d] < m->dlo[d] || x[d] > m->dhi[d]) {
                    outside = true;
                }
            }
            if (outside) continue;
            int n = amr_find(m, x);
            if (n >= 0 && std::find(out.begin(), out.end(), n) == out.end()) out.push_back(n);
        }
}

/* dominance: finest along the edge, then finest across, then lowest index */
bool dominates(const ora_amr* m, int a, int c, int e) {
    const AmrBlk& A = m->b[a];
    const AmrBlk& C = m->b[c];
    if (A.h[e] != C.h[e]) return A.h[e] < C.h[e];
    double va = A.h[1] * A.h[2] * A.h[3], vc = C.h[1] * C.h[2] * C.h[3];
    if (va != vc) return va < vc;
    return a < c;
}

/* padded index in block n of the edge segments of direction e covering the
 * segment [p[e] - he/2, p[e] + he/2] at corner point p */
void edge_cover(const ora_amr* m, int n, const double p[4], int e, double he, std::vector<long>& out) {
    const AmrBlk& N = m->b[n];
    out.clear();
    int idx[4];
    for (int d = 1; d <= 3; d++) {
        if (d == e) continue;
        double x = p[d];
        if (m->per[d]) {
            const double L = m->dhi[d] - m->dlo[d];
            if (x < N.lo[d] - 1e-9 * L) x += L;
            if (x > N.hi[d] + 1e-9 * L) x -= L;
        }
        idx[d] = (int)std::lround((x - N.lo[d]) / N.h[d]);
    }
    int cnt = (int)std::lround(he / N.h[e]);
    if (cnt < 1) cnt = 1;
    double x0 = p[e] - 0.5 * he;
    if (m->per[e]) {
        const double L = m->dhi[e] - m->dlo[e];
        if (x0 < N.lo[e] - 1e-9 * L) x0 += L;
        if (x0 > N.hi[e] - 1e-9 * L) x0 -= L;
    }
    int i0 = (int)std::lround((x0 - N.lo[e]) / N.h[e]);
    for (int c = 0; c < cnt; c++) {
        idx[e] = i0 + c;
        out.push_back(cidx(N.g, idx[1], idx[2], idx[3]));
    }
}

/* padded face indices in block n (direction d) covering a face of block b centred at p */
void face_cover(const ora_amr* m, int n, const double p[4], int d, const double hb[4], std::vector<long>& out) {
    const AmrBlk& N = m->b[n];
    out.clear();
    int i0[4], cnt[4];
    for (int e = 1; e <= 3; e++) {
        double x = p[e];
        if (m->per[e]) {
            const double L = m->dhi[e] - m->dlo[e];
            if (x < N.lo[e] - 1e-9 * L) x += L;
            if (x > N.hi[e] + 1e-9 * L) x -= L;
        }
        if (e == d) {
            i0[e] = (int)std::lround((x - N.lo[e]) / N.h[e]);
            cnt[e] = 1;
        } else {
            cnt[e] = std::max(1, (int)std::lround(hb[e] / N.h[e]));
            i0[e] = (int)std::lround((x - 0.5 * hb[e] - N.lo[e]) / N.h[e]);
        }
    }
    for (int c3 = 0; c3 < cnt[3]; c3++)
        for (int c2 = 0; c2 < cnt[2]; c2++)
            for (int c1 = 0; c1 < cnt[1]; c1++) out.push_back(cidx(N.g, i0[1] + c1, i0[2] + c2, i0[3] + c3));
}

bool finer(const AmrBlk& A, const AmrBlk& C) {  /* A strictly finer than C in some dimension, nowhere coarser */
    bool st = false;
    for (int d = 1; d <= 3; d++) {
        if (A.h[d] > C.h[d] * (1 + 1e-9)) return false;
        if (A.h[d] < C.h[d] * (1 - 1e-9)) st = true;
    }
    return st;
}

void amr_build_links(ora_amr* m) {
    const int nb = (int)m->b.size();
    for (int b = 0; b < nb; b++) {
        AmrBlk& B = m->b[b];
        const ora_desc& d = B.g->d;
        const int nn[4] = {0, d.n1, d.n2, d.n3};
        /* faces */
        for (int fd = 1; fd <= 3; fd++)
            for (int side = 0; side < 2; side++) {
                if (d.bc[2 * (fd - 1) + side] != ORA_BC_BLOCK && d.bc[2 * (fd - 1) + side] != ORA_BC_PERIODIC) continue;
                int t1 = (fd == 1) ? 2 : 1, t2 = (fd == 3) ? 2 : 3;
                for (int b2 = 0; b2 < nn[t2]; b2++)
                    for (int b1 = 0; b1 < nn[t1]; b1++) {
                        int ii[4];
                        ii[fd] = side ? nn[fd] : 0;
                        ii[t1] = b1;
                        ii[t2] = b2;
                        double p[4] = {0, B.lo[1] + (ii[1] + 0.5) * B.h[1], B.lo[2] + (ii[2] + 0.5) * B.h[2],
                                       B.lo[3] + (ii[3] + 0.5) * B.h[3]};
                        p[fd] = side ? B.hi[fd] : B.lo[fd];
                        double q[4] = {0, p[1], p[2], p[3]};
                        q[fd] += (side ? 0.25 : -0.25) * B.h[fd];
                        if (m->per[fd]) {
                            const double L = m->dhi[fd] - m->dlo[fd];
                            if (q[fd] < m->dlo[fd]) q[fd] += L;
                            if (q[fd] >= m->dhi[fd]) q[fd] -= L;
                        }
                        int n = amr_find(m, q);
                        if (n < 0 || n == b) continue;
                        AmrBlk& N = m->b[n];
                        if (!finer(N, B) && !(N.lat < B.lat)) continue;
                        long fi = cidx(B.g, ii[1], ii[2], ii[3]);
                        double pn[4] = {0, p[1], p[2], p[3]};
                        if (m->per[fd]) {
                            const double L = m->dhi[fd] - m->dlo[fd];
                            if (pn[fd] < N.lo[fd] - 1e-9 * L) pn[fd] += L;
                            if (pn[fd] > N.hi[fd] + 1e-9 * L) pn[fd] -= L;
                        }
                        std::vector<long> cov;
                        face_cover(m, n, pn, fd, B.h, cov);
                        if (N.lat == B.lat) {
                            if (!finer(N, B)) continue;
                            SyncRec r;
                            r.dst = b;
                            r.d = fd;
                            r.di = fi;
                            r.src = n;
                            r.si = cov;
                            m->fsync.push_back(r);
                        } else {
                            FaceRec r;
                            r.c = b;
                            r.d = fd;
                            r.side = side;
                            r.i = ii[1];
                            r.j = ii[2];
                            r.k = ii[3];
                            r.f = n;
                            r.ff = cov;
                            m->frec.push_back(r);
                        }
                    }
            }
        /* edges on the block boundary */
        for (int e = 1; e <= 3; e++) {
            int a1 = (e == 1) ? 2 : 1, a2 = (e == 3) ? 2 : 3;
            for (int k = 0; k <= nn[3]; k++)
                for (int j = 0; j <= nn[2]; j++)
                    for (int i = 0; i <= nn[1]; i++) {
                        int ii[4] = {0, i, j, k};
                        if (ii[e] >= nn[e]) continue;
                        bool bnd = (ii[a1] == 0 || ii[a1] == nn[a1] || ii[a2] == 0 || ii[a2] == nn[a2]);
                        if (!bnd) continue;
                        /* axis edges hold 0 */
                        if (e != 2 && ((d.bc[2] == ORA_BC_POLAR && j == 0) || (d.bc[3] == ORA_BC_POLAR && j == nn[2])))
                            continue;
                        double p[4];
                        for (int dd = 1; dd <= 3; dd++) p[dd] = B.lo[dd] + ii[dd] * B.h[dd];
                        p[e] += 0.5 * B.h[e];
                        std::vector<int> around;
                        edge_blocks(m, b, p, e, around);
                        /* global dominant: finest time level, then spatial dominance */
                        int gd = b;
                        for (int n : around)
                            if (m->b[n].lat < m->b[gd].lat || (m->b[n].lat == m->b[gd].lat && dominates(m, n, gd, e)))
                                gd = n;
                        /* same-level dominant */
                        int sd = b;
                        for (int n : around)
                            if (m->b[n].lat == B.lat && dominates(m, n, sd, e)) sd = n;
                        long ei = cidx(B.g, i, j, k);
                        if (sd != b) {
                            SyncRec r;
                            r.dst = b;
                            r.d = e;
                            r.di = ei;
                            r.src = sd;
                            edge_cover(m, sd, p, e, B.h[e], r.si);
                            m->esync.push_back(r);
                        }
                        if (m->b[gd].lat < B.lat) {
                            EdgeRec r;
                            r.c = b;
                            r.e = e;
                            r.i = i;
                            r.j = j;
                            r.k = k;
                            r.f = gd;
                            edge_cover(m, gd, p, e, B.h[e], r.fe);
                            m->erec.push_back(r);
                        }
                    }
        }
    }
}

double amr_avg(const double* a, long off, const std::vector<long>& idx) {
    double s = 0.0;
    for (long q : idx) s += a[off + q];
    return s * (1.0 / (double)idx.size());
}

/* fluxes and EMFs of one stage of a group of same-level blocks, synchronised */
void amr_fluxes_group(ora_amr* m, const std::vector<int>& grp, int sigma) {
    const int lat = m->b[grp[0]].lat;
    for (int b : grp) {
        AmrBlk& B = m->b[b];
        double* Pf = sigma ? B.Ph.data() : B.g->prim.data();
        double* Bff = sigma ? B.Bh.data() : B.g->bface.data();
        amr_fill_block(m, b, sigma, Pf, Bff);
    }
    for (int b : grp) {
        AmrBlk& B = m->b[b];
        const double* Pf = sigma ? B.Ph.data() : B.g->prim.data();
        const double* Bff = sigma ? B.Bh.data() : B.g->bface.data();
        stage_fluxes(B.g, Pf, Bff, B.F);
    }
    for (const SyncRec& r : m->fsync) {
        if (m->b[r.dst].lat != lat) continue;
        AmrBlk& D = m->b[r.dst];
        const AmrBlk& S = m->b[r.src];
        for (int q = 0; q < NFX; q++)
            D.F[r.d][(size_t)q * D.g->ncell + r.di] = amr_avg(S.F[r.d].data(), (long)q * S.g->ncell, r.si);
    }
    for (int b : grp) stage_emf(m->b[b].g, m->b[b].F, sigma ? m->b[b].Ph.data() : m->b[b].g->prim.data(), m->b[b].E);
    std::vector<double> vals(m->esync.size());
    for (size_t q = 0; q < m->esync.size(); q++) {  /* read all, then write: sources may be synced too */
        const SyncRec& r = m->esync[q];
        if (m->b[r.dst].lat != lat) continue;
        const AmrBlk& S = m->b[r.src];
        vals[q] = amr_avg(S.E.data(), (long)(r.d - 1) * S.g->ncell, r.si);
    }
    for (size_t q = 0; q < m->esync.size(); q++) {
        const SyncRec& r = m->esync[q];
        if (m->b[r.dst].lat != lat) continue;
        AmrBlk& D = m->b[r.dst];
        D.E[(size_t)(r.d - 1) * D.g->ncell + r.di] = vals[q];
    }
    /* internal SMR: each block's EMFs as its groups' after the exchange (groups that meet at a shared
       edge cover the same phi range, so both sides average the same values) */
    for (int b : grp)
        if (m->b[b].g->d.smr > 0) smr_emf(m->b[b].g, m->b[b].E);
}

/* one midpoint step of every block of a same-level group (Sec. 2.1) */
void amr_step_group(ora_amr* m, const std::vector<int>& grp, double dtf) {
    for (int b : grp) {
        AmrBlk& B = m->b[b];
        B.Pold = B.g->prim;
        B.Bold = B.g->bface;
        B.s0 = m->s;
    }
    amr_fluxes_group(m, grp, 0);
    for (int b : grp) {
        AmrBlk& B = m->b[b];
        const double dt = dtf * (double)(1L << B.lat);
        stage_ct(B.g, B.E, B.Bold.data(), 0.5 * dt, B.Bh.data());
        stage_update(B.g, B.F, B.Pold.data(), B.Pold.data(), B.Bh.data(), 0.5 * dt, B.Ph.data());
    }
    amr_fluxes_group(m, grp, 1);
    const int lat = m->b[grp[0]].lat;
    /* reflux records: the coarse side's own integral, the fine side's accumulation */
    for (FaceRec& r : m->frec) {
        if (m->b[r.c].lat == lat) {
            const AmrBlk& C = m->b[r.c];
            const double dt = dtf * (double)(1L << C.lat);
            long fi = cidx(C.g, r.i, r.j, r.k);
            for (int q = 0; q < NFX; q++) {
                r.own[q] = dt * C.F[r.d][(size_t)q * C.g->ncell + fi];
                r.acc[q] = 0.0;
            }
        }
    }
    for (EdgeRec& r : m->erec) {
        if (m->b[r.c].lat == lat) {
            const AmrBlk& C = m->b[r.c];
            const double dt = dtf * (double)(1L << C.lat);
            r.own = dt * C.E[(size_t)(r.e - 1) * C.g->ncell + cidx(C.g, r.i, r.j, r.k)];
            r.acc = 0.0;
        }
    }
    for (FaceRec& r : m->frec) {
        if (m->b[r.f].lat == lat) {
            const AmrBlk& F = m->b[r.f];
            const double dt = dtf * (double)(1L << F.lat);
            for (int q = 0; q < NFX; q++) r.acc[q] += dt * amr_avg(F.F[r.d].data(), (long)q * F.g->ncell, r.ff);
        }
    }
    for (EdgeRec& r : m->erec) {
        if (m->b[r.f].lat == lat) {
            const AmrBlk& F = m->b[r.f];
            const double dt = dtf * (double)(1L << F.lat);
            r.acc += dt * amr_avg(F.E.data(), (long)(r.e - 1) * F.g->ncell, r.fe);
        }
    }
    for (int b : grp) {
        AmrBlk& B = m->b[b];
        const double dt = dtf * (double)(1L << B.lat);
        stage_ct(B.g, B.E, B.Bold.data(), dt, B.g->bface.data());
        stage_update(B.g, B.F, B.Pold.data(), B.Ph.data(), B.g->bface.data(), dt, B.g->prim.data());
    }
}

/* internal SMR at a reflux: a group is inverted as one cell, so every cell of
 * a group with a marked cell is marked */
void smr_mark(const ora_grid* g, std::vector<char>& mark) {
    const ora_desc& d = g->d;
    for (int j = 0; j < d.n2; j++) {
        const int w = smr_width(g, j);
        if (w == 1) continue;
        for (int k0 = 0; k0 < d.n3; k0 += w)
            for (int i = 0; i < d.n1; i++) {
                bool any = false;
                for (int q = 0; q < w; q++) any = any || mark[cidx(g, i, j, k0 + q)];
                if (any)
                    for (int q = 0; q < w; q++) mark[cidx(g, i, j, k0 + q)] = 1;
            }
    }
}

/* end of a coarse step (Sec. 3.2 refluxing, Sec. 3.4 flux correction): the
 * coarse block's face fluxes and edge EMFs are replaced by the time
 * integrals of the finer level's; the cells next to changed faces are
 * inverted again from U(P) + the flux correction. With internal SMR the
 * replaced EMFs are the finer side's averaged ones (the same phi ranges,
 * so the correction keeps the group structure of the field's change) and
 * grouped cells are inverted as groups (smr_mark). */
void amr_reflux(ora_amr* m, int c) {
    AmrBlk& C = m->b[c];
    ora_grid* g = C.g;
    const ora_desc& d = g->d;
    const long nc = g->ncell;
    std::vector<double> dU((size_t)NCONS * nc, 0.0), dE((size_t)3 * nc, 0.0);
    std::vector<char> mark(nc, 0);
    bool any = false;
    for (const FaceRec& r : m->frec) {
        if (r.c != c) continue;
        int ii[4] = {0, r.i, r.j, r.k};
        if (r.side == 1) ii[r.d]--;
        long cc = cidx(g, ii[1], ii[2], ii[3]);
        const double sgn = r.side ? -1.0 : 1.0;
        for (int q = 0; q < NCONS; q++) dU[(size_t)q * nc + cc] += sgn * (r.acc[q] - r.own[q]) / C.h[r.d];
        mark[cc] = 1;
        any = true;
    }
    for (const EdgeRec& r : m->erec) {
        if (r.c != c) continue;
        dE[(size_t)(r.e - 1) * nc + cidx(g, r.i, r.j, r.k)] = r.acc - r.own;
        any = true;
    }
    if (!any) return;
    std::vector<double> Bnew(g->bface.size());
    stage_ct(g, dE, g->bface.data(), 1.0, Bnew.data());
    /* cells on both sides of every face bounded by a corrected edge */
    for (const EdgeRec& r : m->erec) {
        if (r.c != c) continue;
        const int a1 = (r.e == 1) ? 2 : 1, a2 = (r.e == 3) ? 2 : 3;
        for (int fa = 0; fa < 2; fa++) {
            const int dfa = fa ? a2 : a1, ob = fa ? a1 : a2;
            for (int off = -1; off <= 0; off++)
                for (int side = -1; side <= 0; side++) {
                    int cell[4] = {0, r.i, r.j, r.k};
                    cell[ob] += off;
                    cell[dfa] += side;
                    if (cell[1] < 0 || cell[2] < 0 || cell[3] < 0 || cell[1] >= d.n1 || cell[2] >= d.n2 ||
                        cell[3] >= d.n3)
                        continue;
                    mark[cidx(g, cell[1], cell[2], cell[3])] = 1;
                }
        }
    }
    if (d.smr > 0) smr_mark(g, mark);
    /* U of the marked cells with the field before the correction */
    std::vector<double> U0((size_t)NCONS * nc, 0.0);
    for (int k = 0; k < d.n3; k++)
        for (int j = 0; j < d.n2; j++)
            for (int i = 0; i < d.n1; i++) {
                long cc = cidx(g, i, j, k);
                if (!mark[cc]) continue;
                const Geom& G = g->gc[gidx(g, i, j)];
                real pr[NPR];
                load_prim(g, g->prim.data(), cc, pr);
                State st;
                get_state(pr, G, st);
                real u9[9];
                prim_to_uf(pr, st, 0, d.gam, u9);
                for (int q = 0; q < NCONS; q++) U0[(size_t)q * nc + cc] = tod(u9[q] * G.gdet);
            }
    g->bface.swap(Bnew);
    for (int k = 0; k < d.n3; k++)
        for (int j = 0; j < d.n2; j++)
            for (int i = 0; i < d.n1; i++) {
                long cc = cidx(g, i, j, k);
                if (!mark[cc] || smr_width(g, j) > 1) continue;
                const Geom& G = g->gc[gidx(g, i, j)];
                real U[NCONS];
                for (int q = 0; q < NCONS; q++) U[q] = U0[(size_t)q * nc + cc] + dU[(size_t)q * nc + cc];
                real Bc[3];
                centre_b(g, g->bface.data(), i, j, k, Bc);
                real pr[NPR], p0[NPR];
                load_prim(g, g->prim.data(), cc, pr);
                for (int v = 0; v < NPR; v++) p0[v] = pr[v];
                pr[B1] = Bc[0];
                pr[B2] = Bc[1];
                pr[B3] = Bc[2];
                int its = 0;
                int st = con2prim(d, U, Bc, G, pr, &its);
                if (st == C2P_FAIL)
                    for (int v = 0; v < 5; v++) pr[v] = p0[v];
                m->stats[st == C2P_OK ? 0 : (st == C2P_ENTROPY ? 1 : 2)]++;
                if (d.floors && apply_floors(d, pr, G, g->rc[gidx(g, i, j)])) m->stats[3]++;
                for (int v = 0; v < NPR; v++) g->prim[v * nc + cc] = tod(pr[v]);
            }
    /* marked internal-SMR groups: the mean of the cells' corrected states inverted once (start: the
       mean of their primitives, field: the mean of their new centre fields), as in stage_update */
    for (int j = 0; j < d.n2 && d.smr > 0; j++) {
        const int w = smr_width(g, j);
        if (w == 1) continue;
        for (int k0 = 0; k0 < d.n3; k0 += w)
            for (int i = 0; i < d.n1; i++) {
                if (!mark[cidx(g, i, j, k0)]) continue;
                const long q2 = gidx(g, i, j);
                const Geom& G = g->gc[q2];
                real U[NCONS], Bc[3] = {0.0, 0.0, 0.0}, pr[NPR];
                for (int q = 0; q < NCONS; q++) U[q] = 0.0;
                for (int v = 0; v < NPR; v++) pr[v] = 0.0;
                for (int a = 0; a < w; a++) {
                    const long cc = cidx(g, i, j, k0 + a);
                    for (int q = 0; q < NCONS; q++)
                        U[q] += real(U0[(size_t)q * nc + cc] + dU[(size_t)q * nc + cc]);
                    real b[3];
                    centre_b(g, g->bface.data(), i, j, k0 + a, b);
                    for (int e = 0; e < 3; e++) Bc[e] += b[e];
                    for (int v = 0; v < 5; v++) pr[v] += g->prim[v * nc + cc];
                }
                for (int q = 0; q < NCONS; q++) U[q] /= w;
                for (int e = 0; e < 3; e++) Bc[e] /= w;
                for (int v = 0; v < 5; v++) pr[v] /= w;
                real p0[5];
                for (int v = 0; v < 5; v++) p0[v] = pr[v];
                pr[B1] = Bc[0];
                pr[B2] = Bc[1];
                pr[B3] = Bc[2];
                int its = 0;
                int st = con2prim(d, U, Bc, G, pr, &its);
                if (st == C2P_FAIL)
                    for (int v = 0; v < 5; v++) pr[v] = p0[v];
                const bool fl = d.floors && apply_floors(d, pr, G, g->rc[q2]);
                for (int a = 0; a < w; a++) {
                    const long cc = cidx(g, i, j, k0 + a);
                    m->stats[st == C2P_OK ? 0 : (st == C2P_ENTROPY ? 1 : 2)]++;
                    if (fl) m->stats[3]++;
                    real b[3];
                    centre_b(g, g->bface.data(), i, j, k0 + a, b);
                    for (int v = 0; v < 5; v++) g->prim[v * nc + cc] = tod(pr[v]);
                    for (int e = 0; e < 3; e++) g->prim[(B1 + e) * nc + cc] = tod(b[e]);
                }
            }
    }
}

/* ------------------------------------------------------------------ */
/* Regridding (Sec. 3.2: (de)refinement)                                */
/* ------------------------------------------------------------------ */
/*
 * The state of a new tree from the old one at the same time. Cell-centred
 * primitives are sampled like ghosts (same cell size: copied; old finer:
 * volume average; old coarser: MINMOD-limited linear prolongation). Reading:
 * primitives, not conserved variables, are prolonged and restricted (the
 * paper allows either and calls the primitive form faster and more robust).
 * Face fields: old face at the same size copied, old finer: area average,
 * old coarser: the divergence-free prolongation of Balsara (2001), which
 * fills a coarse cell with a field quadratic in the cell's local coordinates,
 * exactly divergence-free, that matches every coarse face's mean and
 * MINMOD-limited tangential slopes (a slope whose stencil leaves the old
 * block's faces is 0); a fine face takes the polynomial at its centre (its
 * mean, the polynomial being linear on the face). Where a coarse cell borders
 * old finer data, the fine faces on that coarse face are the old ones and the
 * interior fine faces are corrected (interior_fine_face). A face point on a
 * plane between two old blocks is taken from the finer one. A regrid changes
 * a region's cell size by a factor of 2 at most.
 */

/* tangential MINMOD slope of face field a at face (i, j, k) of block N along
 * direction b, per unit of the local coordinate (half the per-cell slope) */
double face_slope(const AmrBlk& N, int a, const int ii[4], int b) {
    const ora_grid* g = N.g;
    const int nn[4] = {0, g->d.n1, g->d.n2, g->d.n3};
    if (ii[b] - 1 < 0 || ii[b] + 1 > nn[b] - 1) return 0.0;
    int im[4] = {0, ii[1], ii[2], ii[3]}, ip[4] = {0, ii[1], ii[2], ii[3]};
    im[b]--;
    ip[b]++;
    const double* B = g->bface.data() + (size_t)(a - 1) * g->ncell;
    const double q0 = B[cidx(g, ii[1], ii[2], ii[3])];
    return 0.5 * minmod(q0 - B[cidx(g, im[1], im[2], im[3])], B[cidx(g, ip[1], ip[2], ip[3])] - q0);
}

/* the coarse cell of N holding point `probe`, and the local coordinates
 * (-1..1 across the cell) of point x in it */
void coarse_cell(const AmrBlk& N, const double x[4], const double probe[4], int ic[4], double xi[4]) {
    const ora_grid* g = N.g;
    const int nn[4] = {0, g->d.n1, g->d.n2, g->d.n3};
    for (int d = 1; d <= 3; d++) {
        ic[d] = (int)std::floor((probe[d] - N.lo[d]) / N.h[d]);
        if (ic[d] < 0) ic[d] = 0;
        if (ic[d] > nn[d] - 1) ic[d] = nn[d] - 1;
        xi[d] = 2.0 * (x[d] - (N.lo[d] + (ic[d] + 0.5) * N.h[d])) / N.h[d];
    }
}

/* Balsara's polynomial of face component fd in coarse cell ic of N at local
 * coordinates xi. B_a = A0 + A_a xi_a + sum_{b != a} (A_b xi_b + A_ab xi_a xi_b)
 * + A_aa xi_a^2: the means Fm, Fp of the lower and upper faces and their
 * tangential slopes Sm, Sp give A_a, A_b, A_ab and A0 + A_aa; divergence-free
 * fixes A^a_aa = -(H_a / 2) sum_{b != a} A^b_ba / H_b. */
double balsara_poly(const AmrBlk& N, const int ic[4], const double xi[4], int fd) {
    const ora_grid* g = N.g;
    double Fm[4], Fp[4], Sm[4][4], Sp[4][4];
    for (int a = 1; a <= 3; a++) {
        int lo[4] = {0, ic[1], ic[2], ic[3]}, hi[4] = {0, ic[1], ic[2], ic[3]};
        hi[a]++;
        const double* B = g->bface.data() + (size_t)(a - 1) * g->ncell;
        Fm[a] = B[cidx(g, lo[1], lo[2], lo[3])];
        Fp[a] = B[cidx(g, hi[1], hi[2], hi[3])];
        for (int b = 1; b <= 3; b++) {
            Sm[a][b] = Sp[a][b] = 0.0;
            if (b == a) continue;
            Sm[a][b] = face_slope(N, a, lo, b);
            Sp[a][b] = face_slope(N, a, hi, b);
        }
    }
    double Aab[4][4];
    for (int a = 1; a <= 3; a++)
        for (int b = 1; b <= 3; b++) Aab[a][b] = (b == a) ? 0.0 : 0.5 * (Sp[a][b] - Sm[a][b]);
    const int a = fd;
    double Aaa = 0.0;
    for (int b = 1; b <= 3; b++)
        if (b != a) Aaa += Aab[b][a] / N.h[b];
    Aaa *= -0.5 * N.h[a];
    double val = 0.5 * (Fp[a] + Fm[a]) - Aaa + 0.5 * (Fp[a] - Fm[a]) * xi[a] + Aaa * xi[a] * xi[a];
    for (int b = 1; b <= 3; b++) {
        if (b == a) continue;
        val += 0.5 * (Sp[a][b] + Sm[a][b]) * xi[b] + Aab[a][b] * xi[a] * xi[b];
    }
    return val;
}

void wrap_periodic(const ora_amr* m, double x[4]);

/* cell widths a narrower than b in some direction (a block finer than b along it) */
bool finer_cells(const double a[4], const double b[4]) {
    return a[1] < b[1] * (1.0 - 1e-9) || a[2] < b[2] * (1.0 - 1e-9) || a[3] < b[3] * (1.0 - 1e-9);
}
double cell_volume(const double h[4]) { return h[1] * h[2] * h[3]; }

/* Refinement factor (1 or 2) along each direction of a new block of cell
 * widths hn inside an old coarser block N: an octree child halves all three
 * widths, a 6-way polar child on the axis keeps N's x3 width (Sec. 3.3.1). */
void refine_factors(const AmrBlk& N, const double hn[4], int f[4]) {
    f[0] = 1;
    for (int d = 1; d <= 3; d++) f[d] = (N.h[d] > 1.5 * hn[d]) ? 2 : 1;
}

/* A fine face (cell widths hn) on the coarse face (a, side) of cell ic; along
 * each tangential direction b < c it is one of the two halves (tb, tc: 0 lower,
 * 1 upper) where the refinement splits that direction, else the whole width
 * (tb, tc = 0). Its value: the old tree's finer data beyond that coarse face if
 * there is any (copied or area-averaged), else the polynomial (the coarse
 * face's linear profile). */
double fine_face_on_coarse(const ora_amr* old, const AmrBlk& N, const int ic[4], int a, int side, int tb, int tc,
                           const double hn[4]) {
    const int b = (a == 1) ? 2 : 1, c = (a == 3) ? 2 : 3;
    int f[4];
    refine_factors(N, hn, f);
    const double ob = (f[b] == 2) ? 0.25 + 0.5 * tb : 0.5, oc = (f[c] == 2) ? 0.25 + 0.5 * tc : 0.5;
    double x[4];
    x[a] = N.lo[a] + (ic[a] + side) * N.h[a];
    x[b] = N.lo[b] + (ic[b] + ob) * N.h[b];
    x[c] = N.lo[c] + (ic[c] + oc) * N.h[c];
    double probe[4] = {0, x[1], x[2], x[3]};
    probe[a] += (side ? 0.25 : -0.25) * hn[a];
    wrap_periodic(old, probe);
    const int n = amr_find(old, probe);
    if (n >= 0 && finer_cells(old->b[n].h, N.h)) {
        double xs[4] = {0, probe[1], probe[2], probe[3]};
        xs[a] -= (side ? 0.25 : -0.25) * hn[a];
        const AmrBlk& B = old->b[n];
        if (B.h[b] > 1.5 * hn[b] || B.h[c] > 1.5 * hn[c]) {
            /* that block's cells are wider than the new face along the plane (an axis child next to
             * octants): its polynomial's linear profile on its face, the value the new block on the
             * other side of the plane takes for this face */
            int icb[4];
            double xib[4];
            coarse_cell(B, xs, probe, icb, xib);
            return balsara_poly(B, icb, xib, a);
        }
        Src S;
        S.Pa = B.g->prim.data();
        S.Ba = B.g->bface.data();
        S.Pb = S.Bb = nullptr;
        S.w = 0.0;
        return amr_sample_face(old, n, S, xs, hn, a);
    }
    double xi[4] = {0, 0.0, 0.0, 0.0};
    xi[a] = side ? 1.0 : -1.0;
    xi[b] = (f[b] == 2) ? (tb ? 0.5 : -0.5) : 0.0;
    xi[c] = (f[c] == 2) ? (tc ? 0.5 : -0.5) : 0.0;
    return balsara_poly(N, ic, xi, a);
}

/* A fine face interior to coarse cell ic (local plane xi_fd = 0), the cell
 * split into f1 x f2 x f3 fine cells (refine_factors; 2 x 2 x 2 for an
 * octree child, 2 x 2 x 1 for a polar child on the axis). Reading: the
 * polynomial's value is a prior; the fine faces on the cell's boundary
 * (fine_face_on_coarse: old finer data where it exists) and the interior faces
 * must make each fine cell divergence-free, and the interior faces take the
 * smallest change (least squares) from the prior that does. With D_c the prior
 * divergence (flux form, face areas A_d) of fine cell c, the change is
 * A_d (lambda_lo - lambda_hi) across a face of direction d, where
 * L lambda = -D and L is the graph Laplacian of the fine cells (weights A_d^2
 * between neighbours along d); solved here with lambda of the first cell fixed
 * at 0 (the change does not depend on that constant). Where the boundary faces
 * follow the polynomial, D = 0 and the prior stands. */
double interior_fine_face(const ora_amr* old, const AmrBlk& N, const int ic[4], const double xi[4], int fd,
                          const double hn[4]) {
    int f[4];
    refine_factors(N, hn, f);
    /* F[a][plane 0..2][t_b][t_c]: planes 0 and 2 on the coarse faces, 1 the interior plane (split a) */
    double F[4][3][2][2];
    for (int a = 1; a <= 3; a++) {
        const int b = (a == 1) ? 2 : 1, c = (a == 3) ? 2 : 3;
        for (int tb = 0; tb < f[b]; tb++)
            for (int tc = 0; tc < f[c]; tc++) {
                F[a][0][tb][tc] = fine_face_on_coarse(old, N, ic, a, 0, tb, tc, hn);
                F[a][2][tb][tc] = fine_face_on_coarse(old, N, ic, a, 1, tb, tc, hn);
                if (f[a] == 2) {
                    double x0[4] = {0, 0.0, 0.0, 0.0};
                    x0[b] = (f[b] == 2) ? (tb ? 0.5 : -0.5) : 0.0;
                    x0[c] = (f[c] == 2) ? (tc ? 0.5 : -0.5) : 0.0;
                    F[a][1][tb][tc] = balsara_poly(N, ic, x0, a);
                }
            }
    }
    const double A[4] = {0, hn[2] * hn[3], hn[1] * hn[3], hn[1] * hn[2]};
    /* the fine cells, c = i1 + 2 i2 + 4 i3 with i_d < f_d */
    int cells[8], nc = 0;
    for (int c = 0; c < 8; c++)
        if ((c & 1) < f[1] && ((c >> 1) & 1) < f[2] && ((c >> 2) & 1) < f[3]) cells[nc++] = c;
    double D[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < nc; q++) {
        const int c = cells[q];
        const int ix[4] = {0, c & 1, (c >> 1) & 1, (c >> 2) & 1};
        double sum = 0.0;
        for (int a = 1; a <= 3; a++) {
            const int b = (a == 1) ? 2 : 1, cc = (a == 3) ? 2 : 3;
            const int lo = (f[a] == 2) ? ix[a] : 0, up = (f[a] == 2) ? ix[a] + 1 : 2;
            sum += A[a] * (F[a][up][ix[b]][ix[cc]] - F[a][lo][ix[b]][ix[cc]]);
        }
        D[c] = sum;
    }
    /* L lambda = -D with lambda of cells[0] = 0: the (nc - 1) x (nc - 1) system by Gaussian elimination */
    const int m = nc - 1;
    double M[7][8];
    for (int r = 0; r < m; r++)
        for (int q = 0; q <= m; q++) M[r][q] = 0.0;
    for (int r = 1; r < nc; r++) {
        const int c = cells[r];
        double diag = 0.0;
        for (int a = 1; a <= 3; a++) {
            if (f[a] != 2) continue;
            diag += A[a] * A[a];
            const int nb = c ^ (1 << (a - 1));
            for (int q = 1; q < nc; q++)
                if (cells[q] == nb) M[r - 1][q - 1] -= A[a] * A[a];
        }
        M[r - 1][r - 1] += diag;
        M[r - 1][m] = -D[c];
    }
    for (int p = 0; p < m; p++)
        for (int r = p + 1; r < m; r++) {
            const double fac = M[r][p] / M[p][p];
            for (int q = p; q <= m; q++) M[r][q] -= fac * M[p][q];
        }
    double lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = m - 1; p >= 0; p--) {
        double sum = M[p][m];
        for (int q = p + 1; q < m; q++) sum -= M[p][q] * lam[cells[q + 1]];
        lam[cells[p + 1]] = sum / M[p][p];
    }
    const int b = (fd == 1) ? 2 : 1, cc = (fd == 3) ? 2 : 3;
    const int tb = (f[b] == 2) ? (xi[b] > 0.0) : 0, tc = (f[cc] == 2) ? (xi[cc] > 0.0) : 0;
    int ix[4] = {0, 0, 0, 0};
    ix[b] = tb;
    ix[cc] = tc;
    ix[fd] = 0;
    const int clo = ix[1] + 2 * ix[2] + 4 * ix[3];
    ix[fd] = 1;
    const int chi = ix[1] + 2 * ix[2] + 4 * ix[3];
    return F[fd][1][tb][tc] + A[fd] * (lam[clo] - lam[chi]);
}

/* x inside the domain's periodic range along the periodic directions */
void wrap_periodic(const ora_amr* m, double x[4]) {
    for (int d = 1; d <= 3; d++) {
        if (!m->per[d]) continue;
        const double L = m->dhi[d] - m->dlo[d];
        while (x[d] >= m->dhi[d]) x[d] -= L;
        while (x[d] < m->dlo[d]) x[d] += L;
    }
}

void amr_regrid_fill(ora_amr* old, ora_amr* m) {
    for (int b = 0; b < (int)m->b.size(); b++) {
        AmrBlk& R = m->b[b];
        ora_grid* g = R.g;
        const ora_desc& d = g->d;
        const long nc = g->ncell;
        const int nn[4] = {0, d.n1, d.n2, d.n3};
        for (int k = 0; k < d.n3; k++)
            for (int j = 0; j < d.n2; j++)
                for (int i = 0; i < d.n1; i++) {
                    double x[4] = {0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2],
                                   R.lo[3] + (k + 0.5) * R.h[3]};
                    const int n = amr_find(old, x);
                    if (n < 0) continue;
                    Src S;
                    S.Pa = old->b[n].g->prim.data();
                    S.Ba = old->b[n].g->bface.data();
                    S.Pb = S.Bb = nullptr;
                    S.w = 0.0;
                    double out[NPR];
                    amr_sample_cell(old, n, S, x, R.h, out);
                    for (int v = 0; v < 5; v++) g->prim[v * nc + cidx(g, i, j, k)] = out[v];
                }
        for (int fd = 1; fd <= 3; fd++)
            for (int k = 0; k < d.n3 + (fd == 3); k++)
                for (int j = 0; j < d.n2 + (fd == 2); j++)
                    for (int i = 0; i < d.n1 + (fd == 1); i++) {
                        const int ii[4] = {0, i, j, k};
                        double x[4] = {0, R.lo[1] + (i + 0.5) * R.h[1], R.lo[2] + (j + 0.5) * R.h[2],
                                       R.lo[3] + (k + 0.5) * R.h[3]};
                        x[fd] = R.lo[fd] + ii[fd] * R.h[fd];
                        double pl[4] = {0, x[1], x[2], x[3]}, pr[4] = {0, x[1], x[2], x[3]};
                        pl[fd] -= 0.25 * R.h[fd];
                        pr[fd] += 0.25 * R.h[fd];
                        wrap_periodic(old, pl);
                        wrap_periodic(old, pr);
                        const int nl = amr_find(old, pl), nr = amr_find(old, pr);
                        int n = nr;
                        const double* probe = pr;
                        if (n < 0 || (nl >= 0 && cell_volume(old->b[nl].h) < cell_volume(old->b[nr].h) * (1.0 - 1e-9))) {
                            n = nl;
                            probe = pl;
                        }
                        if (n < 0) continue;
                        const AmrBlk& N = old->b[n];
                        /* the face point in the source block's frame (across a periodic boundary) */
                        double xs[4] = {0, probe[1], probe[2], probe[3]};
                        xs[fd] += (probe == pl ? 0.25 : -0.25) * R.h[fd];
                        double v;
                        if (N.h[1] > R.h[1] * 1.5 || N.h[2] > R.h[2] * 1.5 || N.h[3] > R.h[3] * 1.5) {
                            int ic[4];
                            double xi[4];
                            coarse_cell(N, xs, probe, ic, xi);
                            if (std::fabs(xi[fd]) > 0.5)
                                v = balsara_poly(N, ic, xi, fd);  /* on a coarse face: its linear profile */
                            else
                                v = interior_fine_face(old, N, ic, xi, fd, R.h);
                        } else {
                            Src S;
                            S.Pa = N.g->prim.data();
                            S.Ba = N.g->bface.data();
                            S.Pb = S.Bb = nullptr;
                            S.w = 0.0;
                            v = amr_sample_face(old, n, S, xs, R.h, fd);
                        }
                        g->bface[(fd - 1) * nc + cidx(g, i, j, k)] = v;
                    }
        for (int k = 0; k < d.n3; k++)
            for (int j = 0; j < d.n2; j++)
                for (int i = 0; i < d.n1; i++) {
                    real Bc[3];
                    centre_b(g, g->bface.data(), i, j, k, Bc);
                    for (int q = 0; q < 3; q++) g->prim[(B1 + q) * nc + cidx(g, i, j, k)] = tod(Bc[q]);
                }
        (void)nn;
        R.Pold = g->prim;
        R.Bold = g->bface;
        R.s0 = 0;
    }
}

}  // namespace

extern "C" {

ora_amr* ora_amr_new(const ora_desc* phys, int nb, const ora_block* blocks) {
    ora_amr* m = new ora_amr;
    m->phys = *phys;
    m->Lmax = 0;
    m->s = 0;
    for (int q = 0; q < 4; q++) m->stats[q] = 0;
    for (int d = 1; d <= 3; d++) {
        m->dlo[d] = 1e300;
        m->dhi[d] = -1e300;
        m->per[d] = false;
    }
    for (int n = 0; n < nb; n++) {
        const ora_block& o = blocks[n];
        ora_desc d = *phys;
        d.n1 = o.n1;
        d.n2 = o.n2;
        d.n3 = o.n3;
        d.x1min = o.x1min;
        d.x2min = o.x2min;
        d.x3min = o.x3min;
        d.dx1 = o.dx1;
        d.dx2 = o.dx2;
        d.dx3 = o.dx3;
        for (int f = 0; f < 6; f++) d.bc[f] = o.bc[f];
        AmrBlk B;
        B.g = ora_grid_new(&d);
        B.lat = o.lat;
        B.s0 = 0;
        const double x0[4] = {0, o.x1min, o.x2min, o.x3min};
        const double hh[4] = {0, o.dx1, o.dx2, o.dx3};
        const int nn[4] = {0, o.n1, o.n2, o.n3};
        for (int e = 1; e <= 3; e++) {
            B.lo[e] = x0[e];
            B.h[e] = hh[e];
            B.hi[e] = x0[e] + nn[e] * hh[e];
            m->dlo[e] = std::min(m->dlo[e], B.lo[e]);
            m->dhi[e] = std::max(m->dhi[e], B.hi[e]);
            if (o.bc[2 * (e - 1)] == ORA_BC_PERIODIC) m->per[e] = true;
        }
        B.Ph.assign(B.g->prim.size(), 0.0);
        B.Bh.assign(B.g->bface.size(), 0.0);
        B.Pold = B.g->prim;
        B.Bold = B.g->bface;
        m->Lmax = std::max(m->Lmax, o.lat);
        m->b.push_back(B);
    }
    const int nbk = (int)m->b.size();
    /* internal SMR: each polar block's widths against the coarsest polar block's (smr_width) */
    if (phys->smr > 0) {
        double h2b = 0.0, h3b = 0.0;
        for (const AmrBlk& B : m->b)
            if (B.g->d.bc[2] == ORA_BC_POLAR || B.g->d.bc[3] == ORA_BC_POLAR) {
                h2b = std::max(h2b, B.h[2]);
                h3b = std::max(h3b, B.h[3]);
            }
        for (AmrBlk& B : m->b)
            if (B.g->d.bc[2] == ORA_BC_POLAR || B.g->d.bc[3] == ORA_BC_POLAR) {
                B.g->smr_l2 = (int)std::lround(std::log2(h2b / B.h[2]));
                B.g->smr_l3 = (int)std::lround(std::log2(h3b / B.h[3]));
            }
    }
    m->touch.assign(nbk, {});
    for (int a = 0; a < nbk; a++)
        for (int c = 0; c < nbk; c++) {
            if (a == c) continue;
            bool t = true;
            for (int d = 1; d <= 3 && t; d++) {
                const AmrBlk& A = m->b[a];
                const AmrBlk& C = m->b[c];
                const double tol = 1e-9 * (m->dhi[d] - m->dlo[d]);
                bool ok = (A.lo[d] <= C.hi[d] + tol && C.lo[d] <= A.hi[d] + tol);
                if (!ok && m->per[d]) {
                    const double L = m->dhi[d] - m->dlo[d];
                    ok = (A.lo[d] <= C.hi[d] + L + tol && C.lo[d] + L <= A.hi[d] + tol) ||
                         (A.lo[d] <= C.hi[d] - L + tol && C.lo[d] - L <= A.hi[d] + tol);
                }
                t = ok;
            }
            if (t) m->touch[a].push_back(c);
        }
    amr_build_links(m);
    return m;
}

void ora_amr_free(ora_amr* m) {
    for (AmrBlk& B : m->b) ora_grid_free(B.g);
    delete m;
}

void ora_amr_set(ora_amr* m, int b, const double* prim, const double* bface) {
    ora_grid* g = m->b[b].g;
    std::memcpy(g->prim.data(), prim, sizeof(double) * NPR * g->ncell);
    std::memcpy(g->bface.data(), bface, sizeof(double) * 3 * g->ncell);
    const long nc = g->ncell;
    for (int k = 0; k < g->d.n3; k++)
        for (int j = 0; j < g->d.n2; j++)
            for (int i = 0; i < g->d.n1; i++) {
                real Bc[3];
                centre_b(g, g->bface.data(), i, j, k, Bc);
                for (int q = 0; q < 3; q++) g->prim[(B1 + q) * nc + cidx(g, i, j, k)] = tod(Bc[q]);
            }
    /* no history yet: the previous state is the loaded one */
    m->b[b].Pold = g->prim;
    m->b[b].Bold = g->bface;
    m->b[b].s0 = 0;
}

void ora_amr_get(const ora_amr* m, int b, double* prim, double* bface) { ora_grid_get(m->b[b].g, prim, bface); }

void ora_amr_fill(ora_amr* m) {
    /* every source at its current state: all blocks are at the same time */
    for (AmrBlk& B : m->b) {
        B.Pold = B.g->prim;
        B.Bold = B.g->bface;
        B.s0 = 0;
    }
    m->s = 0;
    for (int b = 0; b < (int)m->b.size(); b++) amr_fill_block(m, b, 0, m->b[b].g->prim.data(), m->b[b].g->bface.data());
}

double ora_amr_period(ora_amr* m, double dtf) {
    for (int q = 0; q < 4; q++) m->stats[q] = 0;
    if (!(dtf > 0.0)) {
        dtf = 1e300;
        for (AmrBlk& B : m->b) dtf = std::min(dtf, grid_dt(B.g) / (double)(1L << B.lat));
    }
    const long S = 1L << m->Lmax;
    for (long s = 0; s < S; s++) {
        m->s = s;
        for (int L = m->Lmax; L >= 0; L--) {
            if (s % (1L << L) != 0) continue;
            std::vector<int> grp;
            for (int b = 0; b < (int)m->b.size(); b++)
                if (m->b[b].lat == L) grp.push_back(b);
            if (grp.empty()) continue;
            for (int b : grp) std::fill(m->b[b].g->status.begin(), m->b[b].g->status.end(), 0);
            amr_step_group(m, grp, dtf);
            for (int b : grp)
                for (int q = 0; q < 4; q++) m->stats[q] += m->b[b].g->stats[q], m->b[b].g->stats[q] = 0;
        }
        for (int c = 0; c < (int)m->b.size(); c++)
            if ((s + 1) % (1L << m->b[c].lat) == 0) amr_reflux(m, c);
    }
    m->s = 0;
    return dtf;
}

ora_amr* ora_amr_regrid(ora_amr* old, int nb, const ora_block* blocks) {
    ora_amr_fill(old);
    ora_amr* m = ora_amr_new(&old->phys, nb, blocks);
    amr_regrid_fill(old, m);
    ora_amr_fill(m);
    return m;
}

void ora_amr_stats(const ora_amr* m, long long* counts4) {
    for (int q = 0; q < 4; q++) counts4[q] = m->stats[q];
}

}  /* extern "C" */
