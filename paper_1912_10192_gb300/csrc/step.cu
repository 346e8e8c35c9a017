// step.cu -- the per-block stage kernels of the midpoint step
// (Liska et al. 2019, Sec. 2.1 and 2.5-2.7).
//
// One stage = boundary conditions (3 passes) -> per direction: edge values
// (reconstruction) and face fluxes -> edge EMFs -> CT face update ->
// cell update + inversion + floors (+ CFL reduction in the corrector).
// Fluxes, EMFs and edge values go through HBM: the FP64 path is bound by the
// FP64 pipe, so every face flux and every parabola is computed exactly once
// and re-read from memory instead of recomputed in a halo.
#include <type_traits>

#include "c2p.cuh"
#include "grmhd.cuh"
#include "mlp.cuh"

#include "hamr_internal.h"

namespace hamr {
namespace {

constexpr int BS = 128;

__device__ __forceinline__ long cidx(const BlockView& v, int i, int j, int k) {
    return ((long)(k + NG) * v.n2p + (j + NG)) * v.n1p + (i + NG);
}
__device__ __forceinline__ long gidx(const BlockView& v, int i, int j) { return (long)(j + NG) * v.n1p + (i + NG); }

inline unsigned nblk(long n, int bs = BS) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------- centre B
// B^i = (Bbar^i_lo + Bbar^i_hi) / 2 / sqrt(-g)_centre (Sec. 2.5)
__device__ __forceinline__ void centre_field(const BlockView& v, const double* __restrict__ B, int i, int j, int k,
                                             double ig, double Bc[3]) {  // ig = 1 / sqrt(-g)
    const long c = cidx(v, i, j, k);
    const double hig = 0.5 * ig;
    Bc[0] = (B[c] + B[c + 1]) * hig;
    Bc[1] = (B[v.nc + c] + B[v.nc + c + v.n1p]) * hig;
    Bc[2] = (B[2 * v.nc + c] + B[2 * v.nc + c + (long)v.n1p * v.n2p]) * hig;
}

__device__ __forceinline__ void b_centre_b(const BlockView& v, double* __restrict__ P, const double* __restrict__ B, long t) {
    const long n = (long)v.n1 * v.n2 * v.n3;
    if (t >= n) return;
    const int i = (int)(t % v.n1), j = (int)((t / v.n1) % v.n2), k = (int)(t / ((long)v.n1 * v.n2));
    double Bc[3];
    centre_field(v, B, i, j, k, v.gc[G_IGDET * v.n2d + gidx(v, i, j)], Bc);
    const long c = cidx(v, i, j, k);
    P[B1 * v.nc + c] = Bc[0];
    P[B2 * v.nc + c] = Bc[1];
    P[B3 * v.nc + c] = Bc[2];
}

__global__ void k_centre_b(BlockView v, double* __restrict__ P, const double* __restrict__ B) {
    b_centre_b(v, P, B, (long)blockIdx.x * blockDim.x + threadIdx.x);
}


// ---------------------------------------------------------------- boundaries
// One pass per direction e, in the order x3, x2, x1, each over the full
// padded extent of the other two directions. Polar (x2): ghost (j = -1-m, k)
// takes (j = m, k + n3/2) with utilde^2, B^2 and Bbar^2 negated; axis faces 0.
// Outflow: copy of the last interior cell/face; NOINFLOW clamps utilde^1.
// Periodic: wrap; face n takes face 0.
__device__ __forceinline__ int cell_src(int bc, int n, int g) {
    if (bc == HAMR_BC_PERIODIC) return g < 0 ? g + n : g - n;
    if (bc == HAMR_BC_POLAR) return g < 0 ? -1 - g : 2 * n - 1 - g;
    return g < 0 ? 0 : n - 1;
}
__device__ __forceinline__ int face_src(int bc, int n, int g) {
    if (bc == HAMR_BC_PERIODIC) return g < 0 ? g + n : g - n;
    if (bc == HAMR_BC_POLAR) return g < 0 ? -g : 2 * n - g;
    return g < 0 ? 0 : n;
}

// P32, K32 (mixed precision on a single block, else null): the ghost cells of the FP32 copy of the
// primitives and of its entropy tracer kappa, from the same sources
__global__ void k_bc_pass(BlockView v, double* __restrict__ P, double* __restrict__ B, int e, float* __restrict__ P32,
                          float* __restrict__ K32) {
    const int nn[4] = {0, v.n1, v.n2, v.n3};
    const int ta = (e == 1) ? 2 : 1, tb = (e == 3) ? 2 : 3;
    const int na = nn[ta] + 2 * NG, nb = nn[tb] + 2 * NG;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long total = 2L * NG * na * nb;
    if (t >= total) return;
    const int a = (int)(t % na) - NG;
    const int b = (int)((t / na) % nb) - NG;
    const int m = (int)((t / ((long)na * nb)) % NG);
    const int side = (int)(t / ((long)na * nb * NG));
    const int bc = v.bc[2 * (e - 1) + side];
    const bool polar = (bc == HAMR_BC_POLAR);
    int ss[4] = {0, 0, 0, 0}, dd[4] = {0, 0, 0, 0};
    ss[ta] = a;
    ss[tb] = b;
    if (polar) ss[3] = ((b + v.n3 / 2) % v.n3 + v.n3) % v.n3;
    dd[ta] = a;
    dd[tb] = b;
    const int gi = (side == 0) ? -1 - m : nn[e] + m;
    dd[e] = gi;
    ss[e] = cell_src(bc, nn[e], gi);
    long dst = cidx(v, dd[1], dd[2], dd[3]), src = cidx(v, ss[1], ss[2], ss[3]);
#pragma unroll
    for (int q = 0; q < NPRIM; q++) {
        double x = P[q * v.nc + src];
        if (polar && (q == U2 || q == B2)) x = -x;
        if (q == U1 && bc == HAMR_BC_OUTFLOW_NOINFLOW && e == 1) {
            if (side == 1 && x < 0.0) x = 0.0;
            if (side == 0 && x > 0.0) x = 0.0;
        }
        P[q * v.nc + dst] = x;
        if (P32) P32[q * v.nc + dst] = (float)x;
    }
    if (K32) K32[dst] = K32[src];  // kappa depends on rho and u only, which the map keeps
#pragma unroll
    for (int f = 1; f <= 3; f++)
        if (f != e) B[(f - 1) * v.nc + dst] = B[(f - 1) * v.nc + src];
    const int gf = (side == 0) ? -1 - m : nn[e] + (bc == HAMR_BC_PERIODIC ? 0 : 1) + m;
    if (gf < nn[e] + NG) {
        dd[e] = gf;
        ss[e] = face_src(bc, nn[e], gf);
        dst = cidx(v, dd[1], dd[2], dd[3]);
        src = cidx(v, ss[1], ss[2], ss[3]);
        const double x = B[(e - 1) * v.nc + src];
        B[(e - 1) * v.nc + dst] = polar ? -x : x;
    }
}

// axis faces hold 0 (after the x2 pass wrote its ghosts)
__global__ void k_bc_axis(BlockView v, double* __restrict__ B) {
    const int na = v.n1 + 2 * NG, nb = v.n3 + 2 * NG;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2L * na * nb) return;
    const int i = (int)(t % na) - NG;
    const int k = (int)((t / na) % nb) - NG;
    const int side = (int)(t / ((long)na * nb));
    if (v.bc[2 + side] != HAMR_BC_POLAR) return;
    B[v.nc + cidx(v, i, side == 0 ? 0 : v.n2, k)] = 0.0;
}

// ---------------------------------------------------------------- reconstruction
// Edge values of every cell that borders a flux face of direction dir: cells
// -1..n_dir along dir, -1..n_e across, for the 7 primitives other than B^dir
// and the entropy tracer kappa of the cells (an eighth variable, read from K,
// whose edge values go to the B^dir fields of QL and QR).
// Every slope and every PPM interface value is formed once and shared by the
// two cells that use it: along x1 a warp holds 32 consecutive cells (28 of
// them produced) and passes values between lanes by shuffles; along x2 and
// x3 a thread sweeps recon_seg cells of one pencil (consecutive threads on
// consecutive i, so loads and stores coalesce). T = float (mixed precision)
// reads the FP32 copy of the primitives and writes FP32 edge values.
// Shock flattening (Colella & Woodward 1984), optional with PPM: a coefficient
// f in [0, 1] per cell of the reconstruction range, from p = (gam - 1) u and
// the velocity primitive w along dir. A relative pressure jump across the
// cell above 0.33 of the smaller neighbour with converging flow (w(c-1) >
// w(c+1)) marks a shock; f = 10 (|dp1| / |dp2| - 3/4) clamped to [0, 1], dp1 =
// p(c+1) - p(c-1), dp2 = p(c+2) - p(c-2), and f = 1 for dp2 = 0 (the ratio in
// magnitude: at a narrow pressure peak dp2 is zero up to rounding, and a
// signed ratio would follow the rounding noise). The coefficient stays with its cell
// (no max with the upwind neighbour: its stencil would pass three ghost
// layers). It is written to field 0 of the dir-flux array, which the flux
// kernel of dir fills only afterwards; the reconstruction blends both
// interface values of the cell toward its value, f q + (1 - f) a, before the
// parabola constraints.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

template <int DIR, typename T>
__device__ __forceinline__ void b_flatten(const BlockView& v, PhysArgs ph, const T* __restrict__ P,
                                          T* __restrict__ Fl, long t) {
    const int e1 = v.n1 + 2, e2 = v.n2 + 2, e3 = v.n3 + 2;
    if (t >= (long)e1 * e2 * e3) return;
    const int i = (int)(t % e1) - 1, j = (int)((t / e1) % e2) - 1, k = (int)(t / ((long)e1 * e2)) - 1;
    const long c = cidx(v, i, j, k);
    const long st = (DIR == 1) ? 1 : ((DIR == 2) ? (long)v.n1p : (long)v.n1p * v.n2p);
    const T* u = P + UU * v.nc + c;
    const T* w = P + (U1 + DIR - 1) * v.nc + c;
    const T gm1 = (T)(ph.gam - 1.0);
    // products rounded on their own (no contraction into the differences)
    const T pm = mul_rn(gm1, u[-st]), pp = mul_rn(gm1, u[st]);
    const T dp1 = pp - pm;
    const T dp2 = mul_rn(gm1, u[2 * st] - u[-2 * st]);
    const T pmin = pm < pp ? pm : pp;
    const T a1 = fabs(dp1), a2 = fabs(dp2);
    T f = T(0);
    if (a1 > mul_rn(T(0.33), pmin) && w[-st] > w[st]) {
        if (a2 == T(0)) {
            f = T(1);
        } else {
            const T x = mul_rn(T(10), a1 / a2 - T(0.75));
            f = x < T(0) ? T(0) : (x > T(1) ? T(1) : x);
        }
    }
    Fl[c] = f;
}

template <int DIR, typename T>
__global__ void k_flatten(BlockView v, PhysArgs ph, const T* __restrict__ P, T* __restrict__ Fl) {
    b_flatten<DIR, T>(v, ph, P, Fl, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__device__ __forceinline__ void flatten_edges(T f, T qc, T& l, T& r) {
    l = f * qc + (T(1) - f) * l;
    r = f * qc + (T(1) - f) * r;
}

// entropy tracer kappa = p / rho^gam of every padded cell into K: one power per
// cell; the reconstruction carries kappa to the faces like a primitive
// (predictor: also into Kn, the entropy slot of the U^n cache, where the cell
// update takes it for U^n instead of forming the power again; in mixed
// precision this kappa is the FP32 one, like the entropy fluxes)
template <typename T>
__device__ __forceinline__ void b_kappa(const BlockView& v, T gam, const T* __restrict__ P, T* __restrict__ K,
                                        long t, double* __restrict__ Kn = nullptr) {
    const long n = (long)v.n1p * v.n2p * v.n3p;
    if (t >= n) return;
    const T kap = (gam - T(1)) * P[UU * v.nc + t] * pow_pos(P[RHO * v.nc + t], -gam);
    K[t] = kap;
    if (Kn) Kn[t] = (double)kap;
}

template <typename T>
__global__ void k_kappa(BlockView v, T gam, const T* __restrict__ P, T* __restrict__ K, double* __restrict__ Kn) {
    b_kappa<T>(v, gam, P, K, (long)blockIdx.x * blockDim.x + threadIdx.x, Kn);
}

template <int DIR>
__device__ __forceinline__ int recon_var(int n) {  // the n-th of the 7 reconstructed primitives
    return n + (n >= B1 + DIR - 1 ? 1 : 0);
}

template <typename T>
__device__ __forceinline__ T limited_slope(int recon, T qm, T q0, T qp) {
    return (recon == HAMR_RECON_MC) ? mc_slope_i(qm, q0, qp) : minmod_slope_i(qm, q0, qp);
}

// the n-th reconstructed variable's source field and its edge-value field
template <int DIR, typename T>
__device__ __forceinline__ const T* recon_src(const BlockView& v, int n, const T* P, const T* K) {
    return (n < 7) ? P + (long)recon_var<DIR>(n) * v.nc : K;
}
template <int DIR>
__device__ __forceinline__ int recon_dst(int n) {
    return (n < 7) ? recon_var<DIR>(n) : B1 + DIR - 1;
}

template <typename T>
__device__ __forceinline__ void b_recon_row(const BlockView& v, PhysArgs ph, const T* __restrict__ P,
                                            const T* __restrict__ K, const T* __restrict__ Fl,
                                            T* __restrict__ QL, T* __restrict__ QR, long t) {
    const int n2 = v.n2 + 2, n3 = v.n3 + 2;
    const int ntile = (v.n1 + 2 + RECON_TILE - 1) / RECON_TILE;
    const long w = t >> 5;  // whole warps leave or stay together
    if (w >= (long)ntile * n2 * n3 * 8) return;
    const int lane = (int)(t & 31);
    const int tile = (int)(w % ntile);
    long rest = w / ntile;
    const int j = (int)(rest % n2) - 1;
    rest /= n2;
    const int k = (int)(rest % n3) - 1;
    const int nv = (int)(rest / n3);
    const int q = recon_dst<1>(nv);
    const int i = RECON_TILE * tile - 3 + lane;               // lanes 2..29 produce cells tile*28-1 .. +27
    const int ic = min(max(i, -NG), v.n1 + NG - 1);           // loads stay inside the padded row
    const long c = cidx(v, 0, j, k);
    const T qc = recon_src<1>(v, nv, P, K)[c + ic];
    const T qm = __shfl_up_sync(0xffffffffu, qc, 1);
    const T qp = __shfl_down_sync(0xffffffffu, qc, 1);
    T l, r;
    if (ph.recon == HAMR_RECON_PPM) {
        // the same differences and formulas as the pencil sweep (identical edge values)
        const T dr = qp - qc;
        const T dl = __shfl_up_sync(0xffffffffu, dr, 1);
        const T sc = mc_slope_d(dl, dr, qp - qm);             // valid on lanes 1..30
        const T sp = __shfl_down_sync(0xffffffffu, sc, 1);
        r = ppm_face_d(qc, dr, sc, sp);                       // interface i+1/2, valid on lanes 1..29
        l = __shfl_up_sync(0xffffffffu, r, 1);                // interface i-1/2, valid on lanes 2..30
        if (ph.flatten) flatten_edges(Fl[c + ic], qc, l, r);
        ppm_limit(qc, l, r);
    } else {
        const T dq = limited_slope(ph.recon, qm, qc, qp);
        l = qc - T(0.5) * dq;
        r = qc + T(0.5) * dq;
    }
    if (lane >= 2 && lane <= 29 && i <= v.n1) {
        QL[q * v.nc + c + i] = l;
        QR[q * v.nc + c + i] = r;
    }
}

template <int DIR, typename T>
__device__ __forceinline__ void b_recon_sweep(const BlockView& v, PhysArgs ph, const T* __restrict__ P,
                                              const T* __restrict__ K, const T* __restrict__ Fl,
                                              T* __restrict__ QL, T* __restrict__ QR, long t) {
    // cells along the sweep: -1..n_dir; across: the two other directions, the faster one first
    // (x1 for the x2 and x3 sweeps, so that loads and stores coalesce; x2 for the x1 sweep)
    const int na = (DIR == 1 ? v.n1 : (DIR == 2 ? v.n2 : v.n3)) + 2;
    const int seglen = ph.recon_seg;
    const int nseg = (na + seglen - 1) / seglen;
    const int n1 = (DIR == 1 ? v.n2 : v.n1) + 2, no = (DIR == 3 ? v.n2 : v.n3) + 2;
    if (t >= (long)n1 * no * nseg * 8) return;
    const int i = (int)(t % n1) - 1;
    long rest = t / n1;
    const int o = (int)(rest % no) - 1;
    rest /= no;
    const int seg = (int)(rest % nseg);
    const int nv = (int)(rest / nseg);
    const long st = (DIR == 1) ? 1L : ((DIR == 2) ? (long)v.n1p : (long)v.n1p * v.n2p);
    const int a0 = seg * seglen - 1;
    const int ncell = min(seglen, na - 1 - a0);           // cells a0 .. a0 + ncell - 1 (<= n_dir)
    const long co = (DIR == 1) ? cidx(v, a0, i, o) : ((DIR == 2) ? cidx(v, i, a0, o) : cidx(v, i, o, a0));
    const long c0 = (long)recon_dst<DIR>(nv) * v.nc + co;
    const T* p = recon_src<DIR>(v, nv, P, K) + co;
    if (ph.recon == HAMR_RECON_PPM) {
        // each difference of neighbours is formed once and serves two slopes and a face
        const T qmm = p[-2 * st], qm = p[-st];
        T qc = p[0], qp = p[st];
        const T dmm = qm - qmm, dm = qc - qm;
        T dc = qp - qc;
        const T sm = mc_slope_d(dmm, dm, qc - qmm);
        T sc = mc_slope_d(dm, dc, qp - qm);
        T fl = ppm_face_d(qm, dm, sm, sc);  // interface a0 - 1/2
        for (int m = 0; m < ncell; m++) {
            const T qpp = p[(m + 2) * st];
            const T dp = qpp - qp;
            const T sp = mc_slope_d(dc, dp, qpp - qc);
            const T fr = ppm_face_d(qc, dc, sc, sp);  // interface a + 1/2
            T l = fl, r = fr;
            if (ph.flatten) flatten_edges(Fl[co + m * st], qc, l, r);
            ppm_limit(qc, l, r);
            QL[c0 + m * st] = l;
            QR[c0 + m * st] = r;
            qc = qp;
            qp = qpp;
            dc = dp;
            sc = sp;
            fl = fr;
        }
    } else {
        T qm = p[-st], qc = p[0];
        for (int m = 0; m < ncell; m++) {
            const T qp = p[(m + 1) * st];
            const T dq = limited_slope(ph.recon, qm, qc, qp);
            QL[c0 + m * st] = qc - T(0.5) * dq;
            QR[c0 + m * st] = qc + T(0.5) * dq;
            qm = qc;
            qc = qp;
        }
    }
}

// one thread per cell (FP32: the slope and interface arithmetic is cheap next to
// the loads, and a thread per cell keeps more loads in flight than a sweep)
template <int DIR, typename T>
__device__ __forceinline__ void b_recon_cell(const BlockView& v, PhysArgs ph, const T* __restrict__ P,
                                             const T* __restrict__ K, const T* __restrict__ Fl,
                                             T* __restrict__ QL, T* __restrict__ QR, long t) {
    const int e1 = v.n1 + 2, e2 = v.n2 + 2, e3 = v.n3 + 2;
    if (t >= (long)e1 * e2 * e3) return;
    const int i = (int)(t % e1) - 1, j = (int)((t / e1) % e2) - 1, k = (int)(t / ((long)e1 * e2)) - 1;
    const long c = cidx(v, i, j, k);
    const long st = (DIR == 1) ? 1 : ((DIR == 2) ? (long)v.n1p : (long)v.n1p * v.n2p);
#pragma unroll
    for (int n = 0; n < 8; n++) {
        const int q = recon_dst<DIR>(n);
        const T* p = recon_src<DIR>(v, n, P, K) + c;
        T l, r;
        if (ph.recon == HAMR_RECON_PPM) {
            const T qmm = p[-2 * st], qm = p[-st], qc = p[0], qp = p[st], qpp = p[2 * st];
            const T dmm = qm - qmm, dm = qc - qm, dp = qp - qc, dpp = qpp - qp;
            const T sm = mc_slope_d(dmm, dm, qc - qmm), sc = mc_slope_d(dm, dp, qp - qm),
                    sp = mc_slope_d(dp, dpp, qpp - qc);
            l = ppm_face_d(qm, dm, sm, sc);
            r = ppm_face_d(qc, dp, sc, sp);
            if (ph.flatten) flatten_edges(Fl[c], qc, l, r);
            ppm_limit(qc, l, r);
        } else {
            const T dq = limited_slope(ph.recon, p[-st], p[0], p[st]);
            l = p[0] - T(0.5) * dq;
            r = p[0] + T(0.5) * dq;
        }
        QL[q * v.nc + c] = l;
        QR[q * v.nc + c] = r;
    }
}

// FP64: the non-redundant row and pencil forms; FP32: one thread per cell
template <int DIR, typename T>
__device__ __forceinline__ void b_recon(const BlockView& v, PhysArgs ph, const T* __restrict__ P,
                                        const T* __restrict__ K, const T* __restrict__ Fl, T* __restrict__ QL,
                                        T* __restrict__ QR, long t) {
    if constexpr (!std::is_same<T, double>::value)
        b_recon_cell<DIR>(v, ph, P, K, Fl, QL, QR, t);
    else if constexpr (DIR == 1) {
        if (ph.recon_x1_sweep)
            b_recon_sweep<1>(v, ph, P, K, Fl, QL, QR, t);
        else
            b_recon_row(v, ph, P, K, Fl, QL, QR, t);
    } else {
        b_recon_sweep<DIR>(v, ph, P, K, Fl, QL, QR, t);
    }
}

template <int DIR, typename T>
__global__ void k_recon(BlockView v, PhysArgs ph, const T* __restrict__ P, const T* __restrict__ K,
                        const T* __restrict__ Fl, T* __restrict__ QL, T* __restrict__ QR) {
    b_recon<DIR, T>(v, ph, P, K, Fl, QL, QR, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// FP32 copy of the 8 primitive fields over the whole padded block (mixed precision)
__device__ __forceinline__ void b_to_f32(const BlockView& v, const double* __restrict__ P, float* __restrict__ P32,
                                         long t) {
    const long n = (long)v.n1p * v.n2p * v.n3p;
    if (t >= n) return;
#pragma unroll
    for (int q = 0; q < NPRIM; q++) P32[q * v.nc + t] = (float)P[q * v.nc + t];
}

__global__ void k_to_f32(BlockView v, const double* __restrict__ P, float* __restrict__ P32) {
    b_to_f32(v, P, P32, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// the tables a face flux of direction DIR reads, in the flux precision
template <int DIR, typename T>
__device__ __forceinline__ const T* face_table(const BlockView& v) {
    if constexpr (std::is_same<T, double>::value)
        return (DIR == 1) ? v.gf1 : ((DIR == 2) ? v.gf2 : v.gc);
    else
        return (DIR == 1) ? v.gf1_32 : ((DIR == 2) ? v.gf2_32 : v.gc32);
}


// ---------------------------------------------------------------- fluxes
// One side's share of an HLL face flux: cF F + cU U of that side's state, where F is its flux row
// along DIR and U its conserved row (both without sqrt(-g), which the weights carry), accumulated
// into acc (FIRST: acc is set). Uses that the two rows differ only in the contravariant index:
//   cF F_q + cU U_q = eta (cF u^D + cU u^t) u_q - (cF b^D + cU b^t) b_q + (cF delta^D_q + cU delta^t_q) ptot,
// the mass row rho (cF u^D + cU u^t), the energy row adding it, the entropy row kappa times it, and
// the transverse B slots cF (b^i u^D - b^D u^i) + cU B^i (U's B^i slot is the edge value itself).
template <int DIR, bool FIRST, typename T>
__device__ __forceinline__ void hll_side(const T pr[NPRIM], const Fluid<T>& s, T gam, T kappa, T cF, T cU,
                                         T acc[NFLUX]) {
    const T p = (gam - T(1)) * pr[UU];
    const T eta = pr[RHO] + pr[UU] + p + s.bsq;
    const T ptot = p + T(0.5) * s.bsq;
    const T tu = cF * s.ucon[DIR] + cU * s.ucon[0];
    const T tb = cF * s.bcon[DIR] + cU * s.bcon[0];
    const T a = eta * tu;
    const T mass = pr[RHO] * tu;
    const T cfp = cF * ptot;
    constexpr int i1 = (DIR == 1) ? 2 : 1, i2 = (DIR == 3) ? 2 : 3;
    const T fu = cF * s.ucon[DIR], fb = cF * s.bcon[DIR];
    // the second side's terms are summed into the running total innermost, so its products fuse
    // with the accumulation (no separate addition per component)
    T r[NFLUX];
#pragma unroll
    for (int q = 0; q < NFLUX; q++) r[q] = acc[q];
    if constexpr (FIRST) {
        acc[0] = mass;
        acc[1] = a * s.ucov[0] + (-tb * s.bcov[0] + (cU * ptot + mass));
        acc[2] = (DIR == 1) ? a * s.ucov[1] + (-tb * s.bcov[1] + cfp) : a * s.ucov[1] - tb * s.bcov[1];
        acc[3] = (DIR == 2) ? a * s.ucov[2] + (-tb * s.bcov[2] + cfp) : a * s.ucov[2] - tb * s.bcov[2];
        acc[4] = (DIR == 3) ? a * s.ucov[3] + (-tb * s.bcov[3] + cfp) : a * s.ucov[3] - tb * s.bcov[3];
        acc[5] = kappa * mass;
        acc[6] = s.bcon[i1] * fu + (-fb * s.ucon[i1] + cU * pr[B1 + i1 - 1]);
        acc[7] = s.bcon[i2] * fu + (-fb * s.ucon[i2] + cU * pr[B1 + i2 - 1]);
    } else {
        acc[0] = r[0] + mass;
        acc[1] = a * s.ucov[0] + (-tb * s.bcov[0] + (cU * ptot + (mass + r[1])));
        acc[2] = a * s.ucov[1] + (-tb * s.bcov[1] + ((DIR == 1) ? cfp + r[2] : r[2]));
        acc[3] = a * s.ucov[2] + (-tb * s.bcov[2] + ((DIR == 2) ? cfp + r[3] : r[3]));
        acc[4] = a * s.ucov[3] + (-tb * s.bcov[3] + ((DIR == 3) ? cfp + r[4] : r[4]));
        acc[5] = kappa * mass + r[5];
        acc[6] = s.bcon[i1] * fu + (-fb * s.ucon[i1] + (cU * pr[B1 + i1 - 1] + r[6]));
        acc[7] = s.bcon[i2] * fu + (-fb * s.ucon[i2] + (cU * pr[B1 + i2 - 1] + r[7]));
    }
}

// HLLE (or LLF) flux through every dir-face: faces 0..n_dir, -1..n_e across.
template <int DIR, typename T>
__device__ __forceinline__ void b_flux(const BlockView& v, PhysArgs ph, const T* __restrict__ QL,
                                             const T* __restrict__ QR, const double* __restrict__ Bf,
                                             double* __restrict__ F, long t) {
    const int nn[4] = {0, v.n1, v.n2, v.n3};
    const int e1 = (DIR == 1) ? nn[1] + 1 : nn[1] + 2;
    const int e2 = (DIR == 2) ? nn[2] + 1 : nn[2] + 2;
    const int e3 = (DIR == 3) ? nn[3] + 1 : nn[3] + 2;
    if (t >= (long)e1 * e2 * e3) return;
    const int i = (int)(t % e1) - (DIR == 1 ? 0 : 1);
    const int j = (int)((t / e1) % e2) - (DIR == 2 ? 0 : 1);
    const int k = (int)(t / ((long)e1 * e2)) - (DIR == 3 ? 0 : 1);
    const long c = cidx(v, i, j, k);
    const long st = (DIR == 1) ? 1 : ((DIR == 2) ? (long)v.n1p : (long)v.n1p * v.n2p);
    Metric<T> m;
    load_metric(face_table<DIR, T>(v), v.n2d, gidx(v, i, j), m);
    // single-block mixed precision: the two field slots (6, 7) also in FP32, after the FP64 fields
    float* F32 = (std::is_same<T, float>::value && ph.flux32) ? reinterpret_cast<float*>(F + NFLUX * v.nc) : nullptr;
    if (m.gdet == T(0)) {  // face on the polar axis: no area
#pragma unroll
        for (int q = 0; q < NFLUX; q++) F[q * v.nc + c] = 0.0;
        if (F32) F32[c] = F32[v.nc + c] = 0.0f;
        return;
    }
    T pl[NPRIM], pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) {
        if (q == B1 + DIR - 1) continue;
        pl[q] = QR[q * v.nc + c - st];
        pr[q] = QL[q * v.nc + c];
    }
    const T bn = (T)Bf[(DIR - 1) * v.nc + c] * m.igdet;
    pl[B1 + DIR - 1] = bn;
    pr[B1 + DIR - 1] = bn;
    // the entropy tracer's edge values sit in the B^dir fields
    const T kapl = QR[(B1 + DIR - 1) * v.nc + c - st], kapr = QL[(B1 + DIR - 1) * v.nc + c];
    const T gam = (T)ph.gam;
    Fluid<T> sl, sr;
    T Al, Bl, sdl, Ar, Br, sdr;
    fluid_state(pl, m, sl);
    wave_quadratic(pl, sl, m, DIR, gam, Al, Bl, sdl);
    fluid_state(pr, m, sr);
    wave_quadratic(pr, sr, m, DIR, gam, Ar, Br, sdr);
    // F sqrt(-g) = wl F_L + wr F_R - wc (U_R - U_L): the weights first, then each side's
    // wl F_L + wc U_L (wr F_R - wc U_R) from its fluid state in one pass (hll_side), which forms no
    // U or F row on its own
    T wl, wr, wc;
    const T half = T(0.5) * m.gdet;
    // FP64 HLL with both sides' A > 0 (always for admissible states: A = u^t u^t (w - gam p) - (b^2 + gam p) g^{tt}
    // with g^{tt} < 0 and w - gam p > 0 for gam < 2): the speeds are numerators over AA = A_L A_R, so the
    // maxima compare numerators and the weights
    //   wl = Nmax sqrt(-g) / (Nmax + Nmin), wr = Nmin sqrt(-g) / (Nmax + Nmin), wc = wl Nmin / AA
    // come from one division. AA (Nmax + Nmin) ~ A^4 leaves FP32's range in the floored atmosphere (A ~ rho),
    // so FP32 keeps the form below (its divisions do not take the FP64 pipe).
    const T AA = Al * Ar;
    if (std::is_same<T, double>::value && ph.riemann != HAMR_FLUX_LLF && FBits<T>::of(Al) > 0 &&
        FBits<T>::of(Ar) > 0) {  // sign tests on the integer pipe
        const T npl = (Bl + sdl) * Ar, nml = (Bl - sdl) * Ar;
        const T npr = (Br + sdr) * Al, nmr = (Br - sdr) * Al;
        const T nmax = max_i(T(0), max_i(npl, npr));
        const T nmin = max_i(T(0), max_i(-nml, -nmr));
        const T ns = nmax + nmin;
        if (FBits<T>::of(ns) > 0) {  // ns >= 0
            const T r = m.gdet * (T(1) / (AA * ns));  // a reciprocal: 5 FP64 instructions, a quotient 8
            const T ra = r * AA;
            wl = nmax * ra;
            wr = nmin * ra;
            wc = nmax * nmin * r;
        } else {
            wl = wr = half;
            wc = T(0);
        }
    } else {
        // general form: the two sides' 1/A from one division
        const T iAA = T(1) / AA;
        const T iAl = Ar * iAA, iAr = Al * iAA;
        const T vpl = (Bl + sdl) * iAl, vml = (Bl - sdl) * iAl;
        const T vpr = (Br + sdr) * iAr, vmr = (Br - sdr) * iAr;
        // maxima on the integer pipe
        const T cmax = max_i(T(0), max_i(vpl, vpr));
        const T cmin = max_i(T(0), max_i(-vml, -vmr));
        if (ph.riemann == HAMR_FLUX_LLF) {
            wl = wr = half;
            wc = half * max_i(cmax, cmin);
        } else if (cmax + cmin > T(0)) {
            // (cmin F_R + cmax F_L - cmax cmin (U_R - U_L)) sqrt(-g) / (cmax + cmin)
            const T w = m.gdet / (cmax + cmin);
            wl = cmax * w;
            wr = cmin * w;
            wc = cmax * wr;
        } else {
            wl = wr = half;
            wc = T(0);
        }
    }
    T acc[NFLUX];
    hll_side<DIR, true>(pl, sl, gam, kapl, wl, wc, acc);
    hll_side<DIR, false>(pr, sr, gam, kapr, wr, -wc, acc);
#pragma unroll
    for (int q = 0; q < NFLUX; q++) F[q * v.nc + c] = (double)acc[q];
    if (F32) {
        F32[c] = (float)acc[6];
        F32[v.nc + c] = (float)acc[7];
    }
}

template <int DIR, typename T>
__global__ void __launch_bounds__(256, 2) k_flux(BlockView v, PhysArgs ph, const T* __restrict__ QL,
                                             const T* __restrict__ QR, const double* __restrict__ Bf,
                                             double* __restrict__ F) {
    b_flux<DIR, T>(v, ph, QL, QR, Bf, F, (long)blockIdx.x * blockDim.x + threadIdx.x);
}


// ---------------------------------------------------------------- EMFs
// edge EMFs as the average of the 4 neighbouring face fluxes of B (Sec. 2.5).
// E1 and E3 on the polar axis are 0. With T = float (mixed precision) the
// average is formed in FP32; every face shares the one stored edge value, so
// the FP64 curl in the CT update still keeps div B at FP64 roundoff.
//
// Upwinded EMFs (Ec != nullptr; Gardiner & Stone 2005, the paper's usual
// setting): for an edge between face directions p and q, with e_p / e_q the
// EMF values the p- / q-faces carry and Ec the EMF of the cell-centred state,
//   E = average + 1/4 [D_q(q-3/4) - D_q(q-1/4)] + 1/4 [D_p(p-3/4) - D_p(p-1/4)],
//   D_q(q-1/4) = Ec(c, q) - e_q(c, q-1/2), D_q(q-3/4) = e_q(c, q-1/2) - Ec(c, q-1),
// in the cell column c (p-1 or p) upwind of the mass flux through the p-face
// beside the edge (both averaged when it is zero); D_p likewise.

// the cell-centred EMFs sqrt(-g)(b^2 u^3 - b^3 u^2, b^3 u^1 - b^1 u^3, b^1 u^2 - b^2 u^1)
// of every cell -1..n of the block, from the stage state (centre B in slots 5..7)
__device__ __forceinline__ void b_cell_emf(const BlockView& v, const double* __restrict__ P, double* __restrict__ Ec,
                                           long t) {
    const int e1 = v.n1 + 2, e2 = v.n2 + 2, e3 = v.n3 + 2;
    if (t >= (long)e1 * e2 * e3) return;
    const int i = (int)(t % e1) - 1, j = (int)((t / e1) % e2) - 1, k = (int)(t / ((long)e1 * e2)) - 1;
    const long c = cidx(v, i, j, k);
    Metric<double> m;
    load_metric(v.gc, v.n2d, gidx(v, i, j), m);
    double pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pr[q] = P[q * v.nc + c];
    Fluid<double> s;
    fluid_state(pr, m, s);
    Ec[c] = (s.bcon[2] * s.ucon[3] - s.bcon[3] * s.ucon[2]) * m.gdet;
    Ec[v.nc + c] = (s.bcon[3] * s.ucon[1] - s.bcon[1] * s.ucon[3]) * m.gdet;
    Ec[2 * v.nc + c] = (s.bcon[1] * s.ucon[2] - s.bcon[2] * s.ucon[1]) * m.gdet;
}

__global__ void k_cell_emf(BlockView v, const double* __restrict__ P, double* __restrict__ Ec) {
    b_cell_emf(v, P, Ec, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__device__ __forceinline__ T upwind_pick(T mass_flux, T lower, T upper) {
    return mass_flux > T(0) ? lower : (mass_flux < T(0) ? upper : T(0.5) * (lower + upper));
}

// the Gardiner-Stone corrections of one edge. Offsets are cells along p and q from the
// edge's cell c: sp, sq the index strides of p and q; Fp / Fq the flux arrays of the p / q
// faces, slp / slq their B-flux slots with signs gp / gq (the EMF a face carries is g F[sl]);
// ec the cell-EMF field of the component
// field slot `slot` (6 or 7) of a face flux at cell offset i as T: the FP64 field converted, or (F32)
// the FP32 copy of slots 6 and 7 kept after the FP64 fields
template <typename T, bool F32>
__device__ __forceinline__ T ld_bflux(const double* __restrict__ F, int slot, long nc, long i) {
    if constexpr (F32) {
        static_assert(std::is_same<T, float>::value, "the FP32 slot copy serves the FP32 EMFs");
        return reinterpret_cast<const float*>(F + NFLUX * nc)[(slot - 6) * nc + i];
    } else {
        return (T)F[slot * nc + i];
    }
}

template <typename T>
__device__ __forceinline__ T gs_correction(long c, long sp, long sq, long nc, const double* __restrict__ Fp,
                                           const double* __restrict__ Fq, int slp, int slq, T gp, T gq,
                                           const double* __restrict__ ec) {
    auto ep = [&](long o) { return gp * (T)Fp[slp * nc + c + o]; };  // p-face value at cell offset o
    auto eq = [&](long o) { return gq * (T)Fq[slq * nc + c + o]; };
    auto E = [&](long o) { return (T)ec[c + o]; };
    auto mp = [&](long o) { return (T)Fp[c + o]; };  // mass flux (slot 0) through a p-face
    auto mq = [&](long o) { return (T)Fq[c + o]; };
    const T dq_lo = upwind_pick(mp(-sq), eq(-sp) - E(-sp - sq), eq(0) - E(-sq));  // D_q(q-3/4)
    const T dq_hi = upwind_pick(mp(0), E(-sp) - eq(-sp), E(0) - eq(0));           // D_q(q-1/4)
    const T dp_lo = upwind_pick(mq(-sp), ep(-sq) - E(-sp - sq), ep(0) - E(-sp));  // D_p(p-3/4)
    const T dp_hi = upwind_pick(mq(0), E(-sq) - ep(-sq), E(0) - ep(0));           // D_p(p-1/4)
    return T(0.25) * (dq_lo - dq_hi) + T(0.25) * (dp_lo - dp_hi);
}

template <typename T, bool F32 = false>
__device__ __forceinline__ void b_emf(const BlockView& v, const double* __restrict__ F1, const double* __restrict__ F2,
                      const double* __restrict__ F3, double* __restrict__ E, const double* __restrict__ Ec, long t) {
    const int e1 = v.n1 + 1, e2 = v.n2 + 1, e3 = v.n3 + 1;
    if (t >= (long)e1 * e2 * e3) return;
    const int i = (int)(t % e1), j = (int)((t / e1) % e2), k = (int)(t / ((long)e1 * e2));
    const long c = cidx(v, i, j, k);
    const long si = 1, sj = v.n1p, sk = (long)v.n1p * v.n2p, nc = v.nc;
    const bool axis = (v.bc[2] == HAMR_BC_POLAR && j == 0) || (v.bc[3] == HAMR_BC_POLAR && j == v.n2);
    const T q = T(0.25);
    // flux slots: F1 -> (B2: 6, B3: 7), F2 -> (B1: 6, B3: 7), F3 -> (B1: 6, B2: 7)
    if (i < v.n1) {
        T x = q * (ld_bflux<T, F32>(F3, 7, nc, c) + ld_bflux<T, F32>(F3, 7, nc, c - sj) -
                   ld_bflux<T, F32>(F2, 7, nc, c - sk) - ld_bflux<T, F32>(F2, 7, nc, c));
        // p = x2 faces (value -F2(B3)), q = x3 faces (value F3(B2))
        if (Ec) x += gs_correction<T>(c, sj, sk, nc, F2, F3, 7, 7, T(-1), T(1), Ec);
        E[c] = axis ? 0.0 : (double)x;
    }
    if (j < v.n2) {
        T x = q * (ld_bflux<T, F32>(F1, 7, nc, c - sk) + ld_bflux<T, F32>(F1, 7, nc, c) -
                   ld_bflux<T, F32>(F3, 6, nc, c) - ld_bflux<T, F32>(F3, 6, nc, c - si));
        // p = x1 faces (value F1(B3)), q = x3 faces (value -F3(B1))
        if (Ec) x += gs_correction<T>(c, si, sk, nc, F1, F3, 7, 6, T(1), T(-1), Ec + nc);
        E[nc + c] = (double)x;
    }
    if (k < v.n3) {
        T x = q * (ld_bflux<T, F32>(F2, 6, nc, c - si) + ld_bflux<T, F32>(F2, 6, nc, c) -
                   ld_bflux<T, F32>(F1, 6, nc, c) - ld_bflux<T, F32>(F1, 6, nc, c - sj));
        // p = x1 faces (value -F1(B2)), q = x2 faces (value F2(B1))
        if (Ec) x += gs_correction<T>(c, si, sj, nc, F1, F2, 6, 6, T(-1), T(1), Ec + 2 * nc);
        E[2 * nc + c] = axis ? 0.0 : (double)x;
    }
}

template <typename T, bool F32 = false>
__global__ void k_emf(BlockView v, const double* __restrict__ F1, const double* __restrict__ F2,
                      const double* __restrict__ F3, double* __restrict__ E, const double* __restrict__ Ec) {
    b_emf<T, F32>(v, F1, F2, F3, E, Ec, (long)blockIdx.x * blockDim.x + threadIdx.x);
}


// ---------------------------------------------------------------- CT
// staggered face update Bbar += dt curl E (Sec. 2.5, the three CT equations)
__device__ __forceinline__ void b_ct(const BlockView& v, const double* __restrict__ E, const double* Bb, double* Bo,
                     const double* __restrict__ dscal, double fac, long t) {
    const int e1 = v.n1 + 1, e2 = v.n2 + 1, e3 = v.n3 + 1;
    if (t >= (long)e1 * e2 * e3) return;
    const int i = (int)(t % e1), j = (int)((t / e1) % e2), k = (int)(t / ((long)e1 * e2));
    const long c = cidx(v, i, j, k);
    const long sj = v.n1p, sk = (long)v.n1p * v.n2p, nc = v.nc;
    const double dt = dscal[0] * fac;
    const double* E1 = E;
    const double* E2 = E + nc;
    const double* E3 = E + 2 * nc;
    if (j < v.n2 && k < v.n3) {
        const double r = (E2[c + sk] - E2[c]) * v.idx3 - (E3[c + sj] - E3[c]) * v.idx2;
        Bo[c] = Bb[c] + dt * r;
    }
    if (i < v.n1 && k < v.n3) {
        const bool axis = (v.bc[2] == HAMR_BC_POLAR && j == 0) || (v.bc[3] == HAMR_BC_POLAR && j == v.n2);
        const double r = (E3[c + 1] - E3[c]) * v.idx1 - (E1[c + sk] - E1[c]) * v.idx3;
        Bo[nc + c] = axis ? 0.0 : Bb[nc + c] + dt * r;
    }
    if (i < v.n1 && j < v.n2) {
        const double r = (E1[c + sj] - E1[c]) * v.idx2 - (E2[c + 1] - E2[c]) * v.idx1;
        Bo[2 * nc + c] = Bb[2 * nc + c] + dt * r;
    }
}

__global__ void k_ct(BlockView v, const double* __restrict__ E, const double* Bb, double* Bo,
                     const double* __restrict__ dscal, double fac) {
    b_ct(v, E, Bb, Bo, dscal, fac, (long)blockIdx.x * blockDim.x + threadIdx.x);
}


// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// sum_i v_f^i / dx^i at a cell centre (Sec. 2.1 CFL condition), given the fluid state
// (max(|v+|, |v-|) = (|B| + sd)/|A| per direction; the three terms over one denominator)
template <typename T>
__device__ __forceinline__ double inv_dt_fluid(const BlockView& v, const T pr[NPRIM], const Fluid<T>& s,
                                               const Metric<T>& m, T gam) {
    // the quadratic's leading coefficient A = (u^t)^2 (w - gam p) - (b^2 + gam p) g^{tt} is the same
    // in every direction: max(|v+|, |v-|) = (|B_d| + sqrt(B_d^2 - A C_d)) / |A| and one division
    const T p = (gam - T(1)) * pr[UU];
    const T gp = gam * p;
    const T num = s.bsq + gp;
    const T dn = pr[RHO] + pr[UU] + p - gp;
    const T ut = s.ucon[0];
    const T A = ut * ut * dn - num * m.c00;
    const T idx[3] = {to_t<T>(v.idx1), to_t<T>(v.idx2), to_t<T>(v.idx3)};
    T nsum = T(0);
#pragma unroll
    for (int d = 1; d <= 3; d++) {
        const T ud = s.ucon[d];
        const T B = ut * ud * dn - num * gcon0(m, d);
        const T C = ud * ud * dn - num * gcondd(m, d);
        nsum += (fabs(B) + root_pos(B * B - A * C)) * idx[d - 1];
    }
    return to_d(nsum / fabs(A));
}

template <typename T>
__device__ __forceinline__ double inv_dt_cell(const BlockView& v, const T pr[NPRIM], const Metric<T>& m, T gam) {
    Fluid<T> s;
    fluid_state(pr, m, s);
    return inv_dt_fluid(v, pr, s, m, gam);
}

// the rate of a cell in precision T from its (FP64) primitives
// source sqrt(-g) T^k_l Gamma^l_{nu k} at a cell centre in precision T
// (tables gc: metric and connection planes of that precision)
template <typename T, typename TT>
__device__ __forceinline__ void source_q_state(const TT* __restrict__ gc, long n2d, long g, const Metric<T>& m,
                                              const T pf[NPRIM], const Fluid<T>& s, T gam, double Q[4]) {
    const T p = (gam - T(1)) * pf[UU];
    const T eta = pf[RHO] + pf[UU] + p + s.bsq;
    const T ptot = p + T(0.5) * s.bsq;
    T Tm[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
            Tm[a][b] = eta * s.ucon[a] * s.ucov[b] - s.bcon[a] * s.bcov[b] + ((a == b) ? ptot : T(0));
    const TT* cn = gc + (long)C_CONN * n2d + g;
#pragma unroll
    for (int nu = 0; nu < 4; nu++) {
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < 4; l++)
#pragma unroll
            for (int kk = 0; kk < 4; kk++) acc += Tm[kk][l] * (T)cn[(l * 10 + sym(nu, kk)) * n2d];
        Q[nu] = to_d(acc * m.gdet);
    }
}

// The same source in FP64 from the stored metric derivatives: with the Christoffel
// symbols formed from the derivatives d_s g of the metric whose inverse raises T,
// T^k_l Gamma^l_{nu k} = (1/2) T^{kl} d_nu g_{kl} (the terms with d_k g_{l nu} - d_l g_{nu k}
// cancel against the symmetric T^{kl}), so Q_t = Q_phi = 0 (stationary, axisymmetric
// metric) and Q_1, Q_2 contract the 7 non-zero d_s g_{mn}; the same number up to
// rounding order, with a third of the operations.
__device__ __forceinline__ void source_q_dg(const double* __restrict__ gc, long n2d, long g, const Metric<double>& m,
                                            const double pf[NPRIM], const Fluid<double>& s, double gam, double Q[4]) {
    const double p = (gam - 1.0) * pf[UU];
    const double eta = pf[RHO] + pf[UU] + p + s.bsq;
    const double ptot = p + 0.5 * s.bsq;
    const double* u = s.ucon;
    const double* b = s.bcon;
    const double e0 = eta * u[0], e1 = eta * u[1], e3 = eta * u[3];
    const double T[7] = {e0 * u[0] - b[0] * b[0] + ptot * m.c00, e0 * u[1] - b[0] * b[1] + ptot * m.c01,
                         e0 * u[3] - b[0] * b[3],                e1 * u[1] - b[1] * b[1] + ptot * m.c11,
                         e1 * u[3] - b[1] * b[3] + ptot * m.c13, eta * u[2] * u[2] - b[2] * b[2] + ptot * m.c22,
                         e3 * u[3] - b[3] * b[3] + ptot * m.c33};
    const double* d = gc + (long)C_DG * n2d + g;
    double q1 = 0.0, q2 = 0.0;
#pragma unroll
    for (int k = 0; k < 7; k++) {
        q1 += T[k] * d[k * n2d];
        q2 += T[k] * d[(7 + k) * n2d];
    }
    Q[0] = 0.0;
    Q[1] = q1 * m.gdet;
    Q[2] = q2 * m.gdet;
    Q[3] = 0.0;
}

template <typename T, typename TT>
__device__ __forceinline__ void source_q(const TT* __restrict__ gc, long n2d, long g, const Metric<T>& m,
                                        const double pfd[NPRIM], double gam_d, double Q[4]) {
    T pf[NPRIM];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pf[q] = to_t<T>(pfd[q]);
    Fluid<T> s;
    fluid_state(pf, m, s);
    source_q_state(gc, n2d, g, m, pf, s, to_t<T>(gam_d), Q);
}

// ---------------------------------------------------------------- cell update
// U = U(P^n) + dts (Q(Pf) - div F); inversion with guess Pf; floors;
// the corrector also reduces the CFL rate of the new state.
// MLP: the CTA's 128 cells first run the learned guess (mlp.cuh) on the
// tensor cores; Newton starts from it, with the start from Pf as fallback.
// TS: precision of the connection source and of the CFL rate (float in mixed
// precision; the conserved accumulation and the inversion are FP64 always). With
// ph.fp64_inv the mixed form takes the FP64 source and iterates Newton in FP64
// only (without it, its Newton iteration starts in FP32, c2p.cuh).
// Floors in the drift frame (Sec. 2.7, after Ressler et al. 2017): the floor
// material, drho = rho_f - rho and du = u_f - u (each >= 0), moves with the
// drift velocity of the field lines, the part of the normal-frame velocity
// across B, v_d = v - (v.Bn / Bn^2) Bn (v_d = v where B = 0). Its stress-energy
// (no field) is added to the cell's in conserved form, the entropy slot keeps
// the cell's kappa, and the sum is inverted with the same B from rho_f, u_f at
// the drift velocity. The material brings no momentum along B, so a flow along
// the field slows as mass is added; the fluid-frame floor is applied to the
// result. false when the inversion fails (the caller then takes the fluid-frame
// floor).
__device__ __forceinline__ bool drift_floor(const Metric<double>& m, const PhysArgs& ph, double pr[NPRIM],
                                            const Fluid<double>& s, double rf, double uf) {
    const double gam = ph.gam;
    const double q1 = pr[U1], q2 = pr[U2], q3 = pr[U3];
    const double qsq = m.g11 * q1 * q1 + m.g22 * q2 * q2 + m.g33 * q3 * q3 + 2.0 * m.g13 * q1 * q3;
    const double ig = 1.0 / sqrt(1.0 + qsq);
    const double v1 = q1 * ig, v2 = q2 * ig, v3 = q3 * ig;
    const double b1 = m.alpha * pr[B1], b2 = m.alpha * pr[B2], b3 = m.alpha * pr[B3];
    const double bn2 = m.g11 * b1 * b1 + m.g22 * b2 * b2 + m.g33 * b3 * b3 + 2.0 * m.g13 * b1 * b3;
    const double vb = m.g11 * v1 * b1 + m.g22 * v2 * b2 + m.g33 * v3 * b3 + m.g13 * (v1 * b3 + v3 * b1);
    const double f = (bn2 > 0.0) ? vb / bn2 : 0.0;
    const double d1 = v1 - f * b1, d2 = v2 - f * b2, d3 = v3 - f * b3;
    const double vd2 = m.g11 * d1 * d1 + m.g22 * d2 * d2 + m.g33 * d3 * d3 + 2.0 * m.g13 * d1 * d3;
    const double gd = 1.0 / sqrt(1.0 - vd2);
    double pa[NPRIM] = {fmax(rf - pr[RHO], 0.0), fmax(uf - pr[UU], 0.0), gd * d1, gd * d2, gd * d3, 0.0, 0.0, 0.0};
    Fluid<double> sa;
    fluid_state(pa, m, sa);
    double uo[NFLUX], ua[NFLUX];
    flux_row(pr, s, 0, 1, gam, entropy_kappa(pr, gam), uo);
    flux_row(pa, sa, 0, 1, gam, 0.0, ua);
    double U[NCONS];
#pragma unroll
    for (int q = 0; q < 5; q++) U[q] = m.gdet * (uo[q] + ua[q]);
    U[C_ENT] = m.gdet * uo[5] / uo[0] * (uo[0] + ua[0]);
    double x[NPRIM];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) x[q] = pr[q];
    x[RHO] = fmax(pr[RHO], rf);
    x[UU] = fmax(pr[UU], uf);
    x[U1] = pa[U1];
    x[U2] = pa[U2];
    x[U3] = pa[U3];
    const double Bc[3] = {pr[B1], pr[B2], pr[B3]};
    int its = 0;
    if (invert(U, Bc, m, gam, x, &its, false, nullptr, ph.inversion) == INV_FAIL) return false;
    pr[RHO] = fmax(x[RHO], rf);
    pr[UU] = fmax(x[UU], uf);
    pr[U1] = x[U1];
    pr[U2] = x[U2];
    pr[U3] = x[U3];
    return true;
}

// Floors (Sec. 2.7): rho >= max(1e-7/r^2, b^2/50), u >= max(1e-9/r^(10/3),
// b^2/750) with b^2 of pr; HAMR_FLOOR_FLUID raises rho and u (utilde kept),
// HAMR_FLOOR_DRIFT adds the material in the drift frame. s: the fluid state
// of pr on entry, and again on return (recomputed where the velocity moved).
// Returns 1 where a floor applied.
__device__ __forceinline__ int cell_floors(const BlockView& v, long g, const Metric<double>& m, const PhysArgs& ph,
                                           double pr[NPRIM], Fluid<double>& s) {
    const double rf = fmax(v.gc[C_RHOFLR * v.n2d + g], s.bsq * (1.0 / 50.0));
    const double uf = fmax(v.gc[C_UFLR * v.n2d + g], s.bsq * (1.0 / 750.0));
    if (!(pr[RHO] < rf) && !(pr[UU] < uf)) return 0;
    if (ph.floor_frame == HAMR_FLOOR_DRIFT && drift_floor(m, ph, pr, s, rf, uf)) {
        fluid_state(pr, m, s);
        return 1;
    }
    if (pr[RHO] < rf) pr[RHO] = rf;
    if (pr[UU] < uf) pr[UU] = uf;
    return 1;
}

// The same floors with b^2 given (the mixed-precision update takes it from its FP32 fluid
// state); the drift frame forms the FP64 fluid state of pr where a floor applies.
__device__ __forceinline__ int cell_floors_b2(const BlockView& v, long g, const Metric<double>& m, const PhysArgs& ph,
                                              double pr[NPRIM], double bsq) {
    const double rf = fmax(v.gc[C_RHOFLR * v.n2d + g], bsq * (1.0 / 50.0));
    const double uf = fmax(v.gc[C_UFLR * v.n2d + g], bsq * (1.0 / 750.0));
    if (!(pr[RHO] < rf) && !(pr[UU] < uf)) return 0;
    if (ph.floor_frame == HAMR_FLOOR_DRIFT) {
        Fluid<double> s;
        fluid_state(pr, m, s);
        if (drift_floor(m, ph, pr, s, rf, uf)) return 1;
    }
    if (pr[RHO] < rf) pr[RHO] = rf;
    if (pr[UU] < uf) pr[UU] = uf;
    return 1;
}

// the next stage's FP32 copy of cell c (p: the returned primitives rounded to FP32) and its entropy
// tracer kappa = (gam - 1) u / rho^gam formed as the kappa pass forms it; in the corrector also the
// next step's U^n kappa (the entropy slot of the U^n cache, which the predictor reads)
__device__ __forceinline__ void store_stage32(const BlockView& v, const PhysArgs& ph, int corrector, long c,
                                              const float p[NPRIM]) {
#pragma unroll
    for (int q = 0; q < NPRIM; q++) ph.p32w[q * v.nc + c] = p[q];
    const float g32 = narrow(ph.gam);
    const float kap = (g32 - 1.0f) * p[UU] * pow_pos(p[RHO], -g32);
    ph.k32[c] = kap;
    if (corrector == 1) ph.un[(long)C_ENT * v.nc + c] = widen(kap);
}

// The floors of the mixed form in FP32: b^2 of the FP32 fluid state (like the fluxes), thresholds,
// comparisons and floor values in FP32 (pf: the returned primitives rounded to FP32, updated with
// pr); drift-frame floors take the FP64 path of cell_floors_b2
__device__ __forceinline__ int cell_floors_f32(const BlockView& v, long g, const Metric<double>& m, const PhysArgs& ph,
                                               double pr[NPRIM], float pf[NPRIM], float bsq) {
    if (ph.floor_frame == HAMR_FLOOR_DRIFT) {
        const int fl = cell_floors_b2(v, g, m, ph, pr, widen(bsq));
        if (fl)
#pragma unroll
            for (int q = 0; q < NPRIM; q++) pf[q] = narrow(pr[q]);
        return fl;
    }
    const float rf = fmaxf(narrow(v.gc[C_RHOFLR * v.n2d + g]), bsq * (1.0f / 50.0f));
    const float uf = fmaxf(narrow(v.gc[C_UFLR * v.n2d + g]), bsq * (1.0f / 750.0f));
    const bool lr = pf[RHO] < rf, lu = pf[UU] < uf;
    if (!lr && !lu) return 0;
    if (lr) {
        pf[RHO] = rf;
        pr[RHO] = widen(rf);
    }
    if (lu) {
        pf[UU] = uf;
        pr[UU] = widen(uf);
    }
    return 1;
}

template <bool MLP, typename TS>
__device__ __forceinline__ void b_update(const BlockView& v, PhysArgs ph, int corrector, const double* Pb,
                                               const double* __restrict__ Pf, const double* __restrict__ F1,
                                               const double* __restrict__ F2, const double* __restrict__ F3,
                                               const double* __restrict__ Bn, double* Un, double* Po,
                                               uint8_t* __restrict__ status, const double* __restrict__ dscal,
                                               double fac, unsigned long long* dmax, unsigned long long* dcnt, long t) {
    const long n = (long)v.n1 * v.n2 * v.n3;
    bool active = t < n;  // false again for a cell whose inversion its internal-SMR group does
    double inv = 0.0;
    int st = -1, fl = 0, its = 0;
    const double gam = ph.gam;
    Metric<double> m;
    double U[NCONS], Bc[3], pr[NPRIM];
    long c = 0, g = 0;
    int i = 0, j = 0;
    MlpCta C;
    float start32[2] = {0.0f, 0.0f};  // mixed form: the inversion's start in FP32 (see the source)
    bool have32 = false;
    const bool rescue = MLP && ph.mlp_mode == HAMR_MLP_RESCUE;
    extern __shared__ __align__(16) uint8_t mlp_smem[];
    if (MLP && !rescue) mlp_begin(C, mlp_smem, ph.mlp_img);  // the weight image streams in while U is formed
    if (active) {
        i = (int)(t % v.n1);
        j = (int)((t / v.n1) % v.n2);
        const int k = (int)(t / ((long)v.n1 * v.n2));
        c = cidx(v, i, j, k);
        g = gidx(v, i, j);
        const long nc = v.nc;
        load_metric(v.gc, v.n2d, g, m);
        double pf[NPRIM];
#pragma unroll
        for (int q = 0; q < NPRIM; q++) pf[q] = Pf[q * nc + c];
        // in the predictor the base state is the stage state (Pb == Pf): with an FP64
        // source one fluid state serves U^n and the source
        const bool share = std::is_same<TS, double>::value && !corrector && Pb == Pf;
        Fluid<double> sf;
        if (share) fluid_state(pf, m, sf);
        // U^n
        if (!corrector) {
            double row[NFLUX];
            if (share) {  // kappa of P^n from the predictor's entropy-tracer pass
                flux_row(pf, sf, 0, 1, gam, Un[C_ENT * nc + c], row);
            } else {
                double pb[NPRIM];
#pragma unroll
                for (int q = 0; q < NPRIM; q++) pb[q] = Pb[q * nc + c];
                Fluid<double> s;
                fluid_state(pb, m, s);
                flux_row(pb, s, 0, 1, gam, Un[C_ENT * nc + c], row);  // kappa from the tracer pass
            }
#pragma unroll
            for (int q = 0; q < NCONS; q++) {
                U[q] = row[q] * m.gdet;
                Un[q * nc + c] = U[q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < NCONS; q++) U[q] = Un[q * nc + c];
        }
        // source sqrt(-g) T^k_l Gamma^l_{nu k} at the centre, from Pf
        double Q[4];
        if constexpr (std::is_same<TS, double>::value) {
            if (share) {
                source_q_dg(v.gc, v.n2d, g, m, pf, sf, gam, Q);
            } else {
                Fluid<double> s;
                fluid_state(pf, m, s);
                source_q_dg(v.gc, v.n2d, g, m, pf, s, gam, Q);
            }
        } else if (ph.fp64_inv) {  // mixed form with the FP64 source of the FP64 path
            Fluid<double> s;
            fluid_state(pf, m, s);
            source_q_dg(v.gc, v.n2d, g, m, pf, s, gam, Q);
        } else {
            // the FP32 source of the stage state: its FP32 copy, the values (float)pf exactly
            Metric<float> mf;
            load_metric(v.gc32, v.n2d, g, mf);
            float p32[NPRIM];
#pragma unroll
            for (int q = 0; q < NPRIM; q++) p32[q] = v.P32[q * nc + c];
            Fluid<float> s32;
            fluid_state(p32, mf, s32);
            source_q_state(v.gc32, v.n2d, g, mf, p32, s32, narrow(gam), Q);
            // the inversion's start from the same state (it only seeds the FP32 iterations)
            const float qsq = p32[U1] * s32.ucov[1] + p32[U2] * s32.ucov[2] + p32[U3] * s32.ucov[3];
            const float gsq = 1.0f + qsq;
            start32[0] = (p32[RHO] + narrow(gam) * p32[UU]) * gsq;
            start32[1] = qsq / gsq;
            have32 = true;
        }
        const double dts = dscal[0] * fac;
        const double a1 = dts * v.idx1, a2 = dts * v.idx2, a3 = dts * v.idx3;  // dt / dx^i
        const long sj = v.n1p, sk = (long)v.n1p * v.n2p;
#pragma unroll
        for (int q = 0; q < NCONS; q++) {
            // U + dt (Q - div F): the flux differences times dt/dx^i taken off one by one
            double u = (q >= C_EN && q <= C_S3) ? fma(dts, Q[q - C_EN], U[q]) : U[q];
            u = fma(-a1, F1[q * nc + c + 1] - F1[q * nc + c], u);
            u = fma(-a2, F2[q * nc + c + sj] - F2[q * nc + c], u);
            U[q] = fma(-a3, F3[q * nc + c + sk] - F3[q * nc + c], u);
        }
        centre_field(v, Bn, i, j, k, m.igdet, Bc);
#pragma unroll
        for (int q = 0; q < NPRIM; q++) pr[q] = pf[q];
        pr[B1] = Bc[0];
        pr[B2] = Bc[1];
        pr[B3] = Bc[2];
        if (ph.smr > 0 && smr_width(v, ph, j) > 1) {  // inverted with its group (k_smr_cells)
#pragma unroll
            for (int q = 0; q < NCONS; q++) ph.smr_u[q * nc + c] = U[q];
            active = false;
        }
    }
    // inversion: energy attempts from the start(s), then the entropy backup
    C2PWork w;
    if (active)
        c2p_prepare(U, Bc, m, gam, pr, w, ph.inversion, (std::is_same<TS, float>::value && !ph.fp64_inv) ? 1 : 0,
                    have32 ? start32 : nullptr, ph.igam, ph.gfac);
    if (MLP) {
        // first: the network's start, then the plain one; rescue: the plain start, then the
        // network's where it failed (the CTA runs the network only if one of its cells failed)
        if (rescue && active) c2p_attempt_plain(w, gam);
        if (__syncthreads_or(active && !w.ok)) {
            if (rescue) mlp_begin(C, mlp_smem, ph.mlp_img);
            float f[MLP_NIN], y[MLP_NOUT];
            if (active) mlp_features(w.S, U[C_RHO], U[C_ENT], m, v.x1min + (i + 0.5) * v.dx1, gam, f);
            const bool ran = mlp_infer(C, f, active, y);
            mlp_end(C);
            if (!C.ok && threadIdx.x == 0 && ph.mlp_err) atomicExch(ph.mlp_err, 1);
            if (active && ran && !w.ok) {
                double g2[2];
                mlp_guess(w.S.D, y, g2);
                c2p_attempt(w, gam, g2[0], g2[1]);
            }
        } else if (!rescue) {
            mlp_end(C);
        }
    }
    if (active) {
        if (!rescue) c2p_attempt_plain(w, gam);
        its = w.its;
        st = c2p_finish(w, U, m, gam, pr);
        uint8_t sb = (st == INV_ENTROPY) ? ST_ENTROPY : ((st == INV_FAIL) ? ST_FAIL : 0);
        // the fluid state of the returned primitives serves the floors (b^2) and the CFL rate (u^mu,
        // b^mu and b^2 do not depend on rho and u_g, which are all the floors change). The floors take
        // b^2 of these primitives, not of the inversion's own (W, v^2), which differ from them by the
        // Newton tolerance (more where v^2 was clamped), and the floor rho = b^2/50 would carry that.
        if constexpr (std::is_same<TS, double>::value) {
            Fluid<double> s;
            const bool need_fluid = ph.floors || corrector == 1;
            if (need_fluid) fluid_state(pr, m, s);
            if (ph.floors) {
                fl = cell_floors(v, g, m, ph, pr, s);
                if (fl) sb |= ST_FLOOR;
            }
#pragma unroll
            for (int q = 0; q < NPRIM; q++) Po[q * v.nc + c] = pr[q];
            if (corrector == 1) inv = inv_dt_fluid(v, pr, s, m, gam);
        } else {
            // mixed precision: one FP32 fluid state of the returned primitives gives the floors'
            // b^2 (the thresholds b^2/50 and b^2/750 to FP32 accuracy, like the fluxes) and the
            // FP32 CFL rate; drift-frame floors form the FP64 state they need themselves
            Metric<TS> mf;
            load_metric(v.gc32, v.n2d, g, mf);
            TS pf32[NPRIM];
#pragma unroll
            for (int q = 0; q < NPRIM; q++) pf32[q] = to_t<TS>(pr[q]);
            Fluid<TS> s32;
            fluid_state(pf32, mf, s32);
            if (ph.floors) {
                fl = cell_floors_f32(v, g, m, ph, pr, pf32, s32.bsq);
                if (fl) {
                    sb |= ST_FLOOR;
                    if (ph.floor_frame == HAMR_FLOOR_DRIFT && corrector == 1) fluid_state(pf32, mf, s32);
                }
            }
#pragma unroll
            for (int q = 0; q < NPRIM; q++) Po[q * v.nc + c] = pr[q];
            if (corrector == 1) inv = inv_dt_fluid(v, pf32, s32, mf, to_t<TS>(gam));
            if (ph.stage32) store_stage32(v, ph, corrector, c, pf32);
        }
        status[c] |= sb;
    }
    // warp-aggregated counters and CFL max
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long c_ok = warp_sum((unsigned long long)(st == INV_OK));
    const unsigned long long c_en = warp_sum((unsigned long long)(st == INV_ENTROPY));
    const unsigned long long c_fa = warp_sum((unsigned long long)(st == INV_FAIL));
    const unsigned long long c_fl = warp_sum((unsigned long long)fl);
    const unsigned long long c_it = warp_sum((unsigned long long)(active ? its : 0));
    const double wmax = warp_max(inv);
    if (lane == 0) {
        if (c_ok) atomicAdd(&dcnt[0], c_ok);
        if (c_en) atomicAdd(&dcnt[1], c_en);
        if (c_fa) atomicAdd(&dcnt[2], c_fa);
        if (c_fl) atomicAdd(&dcnt[3], c_fl);
        if (c_it) atomicAdd(&dcnt[4], c_it);
        if (corrector == 1 && wmax > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(wmax));
    }
}

template <bool MLP, typename TS>
__global__ void __launch_bounds__(BS) k_update(BlockView v, PhysArgs ph, int corrector, const double* Pb,
                                               const double* __restrict__ Pf, const double* __restrict__ F1,
                                               const double* __restrict__ F2, const double* __restrict__ F3,
                                               const double* __restrict__ Bn, double* Un, double* Po,
                                               uint8_t* __restrict__ status, const double* __restrict__ dscal,
                                               double fac, unsigned long long* dmax, unsigned long long* dcnt) {
    b_update<MLP, TS>(v, ph, corrector, Pb, Pf, F1, F2, F3, Bn, Un, Po, status, dscal, fac, dmax, dcnt,
                      (long)blockIdx.x * blockDim.x + threadIdx.x);
}


__device__ __forceinline__ void b_dt_reduce(const BlockView& v, PhysArgs ph, const double* __restrict__ P, unsigned long long* dmax, long t) {
    const long n = (long)v.n1 * v.n2 * v.n3;
    double inv = 0.0;
    if (t < n) {
        const int i = (int)(t % v.n1), j = (int)((t / v.n1) % v.n2), k = (int)(t / ((long)v.n1 * v.n2));
        const long c = cidx(v, i, j, k);
        Metric<double> m;
        load_metric(v.gc, v.n2d, gidx(v, i, j), m);
        double pr[NPRIM];
#pragma unroll
        for (int q = 0; q < NPRIM; q++) pr[q] = P[q * v.nc + c];
        const int w = smr_width(v, ph, j);
        if (w > 1) {  // an internal-SMR group: its width in x3
            BlockView vw = v;
            vw.idx3 = v.idx3 / w;
            inv = inv_dt_cell(vw, pr, m, ph.gam);
        } else {
            inv = inv_dt_cell(v, pr, m, ph.gam);
        }
    }
    const double wmax = warp_max(inv);
    if ((threadIdx.x & 31u) == 0 && wmax > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(wmax));
}

__global__ void k_dt_reduce(BlockView v, PhysArgs ph, const double* __restrict__ P, unsigned long long* dmax) {
    b_dt_reduce(v, ph, P, dmax, (long)blockIdx.x * blockDim.x + threadIdx.x);
}


// dt of this step: the caller's, or C0 / max rate of the current state;
// resets the accumulators of the new step.
__global__ void k_dt_select(double cour, double user_dt, double* dscal, unsigned long long* dmax,
                            unsigned long long* dcnt) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double mx = __longlong_as_double((long long)dmax[0]);
    dscal[0] = (user_dt > 0.0) ? user_dt : cour / mx;
    dmax[0] = 0ull;
    dcnt[0] = dcnt[1] = dcnt[2] = dcnt[3] = dcnt[4] = 0ull;
}

// ---------------------------------------------------------------- batched (multi-block) wrappers
// blockIdx.y selects the block list[blockIdx.y] of the table; blockIdx.x and
// threadIdx.x index the work inside it exactly as in the single-block kernels.
__device__ __forceinline__ long tidx() { return (long)blockIdx.x * blockDim.x + threadIdx.x; }

// kappa goes to field 0 of the EMF array (free until the EMFs), the flattening
// coefficients of dir to field 0 of the dir-flux array
template <int DIR, typename T>
__global__ void kb_recon(const DevBlock* tab, const int* list, PhysArgs ph, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    const double* Fl = (DIR == 1) ? D.F1 : ((DIR == 2) ? D.F2 : D.F3);
    if constexpr (std::is_same<T, double>::value)
        b_recon<DIR, T>(D.v, ph, sigma ? D.Ph : D.P, D.E, Fl, D.QL, D.QR, tidx());
    else  // the FP32 copy holds the stage's state
        b_recon<DIR, T>(D.v, ph, D.P32, reinterpret_cast<const float*>(D.E), reinterpret_cast<const float*>(Fl),
                        reinterpret_cast<float*>(D.QL), reinterpret_cast<float*>(D.QR), tidx());
}

template <int DIR, typename T>
__global__ void kb_flatten(const DevBlock* tab, const int* list, PhysArgs ph, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    double* Fl = (DIR == 1) ? D.F1 : ((DIR == 2) ? D.F2 : D.F3);
    if constexpr (std::is_same<T, double>::value)
        b_flatten<DIR, T>(D.v, ph, sigma ? D.Ph : D.P, Fl, tidx());
    else
        b_flatten<DIR, T>(D.v, ph, D.P32, reinterpret_cast<float*>(Fl), tidx());
}

template <typename T>
__global__ void kb_kappa(const DevBlock* tab, const int* list, PhysArgs ph, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    if constexpr (std::is_same<T, double>::value)
        b_kappa<T>(D.v, ph.gam, sigma ? D.Ph : D.P, D.E, tidx(), sigma ? nullptr : D.Un + (long)C_ENT * D.v.nc);
    else
        b_kappa<T>(D.v, (float)ph.gam, D.P32, reinterpret_cast<float*>(D.E), tidx(),
                   sigma ? nullptr : D.Un + (long)C_ENT * D.v.nc);
}

__global__ void kb_to_f32(const DevBlock* tab, const int* list, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    b_to_f32(D.v, sigma ? D.Ph : D.P, D.P32, tidx());
}

template <int DIR, typename T>
__global__ void __launch_bounds__(256, 2) kb_flux(const DevBlock* tab, const int* list, PhysArgs ph, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    double* F = (DIR == 1) ? D.F1 : ((DIR == 2) ? D.F2 : D.F3);
    b_flux<DIR, T>(D.v, ph, reinterpret_cast<const T*>(D.QL), reinterpret_cast<const T*>(D.QR), sigma ? D.Bh : D.B, F,
                   tidx());
}

template <typename T, bool F32 = false>
__global__ void kb_emf(const DevBlock* tab, const int* list, int upwind) {
    const DevBlock& D = tab[list[blockIdx.y]];
    b_emf<T, F32>(D.v, D.F1, D.F2, D.F3, D.E, upwind ? D.QL : nullptr, tidx());
}

// cell EMFs of the stage state into the edge-value scratch (free once the fluxes exist)
__global__ void kb_cell_emf(const DevBlock* tab, const int* list, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    b_cell_emf(D.v, sigma ? D.Ph : D.P, D.QL, tidx());
}

__global__ void kb_ct(const DevBlock* tab, const int* list, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    if (sigma == 0)
        b_ct(D.v, D.E, D.B, D.Bh, D.dscal, 0.5, tidx());
    else if (sigma == 1)
        b_ct(D.v, D.E, D.B, D.B, D.dscal, 1.0, tidx());
    else
        b_ct(D.v, D.E, D.B, D.B, D.dscal + 1, 1.0, tidx());
}

template <bool MLP, typename TS>
__global__ void __launch_bounds__(BS, 3) kb_update(const DevBlock* tab, const int* list, PhysArgs ph, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    const bool c = sigma != 0;  // predictor (0) or corrector (2, no CFL rate here) of the block's step
    PhysArgs pb = ph;
    pb.smr_u = D.QR;  // internal SMR: the grouped cells' conserved states (free once the fluxes exist)
    b_update<MLP, TS>(D.v, pb, c ? 2 : 0, D.P, c ? D.Ph : D.P, D.F1, D.F2, D.F3, c ? D.B : D.Bh, D.Un, c ? D.P : D.Ph,
                      D.status, D.dscal, c ? 1.0 : 0.5, D.dmax, D.dcnt, tidx());
}

__global__ void kb_dt_reduce(const DevBlock* tab, const int* list, PhysArgs ph) {
    const DevBlock& D = tab[list[blockIdx.y]];
    b_dt_reduce(D.v, ph, D.P, D.dmax, tidx());
}

// state at the start of a step (the source of finer neighbours' time interpolation), status reset
__global__ void kb_save_old(const DevBlock* tab, const int* list) {
    const DevBlock& D = tab[list[blockIdx.y]];
    const long t = tidx();
    const long n = (long)D.v.n1p * D.v.n2p * D.v.n3p;
    if (t >= n) return;
#pragma unroll
    for (int q = 0; q < NPRIM; q++) D.Pold[q * D.v.nc + t] = D.P[q * D.v.nc + t];
#pragma unroll
    for (int q = 0; q < 3; q++) D.Bold[q * D.v.nc + t] = D.B[q * D.v.nc + t];
    D.status[t] = 0;
}

// refluxed cells: U(P) with the field before the correction, plus the flux corrections
__global__ void k_reflux_u0(const DevBlock* tab, int n, const int* cblk, const long* cix, const int* nrec,
                            const int* recs, const double* rec_dU, int nrec_tot, double* Ucorr, PhysArgs ph) {
    const long i = tidx();
    if (i >= n) return;
    const DevBlock& D = tab[cblk[i]];
    const BlockView& v = D.v;
    const long c = cix[i];
    const long ip = c % v.n1p, jp = (c / v.n1p) % v.n2p;
    Metric<double> m;
    load_metric(v.gc, v.n2d, jp * v.n1p + ip, m);
    double pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pr[q] = D.P[q * v.nc + c];
    Fluid<double> s;
    fluid_state(pr, m, s);
    double row[NFLUX];
    flux_row(pr, s, 0, 1, ph.gam, entropy_kappa(pr, ph.gam), row);
    for (int q = 0; q < NCONS; q++) {
        double du = 0.0;
        for (int r = 0; r < nrec[i]; r++) du += rec_dU[(long)q * nrec_tot + recs[3 * i + r]];
        Ucorr[(long)q * n + i] = row[q] * m.gdet + du;
    }
}

// inversion of the refluxed cells with the corrected field; floors. Ucorr: stride `stride` per field
__global__ void k_reflux_cells(const DevBlock* tab, int n, const int* cblk, const long* cix, const double* Ucorr,
                               long stride, PhysArgs ph) {
    const long i = tidx();
    if (i >= n) return;
    const DevBlock& D = tab[cblk[i]];
    const BlockView& v = D.v;
    const long c = cix[i];
    const int ii = (int)(c % v.n1p) - NG, jj = (int)((c / v.n1p) % v.n2p) - NG, kk = (int)(c / ((long)v.n1p * v.n2p)) - NG;
    const long g = gidx(v, ii, jj);
    Metric<double> m;
    load_metric(v.gc, v.n2d, g, m);
    double U[NCONS];
    for (int q = 0; q < NCONS; q++) U[q] = Ucorr[(long)q * stride + i];
    double Bc[3];
    centre_field(v, D.B, ii, jj, kk, m.igdet, Bc);
    double pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pr[q] = D.P[q * v.nc + c];
    pr[B1] = Bc[0];
    pr[B2] = Bc[1];
    pr[B3] = Bc[2];
    int its;
    const int st = invert(U, Bc, m, ph.gam, pr, &its, false, nullptr, ph.inversion);
    if (st == INV_FAIL)
#pragma unroll
        for (int q = 0; q < 5; q++) pr[q] = D.P[q * v.nc + c];
    int fl = 0;
    if (ph.floors) {
        Fluid<double> s;
        fluid_state(pr, m, s);
        fl = cell_floors(v, g, m, ph, pr, s);
    }
#pragma unroll
    for (int q = 0; q < NPRIM; q++) D.P[q * v.nc + c] = pr[q];
    atomicAdd(&D.dcnt[st == INV_OK ? 0 : (st == INV_ENTROPY ? 1 : 2)], 1ull);
    if (fl) atomicAdd(&D.dcnt[3], 1ull);
}

// refluxed internal-SMR groups (its w cells consecutive in the list from position first[g]): the mean
// of the cells' corrected states inverted once with the mean corrected centre field, from the mean
// primitives; every cell takes the result and keeps its own centre field; floors
__global__ void k_reflux_groups(const DevBlock* tab, int ngrp, const int* first, const int* gw, const int* cblk,
                                const long* cix, const double* Ucorr, long stride, PhysArgs ph) {
    const long t = tidx();
    if (t >= ngrp) return;
    const int f = first[t], w = gw[t];
    const DevBlock& D = tab[cblk[f]];
    const BlockView& v = D.v;
    const long c0 = cix[f];
    const int ii = (int)(c0 % v.n1p) - NG, jj = (int)((c0 / v.n1p) % v.n2p) - NG;
    const int k0 = (int)(c0 / ((long)v.n1p * v.n2p)) - NG;
    const long g = gidx(v, ii, jj);
    Metric<double> m;
    load_metric(v.gc, v.n2d, g, m);
    double U[NCONS], Bc[3] = {0.0, 0.0, 0.0}, pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NCONS; q++) U[q] = 0.0;
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pr[q] = 0.0;
    for (int a = 0; a < w; a++) {
        const long c = cix[f + a];
#pragma unroll
        for (int q = 0; q < NCONS; q++) U[q] += Ucorr[(long)q * stride + f + a];
        double b[3];
        centre_field(v, D.B, ii, jj, k0 + a, m.igdet, b);
        for (int e = 0; e < 3; e++) Bc[e] += b[e];
#pragma unroll
        for (int q = 0; q < 5; q++) pr[q] += D.P[q * v.nc + c];
    }
#pragma unroll
    for (int q = 0; q < NCONS; q++) U[q] /= w;
    for (int e = 0; e < 3; e++) Bc[e] /= w;
#pragma unroll
    for (int q = 0; q < 5; q++) pr[q] /= w;
    double p0[5];
#pragma unroll
    for (int q = 0; q < 5; q++) p0[q] = pr[q];
    pr[B1] = Bc[0];
    pr[B2] = Bc[1];
    pr[B3] = Bc[2];
    int its;
    const int st = invert(U, Bc, m, ph.gam, pr, &its, false, nullptr, ph.inversion);
    if (st == INV_FAIL)
#pragma unroll
        for (int q = 0; q < 5; q++) pr[q] = p0[q];
    int fl = 0;
    if (ph.floors) {
        Fluid<double> s;
        fluid_state(pr, m, s);
        fl = cell_floors(v, g, m, ph, pr, s);
    }
    for (int a = 0; a < w; a++) {
        const long c = cix[f + a];
        double b[3];
        centre_field(v, D.B, ii, jj, k0 + a, m.igdet, b);
#pragma unroll
        for (int q = 0; q < 5; q++) D.P[q * v.nc + c] = pr[q];
        for (int e = 0; e < 3; e++) D.P[(B1 + e) * v.nc + c] = b[e];
    }
    atomicAdd(&D.dcnt[st == INV_OK ? 0 : (st == INV_ENTROPY ? 1 : 2)], (unsigned long long)w);
    if (fl) atomicAdd(&D.dcnt[3], (unsigned long long)w);
}

// ---------------------------------------------------------------- internal SMR
// Rows next to a polar face grouped into cells smr_width wide in x3 (Sec. 3.3.2:
// a group's fluxes and conserved state are averaged). The field: before CT, along
// each x2-line of edges with group width W (that of the adjacent row closer to the
// pole) the E3 of a group take their mean and the inner E1 are linear between the
// group's outer ones; inside each grouped row the inner E2 are linear between the
// group's outer ones. The changes of a group's x1- and x2-faces are then uniform
// and those of its inner x3-faces linear (a wide cell's), and CT keeps div B. The
// cells: after the cell update (which leaves the group's conserved states in the
// scratch U) the group's mean state is inverted once with the mean centre field,
// from the mean primitives, and every cell takes the result (its own centre field
// kept); the CFL rate uses the group's width.
__device__ __forceinline__ int smr_line_width(const BlockView& v, const PhysArgs& ph, int je) {
    int w = 1;
    if (je >= 1) w = max(w, smr_width(v, ph, je - 1));
    if (je < v.n2) w = max(w, smr_width(v, ph, je));
    return w;
}

// sum of w = 2^n values as a balanced binary tree (w equal values sum to exactly w times the
// value): element m closes the subtrees its trailing one bits end
__device__ __forceinline__ double pair_sum_strided(const double* __restrict__ a, long stride, int w) {
    double st[12];
    for (int m = 0; m < w; m++) {
        double t = a[m * stride];
        int l = 0;
        while ((m >> l) & 1) {
            t = st[l] + t;
            l++;
        }
        st[l] = t;
    }
    return st[__ffs(w) - 1];
}

// Threads: i in [0, n1], q over the nr + 1 edge lines and nr rows next to each polar face
// (lines je = 0..nr and n2 - nr..n2, a line counted once when n2 = 2 nr), gi over the groups.
__device__ __forceinline__ void b_smr_emf(const BlockView& v, const PhysArgs& ph, double* __restrict__ E, long t) {
    const int nr = smr_rows(v, ph);
    const int ng = v.n3 / 2;
    const int nq = 2 * (nr + 1);
    if (nr == 0 || t >= (long)(v.n1 + 1) * nq * ng) return;
    const int i = (int)(t % (v.n1 + 1));
    const int q = (int)((t / (v.n1 + 1)) % nq);
    const int gi = (int)(t / ((long)(v.n1 + 1) * nq));
    const long sk = (long)v.n1p * v.n2p;
    double* E1 = E;
    double* E2 = E + v.nc;
    double* E3 = E + 2 * v.nc;
    // the edge line: lower side je = q, upper side je = n2 - 2 nr - 1 + q
    const bool upper = q > nr;
    const int je = upper ? v.n2 - 2 * nr - 1 + q : q;
    const int W = (upper && je <= nr) ? 1 : smr_line_width(v, ph, je);
    if (W > 1 && gi < v.n3 / W) {
        const int k0 = gi * W;
        const long c0 = cidx(v, i, je, k0);
        const double s3 = pair_sum_strided(E3 + c0, sk, W);
        for (int m = 0; m < W; m++) E3[c0 + m * sk] = s3 / W;
        if (i < v.n1) {
            const double e0 = E1[c0], ew = E1[c0 + W * sk];
            for (int m = 1; m < W; m++) E1[c0 + m * sk] = e0 + (ew - e0) * m / W;
        }
    }
    // the row: lower side j = q (q < nr), upper side j = n2 - 2 nr - 1 + q (nr < q <= 2 nr)
    const int j = (q < nr) ? q : ((q > nr && q <= 2 * nr) ? v.n2 - 2 * nr - 1 + q : -1);
    if (j < 0) return;
    const int w = smr_width(v, ph, j);
    if (w > 1 && gi < v.n3 / w) {
        const int k0 = gi * w;
        const long c0 = cidx(v, i, j, k0);
        const double e0 = E2[c0], ew = E2[c0 + w * sk];
        for (int m = 1; m < w; m++) E2[c0 + m * sk] = e0 + (ew - e0) * m / w;
    }
}

// the grouped row of cell-thread row r: rows [0, nr) and [n2 - nr, n2), nr = smr_rows
__device__ __forceinline__ int smr_row(const BlockView& v, const PhysArgs& ph, int r) {
    const int nr = smr_rows(v, ph);
    return (r < nr) ? r : v.n2 - 2 * nr + r;
}

__device__ __forceinline__ void b_smr_cells(const BlockView& v, const PhysArgs& ph, int corrector,
                                            const double* __restrict__ Pf, const double* __restrict__ Bn,
                                            const double* __restrict__ Us, double* Po, uint8_t* __restrict__ status,
                                            unsigned long long* dmax, unsigned long long* dcnt, long t) {
    const int nr = smr_rows(v, ph);
    const int ng = v.n3 / 2;
    if (nr == 0 || t >= (long)v.n1 * 2 * nr * ng) return;
    const int i = (int)(t % v.n1);
    const int r = (int)((t / v.n1) % (2 * nr));
    const int gi = (int)(t / ((long)v.n1 * 2 * nr));
    const int j = smr_row(v, ph, r);
    const int w = smr_width(v, ph, j);
    if (w == 1 || gi >= v.n3 / w) return;
    const int k0 = gi * w;
    const long g = gidx(v, i, j);
    Metric<double> m;
    load_metric(v.gc, v.n2d, g, m);
    double U[NCONS], Bc[3] = {0.0, 0.0, 0.0}, pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NCONS; q++) U[q] = 0.0;
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pr[q] = 0.0;
    for (int a = 0; a < w; a++) {
        const long c = cidx(v, i, j, k0 + a);
#pragma unroll
        for (int q = 0; q < NCONS; q++) U[q] += Us[q * v.nc + c];
        double b[3];
        centre_field(v, Bn, i, j, k0 + a, m.igdet, b);
        for (int e = 0; e < 3; e++) Bc[e] += b[e];
#pragma unroll
        for (int q = 0; q < 5; q++) pr[q] += Pf[q * v.nc + c];
    }
#pragma unroll
    for (int q = 0; q < NCONS; q++) U[q] /= w;
    for (int e = 0; e < 3; e++) Bc[e] /= w;
#pragma unroll
    for (int q = 0; q < 5; q++) pr[q] /= w;
    double pf[5];
#pragma unroll
    for (int q = 0; q < 5; q++) pf[q] = pr[q];
    pr[B1] = Bc[0];
    pr[B2] = Bc[1];
    pr[B3] = Bc[2];
    int its = 0;
    const int st = invert(U, Bc, m, ph.gam, pr, &its, false, nullptr, ph.inversion);
    if (st == INV_FAIL)
#pragma unroll
        for (int q = 0; q < 5; q++) pr[q] = pf[q];
    Fluid<double> s;
    fluid_state(pr, m, s);
    const int fl = ph.floors ? cell_floors(v, g, m, ph, pr, s) : 0;
    const uint8_t sb = ((st == INV_ENTROPY) ? ST_ENTROPY : ((st == INV_FAIL) ? ST_FAIL : 0)) | (fl ? ST_FLOOR : 0);
    for (int a = 0; a < w; a++) {
        const long c = cidx(v, i, j, k0 + a);
        double b[3];
        centre_field(v, Bn, i, j, k0 + a, m.igdet, b);
#pragma unroll
        for (int q = 0; q < 5; q++) Po[q * v.nc + c] = pr[q];
        for (int e = 0; e < 3; e++) Po[(B1 + e) * v.nc + c] = b[e];
        status[c] |= sb;
        if (ph.stage32) {
            float p8[NPRIM];
#pragma unroll
            for (int q = 0; q < 5; q++) p8[q] = narrow(pr[q]);
            for (int e = 0; e < 3; e++) p8[B1 + e] = narrow(b[e]);
            store_stage32(v, ph, corrector, c, p8);
        }
    }
    atomicAdd(&dcnt[st == INV_OK ? 0 : (st == INV_ENTROPY ? 1 : 2)], (unsigned long long)w);
    if (fl) atomicAdd(&dcnt[3], (unsigned long long)w);
    atomicAdd(&dcnt[4], (unsigned long long)(w * its));
    if (corrector == 1) {  // the CFL rate over the group's width, of each cell with its own centre field
        BlockView vw = v;
        vw.idx3 = v.idx3 / w;
        double inv = 0.0;
        for (int a = 0; a < w; a++) {
            double pa[NPRIM];
#pragma unroll
            for (int q = 0; q < NPRIM; q++) pa[q] = Po[q * v.nc + cidx(v, i, j, k0 + a)];
            Fluid<double> sa;
            fluid_state(pa, m, sa);
            inv = fmax(inv, inv_dt_fluid(vw, pa, sa, m, ph.gam));
        }
        if (inv > 0.0) atomicMax(dmax, (unsigned long long)__double_as_longlong(inv));
    }
}

__global__ void k_smr_emf(BlockView v, PhysArgs ph, double* __restrict__ E) {
    b_smr_emf(v, ph, E, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_smr_cells(BlockView v, PhysArgs ph, int corrector, const double* __restrict__ Pf,
                            const double* __restrict__ Bn, double* Po, uint8_t* __restrict__ status,
                            unsigned long long* dmax, unsigned long long* dcnt) {
    b_smr_cells(v, ph, corrector, Pf, Bn, ph.smr_u, Po, status, dmax, dcnt, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// batched: the EMFs of the stage (after the edge synchronisation) and the cells of the block's
// predictor (sigma 0) or corrector (1, no CFL rate: the period sets dt); scratch: the block's right
// edge values, free once the fluxes are formed
__global__ void kb_smr_emf(const DevBlock* tab, const int* list, PhysArgs ph) {
    const DevBlock& D = tab[list[blockIdx.y]];
    b_smr_emf(D.v, ph, D.E, tidx());
}

__global__ void kb_smr_cells(const DevBlock* tab, const int* list, PhysArgs ph, int sigma) {
    const DevBlock& D = tab[list[blockIdx.y]];
    const bool c = sigma != 0;
    b_smr_cells(D.v, ph, c ? 2 : 0, c ? D.Ph : D.P, c ? D.B : D.Bh, D.QR, c ? D.P : D.Ph, D.status, D.dmax, D.dcnt,
                tidx());
}

// maximum of field q over the interior cells, as ordered bits (ordered_bits)
__global__ void k_block_max(BlockView v, const double* __restrict__ P, int q, unsigned long long* out) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long n = (long)v.n1 * v.n2 * v.n3;
    unsigned long long m = 0ull;
    if (t < n) {
        const int i = (int)(t % v.n1), j = (int)((t / v.n1) % v.n2), k = (int)(t / ((long)v.n1 * v.n2));
        m = ordered_bits(P[q * v.nc + cidx(v, i, j, k)]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_down_sync(0xffffffffu, m, o);
        m = x > m ? x : m;
    }
    if ((threadIdx.x & 31u) == 0 && m) atomicMax(out, m);
}

}  // namespace

cudaError_t launch_smr_emf(const BlockView& v, const PhysArgs& ph, double* E, cudaStream_t s) {
    const long n = smr_emf_threads(v, ph);
    if (n > 0) k_smr_emf<<<nblk(n), BS, 0, s>>>(v, ph, E);
    return cudaGetLastError();
}

cudaError_t launch_smr_cells(const BlockView& v, const PhysArgs& ph, int corrector, const double* Pf, const double* Bn,
                             double* Po, uint8_t* status, unsigned long long* dmax, unsigned long long* dcnt,
                             cudaStream_t s) {
    const long n = smr_cell_threads(v, ph);
    if (n > 0) k_smr_cells<<<nblk(n), BS, 0, s>>>(v, ph, corrector, Pf, Bn, Po, status, dmax, dcnt);
    return cudaGetLastError();
}

long smr_emf_threads(const BlockView& v, const PhysArgs& ph) {
    const int nr = smr_rows(v, ph);
    return nr ? (long)(v.n1 + 1) * 2 * (nr + 1) * (v.n3 / 2) : 0;
}

long smr_cell_threads(const BlockView& v, const PhysArgs& ph) { return (long)v.n1 * 2 * smr_rows(v, ph) * (v.n3 / 2); }

cudaError_t launch_smr_emf_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                 cudaStream_t s) {
    if (nlist == 0 || maxwork == 0) return cudaSuccess;
    kb_smr_emf<<<dim3(nblk(maxwork), nlist), BS, 0, s>>>(tab, list, ph);
    return cudaGetLastError();
}

cudaError_t launch_smr_cells_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                   int sigma, cudaStream_t s) {
    if (nlist == 0 || maxwork == 0) return cudaSuccess;
    kb_smr_cells<<<dim3(nblk(maxwork), nlist), BS, 0, s>>>(tab, list, ph, sigma);
    return cudaGetLastError();
}

cudaError_t launch_block_max(const BlockView& v, const double* P, int q, unsigned long long* out, cudaStream_t s) {
    k_block_max<<<nblk((long)v.n1 * v.n2 * v.n3), BS, 0, s>>>(v, P, q, out);
    return cudaGetLastError();
}

cudaError_t launch_centre_b(const BlockView& v, double* P, const double* B, cudaStream_t s) {
    k_centre_b<<<nblk((long)v.n1 * v.n2 * v.n3), BS, 0, s>>>(v, P, B);
    return cudaGetLastError();
}

cudaError_t launch_bc(const BlockView& v, double* P, double* B, cudaStream_t s, float* P32, float* K32) {
    const int nn[4] = {0, v.n1, v.n2, v.n3};
    for (int e = 3; e >= 1; e--) {
        const int ta = (e == 1) ? 2 : 1, tb = (e == 3) ? 2 : 3;
        const long total = 2L * NG * (nn[ta] + 2 * NG) * (nn[tb] + 2 * NG);
        k_bc_pass<<<nblk(total), BS, 0, s>>>(v, P, B, e, P32, K32);
        if (e == 2) k_bc_axis<<<nblk(2L * (v.n1 + 2 * NG) * (v.n3 + 2 * NG)), BS, 0, s>>>(v, B);
    }
    return cudaGetLastError();
}

cudaError_t launch_flatten(const BlockView& v, const PhysArgs& ph, int dir, const double* P, const float* P32,
                           double* Fl, cudaStream_t s) {
    const long n = (long)(v.n1 + 2) * (v.n2 + 2) * (v.n3 + 2);
    if (ph.mixed) {
        float* F = reinterpret_cast<float*>(Fl);
        if (dir == 1) k_flatten<1, float><<<nblk(n), BS, 0, s>>>(v, ph, P32, F);
        if (dir == 2) k_flatten<2, float><<<nblk(n), BS, 0, s>>>(v, ph, P32, F);
        if (dir == 3) k_flatten<3, float><<<nblk(n), BS, 0, s>>>(v, ph, P32, F);
    } else {
        if (dir == 1) k_flatten<1, double><<<nblk(n), BS, 0, s>>>(v, ph, P, Fl);
        if (dir == 2) k_flatten<2, double><<<nblk(n), BS, 0, s>>>(v, ph, P, Fl);
        if (dir == 3) k_flatten<3, double><<<nblk(n), BS, 0, s>>>(v, ph, P, Fl);
    }
    return cudaGetLastError();
}

cudaError_t launch_kappa(const BlockView& v, const PhysArgs& ph, const double* P, const float* P32, double* K,
                         double* Un, cudaStream_t s) {
    const long n = (long)v.n1p * v.n2p * v.n3p;
    if (ph.mixed)
        k_kappa<float><<<nblk(n), BS, 0, s>>>(v, (float)ph.gam, P32, reinterpret_cast<float*>(K),
                                              Un ? Un + (long)C_ENT * v.nc : nullptr);
    else
        k_kappa<double><<<nblk(n), BS, 0, s>>>(v, ph.gam, P, K, Un ? Un + (long)C_ENT * v.nc : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_recon(const BlockView& v, const PhysArgs& ph, int dir, const double* P, const float* P32,
                         const double* K, const double* Fl, double* QL, double* QR, cudaStream_t s) {
    const long n = recon_threads(v, dir, ph.mixed, ph.recon_seg, ph.recon_x1_sweep);
    const unsigned nb = nblk(n, ph.bs_recon);
    const int bs = ph.bs_recon;
    if (ph.mixed) {
        const float* K32 = reinterpret_cast<const float*>(K);
        const float* F32 = reinterpret_cast<const float*>(Fl);
        float* L = reinterpret_cast<float*>(QL);
        float* R = reinterpret_cast<float*>(QR);
        if (dir == 1) k_recon<1, float><<<nb, bs, 0, s>>>(v, ph, P32, K32, F32, L, R);
        if (dir == 2) k_recon<2, float><<<nb, bs, 0, s>>>(v, ph, P32, K32, F32, L, R);
        if (dir == 3) k_recon<3, float><<<nb, bs, 0, s>>>(v, ph, P32, K32, F32, L, R);
    } else {
        if (dir == 1) k_recon<1, double><<<nb, bs, 0, s>>>(v, ph, P, K, Fl, QL, QR);
        if (dir == 2) k_recon<2, double><<<nb, bs, 0, s>>>(v, ph, P, K, Fl, QL, QR);
        if (dir == 3) k_recon<3, double><<<nb, bs, 0, s>>>(v, ph, P, K, Fl, QL, QR);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const BlockView& v, const double* P, float* P32, cudaStream_t s) {
    k_to_f32<<<nblk((long)v.n1p * v.n2p * v.n3p), BS, 0, s>>>(v, P, P32);
    return cudaGetLastError();
}

cudaError_t launch_flux(const BlockView& v, const PhysArgs& ph, int dir, const double* QL, const double* QR,
                        const double* Bf, double* F, cudaStream_t s) {
    const long n1 = v.n1 + (dir == 1 ? 1 : 2), n2 = v.n2 + (dir == 2 ? 1 : 2), n3 = v.n3 + (dir == 3 ? 1 : 2);
    const long n = n1 * n2 * n3;
    const unsigned nb = nblk(n, ph.bs_flux);
    const int bs = ph.bs_flux;
    if (ph.mixed) {
        const float* L = reinterpret_cast<const float*>(QL);
        const float* R = reinterpret_cast<const float*>(QR);
        if (dir == 1) k_flux<1, float><<<nb, bs, 0, s>>>(v, ph, L, R, Bf, F);
        if (dir == 2) k_flux<2, float><<<nb, bs, 0, s>>>(v, ph, L, R, Bf, F);
        if (dir == 3) k_flux<3, float><<<nb, bs, 0, s>>>(v, ph, L, R, Bf, F);
    } else {
        if (dir == 1) k_flux<1, double><<<nb, bs, 0, s>>>(v, ph, QL, QR, Bf, F);
        if (dir == 2) k_flux<2, double><<<nb, bs, 0, s>>>(v, ph, QL, QR, Bf, F);
        if (dir == 3) k_flux<3, double><<<nb, bs, 0, s>>>(v, ph, QL, QR, Bf, F);
    }
    return cudaGetLastError();
}

cudaError_t launch_emf(const BlockView& v, double* const F[3], double* E, int mixed, const double* P, double* Ec,
                       cudaStream_t s) {
    const long n = (long)(v.n1 + 1) * (v.n2 + 1) * (v.n3 + 1);
    if (Ec) {  // upwinded EMFs: the cell EMFs of the stage state P first
        k_cell_emf<<<nblk((long)(v.n1 + 2) * (v.n2 + 2) * (v.n3 + 2)), BS, 0, s>>>(v, P, Ec);
    }
    if (mixed == 2)  // FP32 EMFs of fluxes stored in FP32
        k_emf<float, true><<<nblk(n), BS, 0, s>>>(v, F[0], F[1], F[2], E, Ec);
    else if (mixed)
        k_emf<float><<<nblk(n), BS, 0, s>>>(v, F[0], F[1], F[2], E, Ec);
    else
        k_emf<double><<<nblk(n), BS, 0, s>>>(v, F[0], F[1], F[2], E, Ec);
    return cudaGetLastError();
}

cudaError_t launch_ct(const BlockView& v, const double* E, const double* Bbase, double* Bout, const double* dscal,
                      double dt_factor, cudaStream_t s) {
    const long n = (long)(v.n1 + 1) * (v.n2 + 1) * (v.n3 + 1);
    k_ct<<<nblk(n), BS, 0, s>>>(v, E, Bbase, Bout, dscal, dt_factor);
    return cudaGetLastError();
}

cudaError_t launch_update(const BlockView& v, const PhysArgs& ph, int corrector, const double* Pbase,
                          const double* Pflux, double* const F[3], const double* Bnew, double* Un, double* Pout,
                          uint8_t* status, const double* dscal, double dt_factor, unsigned long long* dmax,
                          unsigned long long* dcnt, cudaStream_t s) {
    const long n = (long)v.n1 * v.n2 * v.n3;
    const int bs = ph.mlp_img ? MLP_ROWS : ph.bs_update;  // the network needs one row per thread of 128
    const unsigned nb = nblk(n, bs);
    const int sm = ph.mlp_img ? MLP_SMEM_BYTES : 0;
#define HAMR_UPD_ARGS v, ph, corrector, Pbase, Pflux, F[0], F[1], F[2], Bnew, Un, Pout, status, dscal, dt_factor, dmax, dcnt
    if (ph.mlp_img && ph.mixed)
        k_update<true, float><<<nb, bs, sm, s>>>(HAMR_UPD_ARGS);
    else if (ph.mlp_img)
        k_update<true, double><<<nb, bs, sm, s>>>(HAMR_UPD_ARGS);
    else if (ph.mixed)
        k_update<false, float><<<nb, bs, 0, s>>>(HAMR_UPD_ARGS);
    else
        k_update<false, double><<<nb, bs, 0, s>>>(HAMR_UPD_ARGS);
#undef HAMR_UPD_ARGS
    return cudaGetLastError();
}

cudaError_t launch_dt_reduce(const BlockView& v, const PhysArgs& ph, const double* P, unsigned long long* dmax,
                             cudaStream_t s) {
    k_dt_reduce<<<nblk((long)v.n1 * v.n2 * v.n3), BS, 0, s>>>(v, ph, P, dmax);
    return cudaGetLastError();
}

cudaError_t launch_dt_select(const PhysArgs& ph, double user_dt, double* dscal, unsigned long long* dmax,
                             unsigned long long* dcnt, uint8_t* status, long nc, cudaStream_t s) {
    k_dt_select<<<1, 32, 0, s>>>(ph.cour, user_dt, dscal, dmax, dcnt);
    cudaMemsetAsync(status, 0, (size_t)nc, s);
    return cudaGetLastError();
}

namespace {
inline dim3 bgrid(long maxwork, int nlist, int bs = BS) { return dim3(nblk(maxwork, bs), (unsigned)nlist); }
}  // namespace

cudaError_t launch_recon_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                               int dir, int sigma, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    const int bs = ph.bs_recon;
    const dim3 g = bgrid(maxwork, nlist, bs);
    if (ph.mixed) {
        if (dir == 1) kb_recon<1, float><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 2) kb_recon<2, float><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 3) kb_recon<3, float><<<g, bs, 0, s>>>(tab, list, ph, sigma);
    } else {
        if (dir == 1) kb_recon<1, double><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 2) kb_recon<2, double><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 3) kb_recon<3, double><<<g, bs, 0, s>>>(tab, list, ph, sigma);
    }
    return cudaGetLastError();
}

cudaError_t launch_flatten_batch(const DevBlock* tab, const int* list, int nlist, long maxcells, const PhysArgs& ph,
                                 int dir, int sigma, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    const dim3 g = bgrid(maxcells, nlist);
    if (ph.mixed) {
        if (dir == 1) kb_flatten<1, float><<<g, BS, 0, s>>>(tab, list, ph, sigma);
        if (dir == 2) kb_flatten<2, float><<<g, BS, 0, s>>>(tab, list, ph, sigma);
        if (dir == 3) kb_flatten<3, float><<<g, BS, 0, s>>>(tab, list, ph, sigma);
    } else {
        if (dir == 1) kb_flatten<1, double><<<g, BS, 0, s>>>(tab, list, ph, sigma);
        if (dir == 2) kb_flatten<2, double><<<g, BS, 0, s>>>(tab, list, ph, sigma);
        if (dir == 3) kb_flatten<3, double><<<g, BS, 0, s>>>(tab, list, ph, sigma);
    }
    return cudaGetLastError();
}

cudaError_t launch_kappa_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                               int sigma, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    if (ph.mixed)
        kb_kappa<float><<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, ph, sigma);
    else
        kb_kappa<double><<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, ph, sigma);
    return cudaGetLastError();
}

cudaError_t launch_to_f32_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, int sigma,
                                cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    kb_to_f32<<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, sigma);
    return cudaGetLastError();
}

cudaError_t launch_flux_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                              int dir, int sigma, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    const int bs = ph.bs_flux;
    const dim3 g = bgrid(maxwork, nlist, bs);
    if (ph.mixed) {
        if (dir == 1) kb_flux<1, float><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 2) kb_flux<2, float><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 3) kb_flux<3, float><<<g, bs, 0, s>>>(tab, list, ph, sigma);
    } else {
        if (dir == 1) kb_flux<1, double><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 2) kb_flux<2, double><<<g, bs, 0, s>>>(tab, list, ph, sigma);
        if (dir == 3) kb_flux<3, double><<<g, bs, 0, s>>>(tab, list, ph, sigma);
    }
    return cudaGetLastError();
}

cudaError_t launch_emf_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, int mixed, int upwind,
                             long maxcells, int sigma, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    if (upwind) kb_cell_emf<<<bgrid(maxcells, nlist), BS, 0, s>>>(tab, list, sigma);
    if (mixed == 2 && !upwind)  // FP32 EMFs of the FP32 copies of the flux field slots
        kb_emf<float, true><<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, upwind);
    else if (mixed)
        kb_emf<float><<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, upwind);
    else
        kb_emf<double><<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, upwind);
    return cudaGetLastError();
}

cudaError_t launch_ct_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, int sigma, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    kb_ct<<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, sigma);
    return cudaGetLastError();
}

cudaError_t launch_update_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                int sigma, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    const int bs = ph.mlp_img ? MLP_ROWS : ph.bs_update;
    const dim3 gr = bgrid(maxwork, nlist, bs);
    const int sm = ph.mlp_img ? MLP_SMEM_BYTES : 0;
    if (ph.mlp_img && ph.mixed)
        kb_update<true, float><<<gr, bs, sm, s>>>(tab, list, ph, sigma);
    else if (ph.mlp_img)
        kb_update<true, double><<<gr, bs, sm, s>>>(tab, list, ph, sigma);
    else if (ph.mixed)
        kb_update<false, float><<<gr, bs, 0, s>>>(tab, list, ph, sigma);
    else
        kb_update<false, double><<<gr, bs, 0, s>>>(tab, list, ph, sigma);
    return cudaGetLastError();
}

cudaError_t launch_dt_reduce_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, const PhysArgs& ph,
                                   cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    kb_dt_reduce<<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list, ph);
    return cudaGetLastError();
}

cudaError_t launch_save_old_batch(const DevBlock* tab, const int* list, int nlist, long maxwork, cudaStream_t s) {
    if (nlist <= 0) return cudaSuccess;
    kb_save_old<<<bgrid(maxwork, nlist), BS, 0, s>>>(tab, list);
    return cudaGetLastError();
}

cudaError_t launch_reflux_u0(const DevBlock* tab, int n, const int* cblk, const long* cidx_, const int* nrec,
                             const int* recs, const double* rec_dU, int nrec_tot, double* Ucorr, const PhysArgs& ph,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_reflux_u0<<<nblk(n), BS, 0, s>>>(tab, n, cblk, cidx_, nrec, recs, rec_dU, nrec_tot, Ucorr, ph);
    return cudaGetLastError();
}

cudaError_t launch_reflux_cells(const DevBlock* tab, int n, const int* cblk, const long* cidx_, const double* Ucorr,
                                long stride, const PhysArgs& ph, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_reflux_cells<<<nblk(n), BS, 0, s>>>(tab, n, cblk, cidx_, Ucorr, stride, ph);
    return cudaGetLastError();
}

cudaError_t launch_reflux_groups(const DevBlock* tab, int ngrp, const int* first, const int* w, const int* cblk,
                                 const long* cidx_, const double* Ucorr, long stride, const PhysArgs& ph,
                                 cudaStream_t s) {
    if (ngrp <= 0) return cudaSuccess;
    k_reflux_groups<<<nblk(ngrp), BS, 0, s>>>(tab, ngrp, first, w, cblk, cidx_, Ucorr, stride, ph);
    return cudaGetLastError();
}

}  // namespace hamr
